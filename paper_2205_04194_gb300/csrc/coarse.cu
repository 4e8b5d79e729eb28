// Coarse space of the two-level Schwarz preconditioner.
//
// The paper leaves the solver's preconditioner to future work (Section 4) and
// names preconditioned iterations (Section 1, Beatson et al.).  The one-level
// additive Schwarz method of cg.cu solves on leaf neighbourhood patches; on
// flat shapes (c several times the point spacing) it stalls, because the
// smooth error components couple all patches.  The second level adds a
// Galerkin coarse space:
//
//   Z   : one indicator vector per coarse box, the largest tree boxes holding
//         at most cp points (disjoint Morton ranges that cover every point; on a
//         batched plan each problem's own boxes, so E is block diagonal);
//   E   = Z^T A Z, E_ab = sum_{i in a} sum_{j in b} 1 / sqrt(|x_i - x_j|^2 + c^2);
//   Q   = Z E^{-1} Z^T.
//
// E is assembled exactly (every pair: in FP64 up to N^2 = 4e10, beyond that FP32
// kernel values with FP32 partial sums over 32 sources folded into FP64), factored and inverted once in FP64
// (cuSOLVER potrf / potri, a small relative diagonal shift when rounding makes
// it indefinite), and applied as a dense FP64 mat-vec.  cg.cu combines it with
// the patch solves M1 in the deflated form z = y + Q (r - A y), y = M1 r, with
// the inner iterations started from Q r.
#include <cusolverDn.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kGramThreads = 256;
constexpr int kGramTPT = 4;   // targets per thread: coarse boxes up to 1024 points
constexpr double kGramFp64Pairs = 4e10;   // largest N^2 whose Galerkin matrix is assembled in FP64

// E[a][b] = sum over targets of box a (this block) and sources of box b.  Block a
// holds its targets in registers (4 per thread, offsets from the box centre);
// the sources of each box b are staged in shared memory as offsets from b's
// centre shifted by the centre difference, and read back as broadcasts.  The
// warps' totals for 32 boxes b at a time are summed in warp order
// (deterministic).  T = float: FP32 kernel values (rsqrtf), partials over 32
// sources folded into FP64.  T = double: every pair in FP64 (for problems whose
// N^2 the FP64 units finish quickly; the coarse correction amplifies any error
// of E by the patch solves' norm).
// On a batched plan (cprob != nullptr) each coarse box belongs to one problem: pairs of
// different problems are zero (A is block diagonal) and a problem's pairs use its own c.
template <class T>
__global__ void __launch_bounds__(kGramThreads) k_coarse_gram(int nc, const int32_t *__restrict__ cbeg,
                                                               const double2 *__restrict__ ccen,
                                                               const double2 *__restrict__ pos, double c,
                                                               const int32_t *__restrict__ cprob,
                                                               const double *__restrict__ prob_c,
                                                               double *__restrict__ E) {
    __shared__ T srcx[kGramThreads * kGramTPT], srcy[kGramThreads * kGramTPT];
    __shared__ double sh[kGramThreads / 32][32];
    const int a = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int a0 = cbeg[a], na = cbeg[a + 1] - a0;
    const double2 ca = ccen[a];
    T xt[kGramTPT], yt[kGramTPT];
    int nt = 0;
#pragma unroll
    for (int k = 0; k < kGramTPT; ++k) {
        const int i = threadIdx.x + kGramThreads * k;
        xt[k] = 0;
        yt[k] = 0;
        if (i < na) {
            const double2 q = pos[a0 + i];
            xt[k] = (T)(q.x - ca.x);
            yt[k] = (T)(q.y - ca.y);
            nt = k + 1;
        }
    }
    const double ca_c = cprob ? prob_c[cprob[a]] : c;
    const T c2 = (T)(ca_c * ca_c);
    for (int b = 0; b < nc; ++b) {
        const bool same = !cprob || cprob[b] == cprob[a];   // uniform over the block
        const int b0 = cbeg[b], nb = same ? cbeg[b + 1] - b0 : 0;
        const double2 cb = ccen[b];
        const T dx0 = (T)(ca.x - cb.x), dy0 = (T)(ca.y - cb.y);
        __syncthreads();   // the previous box's sources are no longer read
        for (int j = threadIdx.x; j < nb; j += kGramThreads) {
            const double2 q = pos[b0 + j];
            srcx[j] = (T)(q.x - cb.x) - dx0;
            srcy[j] = (T)(q.y - cb.y) - dy0;
        }
        __syncthreads();
        double tot = 0.0;
        for (int j0 = 0; j0 < nb; j0 += 32) {
            const int jn = min(32, nb - j0);
            T part = 0;
            for (int j = 0; j < jn; ++j) {
                const T qx = srcx[j0 + j], qy = srcy[j0 + j];
#pragma unroll
                for (int k = 0; k < kGramTPT; ++k) {
                    if (k < nt) {
                        const T dx = xt[k] - qx, dy = yt[k] - qy;
                        if constexpr (sizeof(T) == 4) part += rsqrtf(fmaf(dx, dx, fmaf(dy, dy, c2)));
                        else part += 1.0 / sqrt(fma(dx, dx, fma(dy, dy, c2)));
                    }
                }
            }
            tot += (double)part;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) tot += __shfl_xor_sync(0xFFFFFFFFu, tot, off);
        if (lane == 0) sh[w][b & 31] = tot;
        if ((b & 31) == 31 || b == nc - 1) {
            __syncthreads();
            if (threadIdx.x <= (b & 31)) {
                double e = 0.0;
                for (int k = 0; k < kGramThreads / 32; ++k) e += sh[k][threadIdx.x];
                E[(size_t)a * nc + (b & ~31) + threadIdx.x] = e;
            }
        }
    }
}

// E = (E + E^T) / 2 (the two halves are separate sums of the same pairs)
__global__ void k_symmetrize(double *__restrict__ E, int n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
    if (j >= i) return;
    const double v = 0.5 * (E[(size_t)i * n + j] + E[(size_t)j * n + i]);
    E[(size_t)i * n + j] = v;
    E[(size_t)j * n + i] = v;
}

// copy the lower triangle (column-major) of a factored inverse to the upper one
__global__ void k_lower_to_full(double *__restrict__ E, int n) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n * n) return;
    const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);   // column j, row i
    if (i < j) E[(size_t)j * n + i] = E[(size_t)i * n + j];
}

__global__ void k_add_diag(double *__restrict__ E, int n, double d) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[(size_t)i * n + i] += d;
}

__device__ __forceinline__ double block_sum_d(double v, double *sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
    return t;
}

// g[a] = sum_{i in box a} (r_i - b_i), b FP32 (b32) or FP64 (b64) or absent; fixed order (deterministic)
__global__ void __launch_bounds__(256) k_coarse_restrict(const int32_t *__restrict__ cbeg,
                                                         const double *__restrict__ r, const float *__restrict__ b32,
                                                         const double *__restrict__ b64, double *__restrict__ g,
                                                         const int *done) {
    __shared__ double sh[8];
    if (done && *done) return;
    const int a = blockIdx.x;
    const int lo = cbeg[a], hi = cbeg[a + 1];
    double acc = 0.0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x)
        acc += b32 ? r[i] - (double)b32[i] : (b64 ? r[i] - b64[i] : r[i]);
    const double t = block_sum_d(acc, sh);
    if (threadIdx.x == 0) g[a] = t;
}

// cc = E^{-1} g: one warp per row, lanes over the columns (coalesced), fixed-order reduction
__global__ void __launch_bounds__(256) k_coarse_gemv(int nc, const double *__restrict__ einv,
                                                     const double *__restrict__ g, double *__restrict__ cc,
                                                     const int *done) {
    if (done && *done) return;
    const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (row >= nc) return;
    const double *er = einv + (size_t)row * nc;
    double acc = 0.0;
    for (int j = lane; j < nc; j += 32) acc = fma(er[j], g[j], acc);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, off);
    if (lane == 0) cc[row] = acc;
}

// z_i = y_i + cc[a] for i in box a (y may be null)
__global__ void __launch_bounds__(256) k_coarse_prolong(const int32_t *__restrict__ cbeg,
                                                        const double *__restrict__ cc, const double *__restrict__ y,
                                                        double *__restrict__ z, const int *done) {
    if (done && *done) return;
    const int a = blockIdx.x;
    const double v = cc[a];
    for (int i = cbeg[a] + threadIdx.x; i < cbeg[a + 1]; i += blockDim.x) z[i] = y ? y[i] + v : v;
}

void cusolver_check(cusolverStatus_t st, const char *what) {
    if (st != CUSOLVER_STATUS_SUCCESS)
        fail(IMQ_CUDA_ERROR, std::string("two-level Schwarz: ") + what + " failed (cusolver status " +
                                 std::to_string((int)st) + ")");
}

}  // namespace

void coarse_setup(Plan &P, int cp, int gram, cudaStream_t s) {
    Coarse &C = P.coarse;
    if (C.ready && C.cp == cp && C.gram_mode == gram) return;
    if (cp < 1 || cp > kGramThreads * kGramTPT)
        fail(IMQ_INVALID_ARG, "two-level Schwarz: coarse_points must be in [1, 1024]");
    // ---- coarse boxes: the largest boxes holding at most cp points, in Morton order
    const int nb = P.nbox;
    const bool batched = P.nprob > 1;
    std::vector<int32_t> beg(nb), en(nb), ch(4 * (size_t)nb), par(nb), bprob(batched ? nb : 0);
    std::vector<double2> cen(nb);
    IMQ_CUDA(cudaMemcpyAsync(par.data(), P.parent.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    if (batched)
        IMQ_CUDA(cudaMemcpyAsync(bprob.data(), P.box_prob.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(beg.data(), P.begin.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(en.data(), P.end.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(ch.data(), P.child.ptr, sizeof(int32_t) * 4 * (size_t)nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(cen.data(), P.centre.ptr, sizeof(double2) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> cb{0}, cpr;
    std::vector<double2> cc;
    // one root per problem (box order = problem order), each walked in Morton order
    std::vector<int> stack;
    for (int b = nb - 1; b >= 0; --b)
        if (par[b] < 0) stack.push_back(b);
    while (!stack.empty()) {
        const int b = stack.back();
        stack.pop_back();
        const int cnt = en[b] - beg[b];
        const bool leaf = ch[4 * (size_t)b] < 0 && ch[4 * (size_t)b + 1] < 0 && ch[4 * (size_t)b + 2] < 0 &&
                          ch[4 * (size_t)b + 3] < 0;
        if (cnt == 0) continue;
        if (cnt <= cp || leaf) {
            if (cnt > kGramThreads * kGramTPT)
                fail(IMQ_UNSUPPORTED, "two-level Schwarz: a leaf holds more than 1024 points");
            if (beg[b] != cb.back()) fail(IMQ_CUDA_ERROR, "two-level Schwarz: coarse boxes are not contiguous");
            cb.push_back(en[b]);
            cc.push_back(cen[b]);
            cpr.push_back(batched ? bprob[b] : 0);
            continue;
        }
        for (int q = 3; q >= 0; --q)   // children in Morton order
            if (ch[4 * (size_t)b + q] >= 0) stack.push_back(ch[4 * (size_t)b + q]);
    }
    if (cb.back() != P.N) fail(IMQ_CUDA_ERROR, "two-level Schwarz: coarse boxes do not cover the points");
    const int nc = (int)cc.size();
    if (nc > kCoarseMax)
        fail(IMQ_INVALID_ARG, "two-level Schwarz: " + std::to_string(nc) + " coarse boxes exceed " +
                                  std::to_string(kCoarseMax) + "; raise coarse_points");
    C.cbeg.alloc(sizeof(int32_t) * (nc + 1));
    IMQ_CUDA(cudaMemcpyAsync(C.cbeg.ptr, cb.data(), sizeof(int32_t) * (nc + 1), cudaMemcpyHostToDevice, s));
    AsyncMem dcen(sizeof(double2) * nc, s), E(sizeof(double) * (size_t)nc * nc, s), dcpr(sizeof(int32_t) * nc, s);
    IMQ_CUDA(cudaMemcpyAsync(dcen.ptr, cc.data(), sizeof(double2) * nc, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyAsync(dcpr.ptr, cpr.data(), sizeof(int32_t) * nc, cudaMemcpyHostToDevice, s));
    const int32_t *cprob = batched ? dcpr.as<int32_t>() : nullptr;
    const double *pc = batched ? P.prob_c.as<double>() : nullptr;
    // ---- Galerkin matrix, every pair
    // FP64 pairs while N^2 stays within about a second of the FP64 units, FP32 pairs beyond
    C.gram_fp64 = gram == 1 || (gram == 0 && (double)P.N * (double)P.N <= kGramFp64Pairs);
    if (C.gram_fp64)
        k_coarse_gram<double><<<nc, kGramThreads, 0, s>>>(nc, C.cbeg.as<int32_t>(), dcen.as<double2>(),
                                                          P.pos.as<double2>(), P.c, cprob, pc, E.as<double>());
    else
        k_coarse_gram<float><<<nc, kGramThreads, 0, s>>>(nc, C.cbeg.as<int32_t>(), dcen.as<double2>(),
                                                         P.pos.as<double2>(), P.c, cprob, pc, E.as<double>());
    IMQ_LAUNCH_CHECK();
    const unsigned gq = blocks_for((int64_t)nc * nc, 256);
    k_symmetrize<<<gq, 256, 0, s>>>(E.as<double>(), nc);
    IMQ_LAUNCH_CHECK();
    std::vector<double> diag(nc);
    IMQ_CUDA(cudaMemcpy2DAsync(diag.data(), sizeof(double), E.ptr, sizeof(double) * (nc + 1), sizeof(double), nc,
                               cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    double mdiag = 0;
    for (double d : diag) mdiag += d / nc;
    // ---- E^{-1} in FP64: Cholesky, then the inverse from the factor; if rounding makes E
    // indefinite, a small diagonal shift relative to its mean diagonal
    cusolverDnHandle_t h = nullptr;
    cusolver_check(cusolverDnCreate(&h), "cusolverDnCreate");
    struct HandleGuard {
        cusolverDnHandle_t h;
        ~HandleGuard() { cusolverDnDestroy(h); }
    } hg{h};
    cusolver_check(cusolverDnSetStream(h, s), "cusolverDnSetStream");
    C.einv.alloc(sizeof(double) * (size_t)nc * nc);
    double *A = C.einv.as<double>();
    int lw1 = 0, lw2 = 0;
    cusolver_check(cusolverDnDpotrf_bufferSize(h, CUBLAS_FILL_MODE_LOWER, nc, A, nc, &lw1), "potrf_bufferSize");
    cusolver_check(cusolverDnDpotri_bufferSize(h, CUBLAS_FILL_MODE_LOWER, nc, A, nc, &lw2), "potri_bufferSize");
    AsyncMem work(sizeof(double) * (size_t)std::max(1, std::max(lw1, lw2)), s), info(sizeof(int), s);
    bool done = false;
    for (double rel : {0.0, 1e-14, 1e-12, 1e-10, 1e-8, 1e-6}) {
        IMQ_CUDA(cudaMemcpyAsync(A, E.ptr, sizeof(double) * (size_t)nc * nc, cudaMemcpyDeviceToDevice, s));
        if (rel > 0) {
            k_add_diag<<<blocks_for(nc, 256), 256, 0, s>>>(A, nc, rel * mdiag);
            IMQ_LAUNCH_CHECK();
        }
        cusolver_check(cusolverDnDpotrf(h, CUBLAS_FILL_MODE_LOWER, nc, A, nc, work.as<double>(), lw1,
                                        info.as<int>()),
                       "potrf");
        int hinfo = 0;
        IMQ_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        if (hinfo != 0) continue;
        cusolver_check(cusolverDnDpotri(h, CUBLAS_FILL_MODE_LOWER, nc, A, nc, work.as<double>(), lw2,
                                        info.as<int>()),
                       "potri");
        IMQ_CUDA(cudaMemcpyAsync(&hinfo, info.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        if (hinfo != 0) continue;
        C.shift = rel;
        done = true;
        break;
    }
    if (!done) fail(IMQ_NUMERICAL, "two-level Schwarz: the coarse matrix could not be factored");
    k_lower_to_full<<<gq, 256, 0, s>>>(A, nc);
    IMQ_LAUNCH_CHECK();
    C.g.alloc(sizeof(double) * nc);
    C.cc.alloc(sizeof(double) * nc);
    IMQ_CUDA(cudaStreamSynchronize(s));
    C.nc = nc;
    C.cp = cp;
    C.gram_mode = gram;
    C.ready = true;
}

void coarse_restrict(const Plan &P, const double *r, const float *b32, const double *b64, const int *done,
                     cudaStream_t s) {
    const Coarse &C = P.coarse;
    k_coarse_restrict<<<C.nc, 256, 0, s>>>(C.cbeg.as<int32_t>(), r, b32, b64, C.g.as<double>(), done);
    IMQ_LAUNCH_CHECK();
}

void coarse_solve(const Plan &P, const int *done, cudaStream_t s) {
    const Coarse &C = P.coarse;
    k_coarse_gemv<<<blocks_for((int64_t)C.nc * 32, 256), 256, 0, s>>>(C.nc, C.einv.as<double>(), C.g.as<double>(),
                                                                      C.cc.as<double>(), done);
    IMQ_LAUNCH_CHECK();
}

void coarse_prolong(const Plan &P, const double *y, double *z, const int *done, cudaStream_t s) {
    const Coarse &C = P.coarse;
    k_coarse_prolong<<<C.nc, 256, 0, s>>>(C.cbeg.as<int32_t>(), C.cc.as<double>(), y, z, done);
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq
