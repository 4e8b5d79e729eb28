// Iterative solve of the interpolation system A coef = f (paper Section 2,
// Eq. (3)-(4)).  The paper names iterative methods as the practical solver
// whose cost is dominated by the matrix-vector product (Section 2) and leaves
// their use with the fast product, and a preconditioner, to future work
// (Section 4).  Built here:
//
//  * preconditioned conjugate gradients (A is symmetric positive definite for
//    distinct points) with the FP32 fast product as the operator and FP64
//    vectors, dots and scalars; all vectors stay in Morton order so an
//    iteration has no gather or scatter;
//  * deterministic reductions: fixed grid, fixed per-block tree, fixed-order
//    second stage, so a solve is bit-reproducible;
//  * iterations captured into a CUDA graph (kIterPerGraph at a time) with the
//    convergence test on the device: once the residual test passes, the
//    remaining captured iterations skip their vector updates; the host reads
//    the state once per graph launch;
//  * symmetric additive Schwarz preconditioner z = sum_b R_b^T (A_b + d I)^{-1} R_b r
//    over patches made of a leaf and its nearest adjacent leaves (whole leaves,
//    nearest centre first, up to nmax points); each patch matrix is factored
//    once in FP32 (Cholesky in shared memory) and applied by one warp with
//    forward/backward substitution; overlapping patch results are summed per
//    point in a fixed order;
//  * outer iterative refinement: r = f - A x with an FP64 product (the plan in
//    FP64, or the dense FP64 product), inner PCG on A d = r, x += d.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kRedBlocks = 608;
constexpr int kRedThreads = 256;
constexpr int kIterPerGraph = 8;

// kBreakdown: a finite p.q <= 0 or r.z <= 0.  A is positive definite, but the
// FP32 product and the shifted patch factors are not exactly so when A is
// nearly singular; the pass then ends and the host restarts from the true
// residual of the best iterate.  kNumerical is reserved for NaN / Inf.
enum CGState : int { kRunning = 0, kConverged = 1, kNumerical = 2, kMaxIter = 3, kBreakdown = 4 };
constexpr int kMaxRestarts = 16;   // restarts after a breakdown when no refinement steps are requested
constexpr double kF32PatchShift = 1e-6;   // least diagonal shift of FP32 Schwarz patches, relative to 1/c

struct CGScalars {
    double rz, rz_new, pq, rr, alpha, beta, rr_target, rr_best, rr0;
    int iter, done, status, maxit, improved, pad;
};

__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = kRedThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    return sh[0];
}

__device__ __forceinline__ double final_sum(const double *part) {
    __shared__ double sh[kRedThreads];
    double v = 0;
    for (int i = threadIdx.x; i < kRedBlocks; i += kRedThreads) v += part[i];
    return block_sum(v, sh);
}

__global__ void __launch_bounds__(kRedThreads) k_p_to_f32(const double *__restrict__ p, float *__restrict__ u,
                                                          int64_t n, const CGScalars *S) {
    if (S && S->done) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = (float)p[i];
}

// q = (double) b and per-block partial of p.q
__global__ void __launch_bounds__(kRedThreads) k_q_dot(const float *__restrict__ b, const double *__restrict__ p,
                                                       double *__restrict__ q, int64_t n, double *__restrict__ part,
                                                       const CGScalars *S) {
    __shared__ double sh[kRedThreads];
    if (S->done) return;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double qi = (double)b[i];
        q[i] = qi;
        acc += p[i] * qi;
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads) k_finish_alpha(const double *__restrict__ part, CGScalars *S) {
    if (S->done) return;
    const double pq = final_sum(part);
    if (threadIdx.x == 0) {
        S->pq = pq;
        if (!isfinite(pq)) {
            S->status = kNumerical;
            S->done = 1;
        } else if (!(pq > 0)) {
            S->status = kBreakdown;
            S->done = 1;
        } else {
            S->alpha = S->rz / pq;
        }
    }
}

__global__ void __launch_bounds__(kRedThreads) k_update_xr(double *__restrict__ x, double *__restrict__ r,
                                                           const double *__restrict__ p, const double *__restrict__ q,
                                                           int64_t n, double *__restrict__ part, const CGScalars *S) {
    __shared__ double sh[kRedThreads];
    if (S->done) return;
    const double a = S->alpha;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads) k_finish_rr(const double *__restrict__ part, CGScalars *S) {
    if (S->done) return;
    const double rr = final_sum(part);
    if (threadIdx.x == 0) {
        S->rr = rr;
        S->iter += 1;
        S->improved = 0;
        if (!isfinite(rr)) {
            S->status = kNumerical;
            S->done = 1;
        } else {
            if (rr < S->rr_best) {
                S->rr_best = rr;
                S->improved = 1;
            }
            if (rr <= S->rr_target) {
                S->status = kConverged;
                S->done = 1;
            } else if (S->iter >= S->maxit) {
                S->status = kMaxIter;
                S->done = 1;
            }
        }
    }
}

// keep the iterate with the smallest recursive residual
__global__ void k_copy_best(const double *__restrict__ x, double *__restrict__ xb, int64_t n, const CGScalars *S) {
    if (!S->improved) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        xb[i] = x[i];
}

__global__ void __launch_bounds__(kRedThreads) k_dot_part(const double *__restrict__ a, const double *__restrict__ b,
                                                          int64_t n, double *__restrict__ part, const CGScalars *S) {
    __shared__ double sh[kRedThreads];
    if (S && S->done) return;
    double acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += a[i] * b[i];
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kRedThreads) k_finish_beta(const double *__restrict__ part, CGScalars *S,
                                                             int use_rr) {
    if (S->done) return;
    const double rzn = use_rr ? S->rr : final_sum(part);
    if (threadIdx.x == 0) {
        S->rz_new = rzn;
        if (!isfinite(rzn)) {
            S->status = kNumerical;
            S->done = 1;
        } else if (!(rzn > 0)) {
            S->status = kBreakdown;
            S->done = 1;
        } else {
            S->beta = rzn / S->rz;
        }
    }
}

// p = z + beta p; also u = (float) p, the next product's input (u may be null), and
// rz = rz_new (one thread; the other blocks read only beta)
__global__ void k_update_p(double *__restrict__ p, const double *__restrict__ z, float *__restrict__ u, int64_t n,
                           CGScalars *S) {
    if (S->done) return;
    const double bt = S->beta;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double pi = z[i] + bt * p[i];
        p[i] = pi;
        if (u) u[i] = (float)pi;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) S->rz = S->rz_new;
}

__global__ void __launch_bounds__(kRedThreads) k_sum_to(const double *__restrict__ part, double *out) {
    const double v = final_sum(part);
    if (threadIdx.x == 0) *out = v;
}

__global__ void k_axpby(double *__restrict__ y, const double *__restrict__ x, double a, double b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = a * x[i] + b * y[i];
}

// r -= (double) b
__global__ void k_sub_f32(double *__restrict__ r, const float *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] -= (double)b[i];
}

// r -= b
__global__ void k_sub_f64(double *__restrict__ r, const double *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] -= b[i];
}

// ---- GMRES (Arnoldi) helpers: V holds nv vectors of length n, one after another
// part[i][block] = this block's partial of V_i . w (fixed order within the block)
__global__ void __launch_bounds__(kRedThreads) k_multi_dot_part(const double *__restrict__ V, int64_t n, int nv,
                                                                const double *__restrict__ w,
                                                                double *__restrict__ part) {
    __shared__ double sh[kRedThreads];
    for (int i = 0; i < nv; ++i) {
        const double *vi = V + (size_t)i * n;
        double acc = 0;
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
            acc += vi[k] * w[k];
        const double t = block_sum(acc, sh);
        if (threadIdx.x == 0) part[(size_t)i * kRedBlocks + blockIdx.x] = t;
        __syncthreads();   // sh is reused by the next vector
    }
}
// h[i] = sum over blocks of part[i][*] (one block per vector, fixed order)
__global__ void __launch_bounds__(kRedThreads) k_multi_sum(const double *__restrict__ part, double *__restrict__ h) {
    const double v = final_sum(part + (size_t)blockIdx.x * kRedBlocks);
    if (threadIdx.x == 0) h[blockIdx.x] = v;
}
// w -= sum_i h[i] V_i
__global__ void __launch_bounds__(kRedThreads) k_multi_axpy(const double *__restrict__ V, int64_t n, int nv,
                                                            const double *__restrict__ h, double *__restrict__ w) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0;
        for (int i = 0; i < nv; ++i) acc += h[i] * V[(size_t)i * n + k];
        w[k] -= acc;
    }
}
// u = sum_i y[i] V_i
__global__ void __launch_bounds__(kRedThreads) k_lincomb(const double *__restrict__ V, int64_t n, int nv,
                                                         const double *__restrict__ y, double *__restrict__ u) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0;
        for (int i = 0; i < nv; ++i) acc += y[i] * V[(size_t)i * n + k];
        u[k] = acc;
    }
}
__global__ void k_scale_to(const double *__restrict__ w, double a, double *__restrict__ v, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) v[i] = a * w[i];
}
__global__ void k_f32_to_f64(const float *__restrict__ b, double *__restrict__ q, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) q[i] = (double)b[i];
}

__global__ void k_sub(double *__restrict__ r, const double *__restrict__ f, const double *__restrict__ ax, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = f[i] - ax[i];
}

__global__ void k_gather_f64(const double *__restrict__ v, const int32_t *__restrict__ perm, int64_t n,
                             double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = v[perm[i]];
}

__global__ void k_scatter_f64(const double *__restrict__ v, const int32_t *__restrict__ perm, int64_t n,
                              double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = v[i];
}

// ------------------------------------------------------------------ Schwarz preconditioner
// Factor one patch: A_b + shift*I assembled in FP32 from FP64 coordinate
// differences, right-looking Cholesky in shared memory; pivots below
// dmin are raised to dmin (the patch matrices of flat shapes are numerically
// singular).  Output (INV = false): the n x n column-major lower factor L.
// INV = true: the inverse factor L^{-1} (column-major, lower), so that the
// apply z = L^{-T} (L^{-1} r) is two dense triangular matrix-vector products
// per patch (bandwidth-bound) instead of two sequential triangular solves
// (latency-bound), and r.z = |L^{-1} r|^2 stays positive in FP32 (an explicit
// FP32 inverse L^{-T} L^{-1} of an ill-conditioned patch need not be).  L^{-1}
// replaces L in shared memory column by column (last column first), with one
// extra column of n values.
// Packed lower-triangular storage of an n x n inverse factor X = L^{-1}: column j holds
// rows j .. n-1 contiguously from inv_packed_col(j, n); a patch's block is padded to a
// multiple of four floats, so every block starts on a 16-byte boundary (one bulk copy).
__host__ __device__ __forceinline__ int inv_packed_col(int j, int n) { return j * (2 * n - j + 1) / 2; }
__host__ __device__ __forceinline__ int inv_packed_size(int n) { return (n * (n + 1) / 2 + 3) & ~3; }

template <class T, bool INV>
__global__ void k_schwarz_factor(int npatch, const int32_t *__restrict__ poff, const int32_t *__restrict__ ppts,
                                 const int64_t *__restrict__ foff, const double2 *__restrict__ pos,
                                 const int32_t *__restrict__ leaves, ShapeC shape, double shift_rel,
                                 double dmin_rel, T *__restrict__ factor, int *nclamped) {
    extern __shared__ __align__(16) unsigned char smraw_f[];
    T *A = reinterpret_cast<T *>(smraw_f);   // n x n, column-major
    __shared__ int s_bad;
    const int b = blockIdx.x;
    if (b >= npatch) return;
    const int o = poff[b], n = poff[b + 1] - o;
    const double cb = shape.of(leaves[b]);
    const T c2 = (T)(cb * cb), shift = (T)(shift_rel / cb);
    T *F = factor + foff[b];
    // INV: an inverse factor that overflows (pivots at the clamp, L^{-1} growing beyond the
    // FP32 range) is recomputed with the clamp raised 1000-fold, up to three times
    for (int attempt = 0; attempt < (INV ? 4 : 1); ++attempt) {
        const T dmin = (T)(dmin_rel / cb * pow(1e3, (double)attempt));
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int j = e / n, i = e - j * n;   // column j, row i
            const double2 pi = pos[ppts[o + i]], pj = pos[ppts[o + j]];
            const T dx = (T)(pi.x - pj.x), dy = (T)(pi.y - pj.y);
            T a = (T)1 / sqrt(dx * dx + dy * dy + c2);
            if (i == j) a += shift;
            A[e] = a;
        }
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();
        for (int k = 0; k < n; ++k) {
            if (threadIdx.x == 0) {
                T d = A[k * n + k];
                if (!(d > dmin)) {
                    d = dmin;
                    if (attempt == 0) atomicAdd(nclamped, 1);
                }
                A[k * n + k] = sqrt(d);
            }
            __syncthreads();
            const T piv = A[k * n + k];
            for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[k * n + i] /= piv;
            __syncthreads();
            const int m = n - k - 1;
            for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
                const int jj = e / m, ii = e - jj * m;
                const int j = k + 1 + jj, i = k + 1 + ii;
                if (i >= j) A[j * n + i] -= A[k * n + i] * A[k * n + j];
            }
            __syncthreads();
        }
        if constexpr (!INV) {
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                const int j = e / n, i = e - j * n;
                F[e] = i >= j ? A[e] : (T)0;
            }
            return;
        } else {
            // L^{-1} in place, column j from the last to the first: X[i][j] = -(sum_{j < k <= i}
            // X[i][k] L[k][j]) / L[j][j] for i > j, X[j][j] = 1 / L[j][j]; column j of L is copied
            // to tmp first because the new column overwrites it
            T *tmp = A + (size_t)n * n;
            for (int jc = n - 1; jc >= 0; --jc) {
                for (int k = jc + 1 + threadIdx.x; k < n; k += blockDim.x) tmp[k] = A[(size_t)jc * n + k];
                __syncthreads();
                const T d = (T)1 / A[(size_t)jc * n + jc];
                for (int i = jc + 1 + threadIdx.x; i < n; i += blockDim.x) {
                    T sum = 0;
                    for (int k = jc + 1; k <= i; ++k) sum += A[(size_t)k * n + i] * tmp[k];
                    const T x = -sum * d;
                    if (!isfinite(x)) s_bad = 1;
                    A[(size_t)jc * n + i] = x;
                }
                if (threadIdx.x == 0) {
                    A[(size_t)jc * n + jc] = d;
                    if (!isfinite(d)) s_bad = 1;
                }
                __syncthreads();
            }
            if (s_bad) continue;
            for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
                const int t = e / n, i = e - t * n;
                if (i >= t) F[inv_packed_col(t, n) + (i - t)] = A[e];
            }
            for (int e = n * (n + 1) / 2 + threadIdx.x; e < inv_packed_size(n); e += blockDim.x) F[e] = (T)0;
            __syncthreads();
            if (!s_bad) return;
        }
    }
    // every attempt overflowed: the patch acts as the diagonal c I (as a point in no patch)
    if constexpr (INV) {
        for (int e = threadIdx.x; e < inv_packed_size(n); e += blockDim.x) F[e] = (T)0;
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) F[inv_packed_col(j, n)] = (T)sqrt(cb);
    }
}

// One warp per patch: y = (L L^T)^{-1} r_patch by forward and backward substitution.
constexpr int kSchwarzRowsPerLane = 8;   // patches up to 256 points
template <class T>
__global__ void k_schwarz_solve(int npatch, const int32_t *__restrict__ poff, const int32_t *__restrict__ ppts,
                                const int64_t *__restrict__ foff, const T *__restrict__ factor,
                                const double *__restrict__ r, double *__restrict__ ypatch, const CGScalars *S) {
    if (S && S->done) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= npatch) return;
    const int o = poff[warp], n = poff[warp + 1] - o;
    const T *F = factor + foff[warp];
    T v[kSchwarzRowsPerLane];
#pragma unroll
    for (int t = 0; t < kSchwarzRowsPerLane; ++t) {
        const int i = lane + 32 * t;
        v[t] = i < n ? (T)r[ppts[o + i]] : (T)0;
    }
    // forward: L y = r
    for (int k = 0; k < n; ++k) {
        const int owner = k & 31, tk = k >> 5;
        T val = 0;
#pragma unroll
        for (int t = 0; t < kSchwarzRowsPerLane; ++t)
            if (t == tk) val = v[t];
        const T yk = __shfl_sync(0xFFFFFFFFu, val / F[(size_t)k * n + k], owner);
#pragma unroll
        for (int t = 0; t < kSchwarzRowsPerLane; ++t) {
            const int i = lane + 32 * t;
            if (i == k) v[t] = yk;
            else if (i > k && i < n) v[t] -= F[(size_t)k * n + i] * yk;
        }
    }
    // backward: L^T z = y
    for (int k = n - 1; k >= 0; --k) {
        T part = 0;
#pragma unroll
        for (int t = 0; t < kSchwarzRowsPerLane; ++t) {
            const int i = lane + 32 * t;
            if (i > k && i < n) part += F[(size_t)k * n + i] * v[t];
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, off);
        const int owner = k & 31, tk = k >> 5;
#pragma unroll
        for (int t = 0; t < kSchwarzRowsPerLane; ++t)
            if (t == tk && lane == owner) v[t] = (v[t] - part) / F[(size_t)k * n + k];
    }
#pragma unroll
    for (int t = 0; t < kSchwarzRowsPerLane; ++t) {
        const int i = lane + 32 * t;
        if (i < n) ypatch[o + i] = (double)v[t];
    }
}

// One CTA per patch: y = L^{-T} (L^{-1} r_patch) with the FP32 inverse factor X = L^{-1}
// (packed lower, n <= 32 * kInvRowsPerLane).  The patch's X arrives in shared memory by one
// bulk copy, so each factor byte crosses HBM once per apply; the two triangular products
// then run from shared memory.  Pass 1, w_i = sum_{j <= i} X_ij r_j: a thread per row,
// consecutive threads on consecutive rows of a column.  Pass 2, y_k = sum_{i >= k} X_ik w_i:
// a thread per column, reading it contiguously.  256 threads (every row of a 224-point patch
// has its own thread) and about 100 KB of shared memory: two CTAs per SM, one computing while
// the other's copy lands.
constexpr int kInvRowsPerLane = 7;   // patches up to 224 points
constexpr int kInvThreads = 256;

size_t inv_apply_smem(int maxn) { return sizeof(float) * ((size_t)inv_packed_size(maxn) + 2 * (size_t)maxn); }

__global__ void __launch_bounds__(kInvThreads) k_schwarz_inv_apply(int npatch, const int32_t *__restrict__ poff,
                                                                  const int32_t *__restrict__ ppts,
                                                                  const int64_t *__restrict__ foff,
                                                                  const float *__restrict__ inv,
                                                                  const double *__restrict__ r,
                                                                  double *__restrict__ ypatch, const CGScalars *S,
                                                                  int *err) {
    extern __shared__ __align__(16) unsigned char smraw_i[];
    __shared__ __align__(8) uint64_t bar;
    if (S && S->done) return;
    const int b = blockIdx.x;
    if (b >= npatch) return;
    const int o = poff[b], n = poff[b + 1] - o, np = inv_packed_size(n);
    float *X = reinterpret_cast<float *>(smraw_i);
    float *rv = X + np, *wv = rv + n;
    if (n == 0) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)(sizeof(float) * np));
        bulk_g2s(X, inv + foff[b], (uint32_t)(sizeof(float) * np), &bar);
    }
    for (int i = threadIdx.x; i < n; i += kInvThreads) rv[i] = (float)r[ppts[o + i]];
    // a CTA-uniform outcome of the bounded wait, so that every thread leaves together
    if (!__syncthreads_and(mbar_wait(&bar, 0) ? 1 : 0)) {
        if (threadIdx.x == 0) set_error(err, kErrWaitTimeout);
        return;   // the results of this apply are invalid; the host reads the error word
    }
    for (int i = threadIdx.x; i < n; i += kInvThreads) {
        float acc = 0.f;
        int cj = i;   // packed index of X_ij for j = 0
        for (int j = 0; j <= i; ++j) {
            acc = fmaf(X[cj], rv[j], acc);
            cj += n - j - 1;
        }
        wv[i] = acc;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += kInvThreads) {
        const float *col = X + inv_packed_col(k, n);
        float acc = 0.f;
        for (int i = k; i < n; ++i) acc = fmaf(col[i - k], wv[i], acc);
        ypatch[o + k] = (double)acc;
    }
}

// z_j = sum over the patch slots holding point j (fixed order); points in no patch get c r_j.
__global__ void k_schwarz_gather(int64_t n, const int32_t *__restrict__ ptoff, const int32_t *__restrict__ ptslot,
                                 const double *__restrict__ ypatch, const double *__restrict__ r, double cdiag,
                                 const int32_t *__restrict__ pt_prob, const double *__restrict__ prob_c,
                                 double *__restrict__ z, const CGScalars *S) {
    if (S && S->done) return;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int a = ptoff[j], e = ptoff[j + 1];
        if (a == e) {
            z[j] = (pt_prob ? prob_c[pt_prob[j]] : cdiag) * r[j];
        } else {
            double s = 0;
            for (int k = a; k < e; ++k) s += ypatch[ptslot[k]];
            z[j] = s;
        }
    }
}

template <class T>
void upload_vec(DevMem &d, const std::vector<T> &h, cudaStream_t s) {
    d.alloc(sizeof(T) * std::max<size_t>(1, h.size()));
    if (!h.empty()) IMQ_CUDA(cudaMemcpyAsync(d.ptr, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s));
}

void build_schwarz(Plan &P, int nmax, double shift, bool fp64, cudaStream_t s) {
    Schwarz &Z = P.schwarz;
    if (Z.ready && Z.nmax == nmax && Z.shift == shift && Z.fp64 == fp64) return;
    const int nb = P.nbox;
    std::vector<int32_t> uoff(nb + 1), beg(nb), en(nb), leaves(P.nleaf);
    std::vector<double2> cen(nb);
    IMQ_CUDA(cudaMemcpyAsync(uoff.data(), P.U.off.ptr, sizeof(int32_t) * (nb + 1), cudaMemcpyDeviceToHost, s));
    std::vector<int32_t> uit(std::max<int64_t>(1, P.U.total));
    if (P.U.total)
        IMQ_CUDA(cudaMemcpyAsync(uit.data(), P.U.items.ptr, sizeof(int32_t) * P.U.total, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(beg.data(), P.begin.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(en.data(), P.end.ptr, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(cen.data(), P.centre.ptr, sizeof(double2) * nb, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(leaves.data(), P.leaves.ptr, sizeof(int32_t) * P.nleaf, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> poff{0}, ppts;
    std::vector<int64_t> foff;
    int64_t fsz = 0;
    int maxn = 0;
    for (int li = 0; li < P.nleaf; ++li) {
        const int b = leaves[li];
        std::vector<std::pair<double, int>> cand;
        for (int k = uoff[b]; k < uoff[b + 1]; ++k) {
            const int q = uit[k];
            const double dx = cen[q].x - cen[b].x, dy = cen[q].y - cen[b].y;
            cand.push_back({q == b ? -1.0 : dx * dx + dy * dy, q});
        }
        std::sort(cand.begin(), cand.end());
        int cnt = 0;
        for (auto &cq : cand) {
            const int q = cq.second, m = en[q] - beg[q];
            if (q != b && cnt + m > nmax) continue;
            for (int j = beg[q]; j < en[q] && cnt < nmax; ++j, ++cnt) ppts.push_back(j);
        }
        poff.push_back((int32_t)ppts.size());
        foff.push_back(fsz);
        fsz += (int64_t)cnt * cnt;
        maxn = std::max(maxn, cnt);
    }
    Z.npatch = P.nleaf;
    Z.total_slots = (int64_t)ppts.size();
    // FP32 patches of at most 32 * kInvRowsPerLane points are applied through their inverse
    // factor, stored packed (lower triangle only)
    Z.inverse = !fp64 && maxn <= 32 * kInvRowsPerLane;
    if (Z.inverse) {
        fsz = 0;
        for (int b = 0; b < P.nleaf; ++b) {
            foff[b] = fsz;
            fsz += inv_packed_size(poff[b + 1] - poff[b]);
        }
    }
    Z.maxn = maxn;
    // reverse map point -> slots, in increasing slot order (deterministic sums)
    std::vector<int32_t> ptcnt(P.N + 1, 0);
    for (auto j : ppts) ptcnt[j + 1]++;
    for (int64_t j = 0; j < P.N; ++j) ptcnt[j + 1] += ptcnt[j];
    std::vector<int32_t> ptslot(ppts.size()), cur(ptcnt.begin(), ptcnt.end() - 1);
    for (size_t sl = 0; sl < ppts.size(); ++sl) ptslot[cur[ppts[sl]]++] = (int32_t)sl;
    upload_vec(Z.patch_off, poff, s);
    upload_vec(Z.patch_pts, ppts, s);
    upload_vec(Z.fac_off, foff, s);
    upload_vec(Z.pt_off, ptcnt, s);
    upload_vec(Z.pt_slot, ptslot, s);
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    Z.factor.alloc(es * std::max<int64_t>(1, fsz));
    Z.ypatch.alloc(sizeof(double) * std::max<int64_t>(1, Z.total_slots));
    AsyncMem ncl(sizeof(int), s);
    IMQ_CUDA(cudaMemsetAsync(ncl.ptr, 0, sizeof(int), s));
    // FP32 patches get a diagonal shift of at least kF32PatchShift / c: a patch matrix that FP32
    // cannot hold as positive definite otherwise meets clamped pivots whose Schur updates grow
    // without bound
    const double fshift = fp64 ? shift : std::max(shift, kF32PatchShift);
    const size_t smem = es * ((size_t)maxn * maxn + (Z.inverse ? (size_t)maxn : 0));
    if (fp64) {
        IMQ_CUDA(cudaFuncSetAttribute(k_schwarz_factor<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
        k_schwarz_factor<double, false><<<Z.npatch, 256, smem, s>>>(
            Z.npatch, Z.patch_off.as<int32_t>(), Z.patch_pts.as<int32_t>(), Z.fac_off.as<int64_t>(),
            P.pos.as<double2>(), P.leaves.as<int32_t>(), P.shape(), shift, 1e-14, Z.factor.as<double>(),
            ncl.as<int>());
    } else {
        auto kern = Z.inverse ? k_schwarz_factor<float, true> : k_schwarz_factor<float, false>;
        IMQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kern<<<Z.npatch, 256, smem, s>>>(Z.npatch, Z.patch_off.as<int32_t>(), Z.patch_pts.as<int32_t>(),
                                         Z.fac_off.as<int64_t>(), P.pos.as<double2>(), P.leaves.as<int32_t>(),
                                         P.shape(), fshift, 1e-6, Z.factor.as<float>(), ncl.as<int>());
    }
    IMQ_LAUNCH_CHECK();
    IMQ_CUDA(cudaStreamSynchronize(s));
    Z.nmax = nmax;
    Z.shift = shift;
    Z.fp64 = fp64;
    Z.ready = true;
}

}  // namespace

void schwarz_apply(const Plan &P, const Schwarz &Z, const double *r, double *z, double c, int64_t n, const void *Sv,
                   cudaStream_t s) {
    const CGScalars *S = static_cast<const CGScalars *>(Sv);
    const unsigned g = blocks_for((int64_t)Z.npatch * 32, 128);
    if (Z.inverse) {
        const size_t smem = inv_apply_smem(Z.maxn);
        IMQ_CUDA(cudaFuncSetAttribute(k_schwarz_inv_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        if (Z.npatch > 0)
            k_schwarz_inv_apply<<<Z.npatch, kInvThreads, smem, s>>>(
                Z.npatch, Z.patch_off.as<int32_t>(), Z.patch_pts.as<int32_t>(), Z.fac_off.as<int64_t>(),
                Z.factor.as<float>(), r, Z.ypatch.as<double>(), S, device_error_word());
    } else if (Z.fp64)
        k_schwarz_solve<double><<<g, 128, 0, s>>>(Z.npatch, Z.patch_off.as<int32_t>(), Z.patch_pts.as<int32_t>(),
                                                  Z.fac_off.as<int64_t>(), Z.factor.as<double>(), r,
                                                  Z.ypatch.as<double>(), S);
    else
        k_schwarz_solve<float><<<g, 128, 0, s>>>(Z.npatch, Z.patch_off.as<int32_t>(), Z.patch_pts.as<int32_t>(),
                                                 Z.fac_off.as<int64_t>(), Z.factor.as<float>(), r,
                                                 Z.ypatch.as<double>(), S);
    k_schwarz_gather<<<kRedBlocks, kRedThreads, 0, s>>>(n, Z.pt_off.as<int32_t>(), Z.pt_slot.as<int32_t>(),
                                                        Z.ypatch.as<double>(), r, c,
                                                        P.nprob > 1 ? P.pt_prob.as<int32_t>() : nullptr,
                                                        P.nprob > 1 ? P.prob_c.as<double>() : nullptr, z, S);
    IMQ_LAUNCH_CHECK();
}

namespace {

struct Work {
    DevMem x, xb, r, p, q, z, u32, b32, part, S, tmp;
    DevMem u2, b2, q2;   // the two-level preconditioner's product (FP32 in / out, or FP64 out)
    DevMem V, hpart, hdev;   // GMRES: Arnoldi basis, partial dots, coefficients
};

double read_dot(const double *a, const double *b, int64_t n, DevMem &part, DevMem &tmp, cudaStream_t s) {
    k_dot_part<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, part.as<double>(), nullptr);
    IMQ_LAUNCH_CHECK();
    k_sum_to<<<1, kRedThreads, 0, s>>>(part.as<double>(), tmp.as<double>());
    IMQ_LAUNCH_CHECK();
    double h = 0;
    IMQ_CUDA(cudaMemcpyAsync(&h, tmp.ptr, sizeof(double), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    return h;
}

// FP64 residual product in the Morton order of plan P: out = A v.  mode 1: the
// dense FP64 product; otherwise the fast product of RP (or P) in FP64.
void residual_product(Plan &P, Plan *RP, int mode, const double *vs, double *outs, cudaStream_t s) {
    const unsigned g = blocks_for(P.N, 256);
    if (mode == 1) {
        dense_matvec_dev(P.pos.as<double>(), P.N, P.c, vs, outs, 1, IMQ_F64, s);
        return;
    }
    if (RP && RP != &P) {   // another plan on the same points: go through the caller's order
        AsyncMem orig(sizeof(double) * P.N, s), us(sizeof(double) * P.N, s), bs(sizeof(double) * P.N, s),
            o2(sizeof(double) * P.N, s);
        k_scatter_f64<<<g, 256, 0, s>>>(vs, P.perm.as<int32_t>(), P.N, orig.as<double>());
        gather_sorted<double, double>(*RP, orig.as<double>(), us.as<double>(), 1, s);
        fmm_apply<double>(*RP, us.as<double>(), bs.as<double>(), 1, s);
        scatter_sorted<double, double>(*RP, bs.as<double>(), o2.as<double>(), 1, s);
        k_gather_f64<<<g, 256, 0, s>>>(o2.as<double>(), P.perm.as<int32_t>(), P.N, outs);
        IMQ_LAUNCH_CHECK();
        return;
    }
    fmm_apply<double>(P, vs, outs, 1, s);
}

}  // namespace

void schwarz_setup(Plan &P, int nmax, double shift, bool fp64, cudaStream_t s) { build_schwarz(P, nmax, shift, fp64, s); }

int schwarz_nmax_of(const imq_cg_options &o) {
    return o.schwarz_nmax > 0 ? o.schwarz_nmax : (o.schwarz_fp64 ? 160 : 224);
}

double device_dot(const double *a, const double *b, int64_t n, cudaStream_t s) {
    DevMem part, tmp;
    part.alloc(8 * kRedBlocks);
    tmp.alloc(64);
    return read_dot(a, b, n, part, tmp, s);
}

void cg_solve(Plan &P, const double *f_dev, double *x_dev, int nrhs, const imq_cg_options &o, Plan *RP,
              imq_cg_info *info, cudaStream_t s) {
    const int64_t n = P.N;
    ensure_ops(P, false, s);
    if (o.residual == IMQ_RESIDUAL_PLAN_F64) ensure_ops(RP ? *RP : P, true, s);
    if (o.inner_operator == IMQ_OPERATOR_FAST_F64) ensure_ops(P, true, s);
    const bool two_level = o.precond == IMQ_PRECOND_SCHWARZ_2L;
    const bool pre = o.precond == IMQ_PRECOND_SCHWARZ || two_level;
    if (pre) build_schwarz(P, schwarz_nmax_of(o), o.schwarz_shift, o.schwarz_fp64 != 0, s);
    if (two_level) coarse_setup(P, o.coarse_points > 0 ? o.coarse_points : P.leaf, o.coarse_gram, s);
    const Schwarz &Z = P.schwarz;
    Work w;
    w.x.alloc(8 * n); w.xb.alloc(8 * n); w.r.alloc(8 * n); w.p.alloc(8 * n); w.q.alloc(8 * n); w.z.alloc(8 * n);
    w.u32.alloc(4 * n); w.b32.alloc(4 * n); w.part.alloc(8 * kRedBlocks); w.S.alloc(sizeof(CGScalars));
    w.tmp.alloc(64);
    if (two_level) {
        w.u2.alloc(4 * n);
        w.b2.alloc(4 * n);
        w.q2.alloc(8 * n);
    }
    DevMem xs, fs, rr_out, ax;
    xs.alloc(8 * n); fs.alloc(8 * n); ax.alloc(8 * n);
    CGScalars *S = w.S.as<CGScalars>();
    double *x = w.x.as<double>(), *r = w.r.as<double>(), *p = w.p.as<double>(), *q = w.q.as<double>();
    double *z = pre ? w.z.as<double>() : r;
    const unsigned g = blocks_for(n, 256);
    const unsigned gr = kRedBlocks;
    // one product outside the capture sets kernel attributes and touches every buffer
    const int op = o.inner_operator;
    IMQ_CUDA(cudaMemsetAsync(w.u32.ptr, 0, 4 * n, s));
    IMQ_CUDA(cudaMemsetAsync(p, 0, 8 * n, s));
    if (op == IMQ_OPERATOR_FAST_F32) fmm_apply<float>(P, w.u32.as<float>(), w.b32.as<float>(), 1, s);
    else if (op == IMQ_OPERATOR_FAST_F64) fmm_apply<double>(P, p, q, 1, s);
    IMQ_CUDA(cudaStreamSynchronize(s));
    // z = M r: the patch solves, and with the coarse level z += Q (r - A z); `done` (device,
    // may be null) lets a converged solve skip the work inside the captured graph
    const int *done_flag = reinterpret_cast<const int *>(reinterpret_cast<const char *>(S) + offsetof(CGScalars, done));
    // the deflation's product A y uses the inner iterations' operator: y carries the patch
    // solves' amplification, so a less accurate product would swamp r - A y
    auto op_product = [&](const double *xin, cudaStream_t st, const CGScalars *Sd, const float **b32,
                          const double **b64) {
        *b32 = nullptr;
        *b64 = nullptr;
        if (op == IMQ_OPERATOR_FAST_F32) {
            k_p_to_f32<<<gr, kRedThreads, 0, st>>>(xin, w.u2.as<float>(), n, Sd);
            IMQ_LAUNCH_CHECK();
            fmm_apply<float>(P, w.u2.as<float>(), w.b2.as<float>(), 1, st);
            *b32 = w.b2.as<float>();
        } else {
            if (op == IMQ_OPERATOR_FAST_F64) fmm_apply<double>(P, xin, w.q2.as<double>(), 1, st);
            else dense_f64_async(P.pos.as<double>(), n, P.c, xin, w.q2.as<double>(), st);
            *b64 = w.q2.as<double>();
        }
    };
    auto precond_apply = [&](const CGScalars *Sd, cudaStream_t st) {
        schwarz_apply(P, Z, r, z, P.c, n, Sd, st);
        if (!two_level) return;
        const int *dn = Sd ? done_flag : nullptr;
        const float *b32;
        const double *b64;
        op_product(z, st, Sd, &b32, &b64);
        coarse_restrict(P, r, b32, b64, dn, st);
        coarse_solve(P, dn, st);
        coarse_prolong(P, z, z, dn, st);
    };

    // ---- GMRES(m): one restart cycle on A d = r (right preconditioning, d = M u), the
    // correction added to w.xb.  Arnoldi basis in w.V, Gram-Schmidt applied twice with
    // FP64 dots in a fixed order, Givens rotations and the triangular solve on the host.
    const bool gmres = o.krylov == IMQ_KRYLOV_GMRES;
    const int gm = o.gmres_m > 0 ? o.gmres_m : 40;
    if (gmres) {
        w.V.alloc(sizeof(double) * (size_t)(gm + 1) * n);
        w.hpart.alloc(sizeof(double) * (size_t)(gm + 1) * kRedBlocks);
        w.hdev.alloc(sizeof(double) * (size_t)(gm + 1));
    }
    auto apply_M = [&](const double *in, double *out) {
        if (!pre) {
            IMQ_CUDA(cudaMemcpyAsync(out, in, 8 * n, cudaMemcpyDeviceToDevice, s));
            return;
        }
        schwarz_apply(P, Z, in, out, P.c, n, nullptr, s);
        if (!two_level) return;
        const float *b32;
        const double *b64;
        op_product(out, s, nullptr, &b32, &b64);
        coarse_restrict(P, in, b32, b64, nullptr, s);
        coarse_solve(P, nullptr, s);
        coarse_prolong(P, out, out, nullptr, s);
    };
    auto apply_A = [&](const double *in, double *out) {
        if (op == IMQ_OPERATOR_FAST_F32) {
            k_p_to_f32<<<gr, kRedThreads, 0, s>>>(in, w.u32.as<float>(), n, nullptr);
            IMQ_LAUNCH_CHECK();
            fmm_apply<float>(P, w.u32.as<float>(), w.b32.as<float>(), 1, s);
            k_f32_to_f64<<<g, 256, 0, s>>>(w.b32.as<float>(), out, n);
            IMQ_LAUNCH_CHECK();
        } else if (op == IMQ_OPERATOR_FAST_F64) {
            fmm_apply<double>(P, in, out, 1, s);
        } else {
            dense_f64_async(P.pos.as<double>(), n, P.c, in, out, s);
        }
    };
    // returns kConverged (target met), kMaxIter (cycle or budget ended) or kNumerical; its += iterations
    auto gmres_cycle = [&](const double *rv, double target, int budget, int &its) -> int {
        double *V = w.V.as<double>(), *zb = w.p.as<double>(), *wv = w.q.as<double>(), *u = w.x.as<double>();
        double *hd = w.hdev.as<double>();
        const double beta0 = std::sqrt(read_dot(rv, rv, n, w.part, w.tmp, s));
        if (!std::isfinite(beta0)) return kNumerical;
        if (beta0 == 0) return kConverged;
        k_scale_to<<<g, 256, 0, s>>>(rv, 1.0 / beta0, V, n);
        IMQ_LAUNCH_CHECK();
        std::vector<double> H((size_t)(gm + 1) * gm, 0.0), cs(gm, 0.0), sn(gm, 0.0), gv(gm + 1, 0.0), hh(gm + 1);
        auto Hij = [&](int i, int j) -> double & { return H[(size_t)j * (gm + 1) + i]; };
        gv[0] = beta0;
        int k = 0, state = kMaxIter;
        for (int j = 0; j < gm && its < budget; ++j) {
            apply_M(V + (size_t)j * n, zb);
            apply_A(zb, wv);
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                k_multi_dot_part<<<kRedBlocks, kRedThreads, 0, s>>>(V, n, j + 1, wv, w.hpart.as<double>());
                k_multi_sum<<<j + 1, kRedThreads, 0, s>>>(w.hpart.as<double>(), hd);
                k_multi_axpy<<<kRedBlocks, kRedThreads, 0, s>>>(V, n, j + 1, hd, wv);
                IMQ_LAUNCH_CHECK();
                IMQ_CUDA(cudaMemcpyAsync(hh.data(), hd, sizeof(double) * (j + 1), cudaMemcpyDeviceToHost, s));
                IMQ_CUDA(cudaStreamSynchronize(s));
                for (int i = 0; i <= j; ++i) Hij(i, j) += hh[i];
            }
            const double hn = std::sqrt(read_dot(wv, wv, n, w.part, w.tmp, s));
            Hij(j + 1, j) = hn;
            ++its;
            k = j + 1;
            for (int i = 0; i < j; ++i) {   // earlier rotations on the new column
                const double a = Hij(i, j), b = Hij(i + 1, j);
                Hij(i, j) = cs[i] * a + sn[i] * b;
                Hij(i + 1, j) = -sn[i] * a + cs[i] * b;
            }
            const double a = Hij(j, j), b = Hij(j + 1, j), rho = std::hypot(a, b);
            if (!std::isfinite(rho)) return kNumerical;
            cs[j] = rho > 0 ? a / rho : 1.0;
            sn[j] = rho > 0 ? b / rho : 0.0;
            Hij(j, j) = rho;
            Hij(j + 1, j) = 0;
            gv[j + 1] = -sn[j] * gv[j];
            gv[j] = cs[j] * gv[j];
            if (std::fabs(gv[j + 1]) <= target || hn == 0) {
                state = kConverged;
                break;
            }
            k_scale_to<<<g, 256, 0, s>>>(wv, 1.0 / hn, V + (size_t)(j + 1) * n, n);
            IMQ_LAUNCH_CHECK();
        }
        if (k == 0) return state;
        std::vector<double> y(k, 0.0);   // H(0:k, 0:k) y = g(0:k), upper triangular
        for (int i = k - 1; i >= 0; --i) {
            double t = gv[i];
            for (int l = i + 1; l < k; ++l) t -= Hij(i, l) * y[l];
            y[i] = Hij(i, i) != 0 ? t / Hij(i, i) : 0.0;
            if (!std::isfinite(y[i])) return kNumerical;
        }
        IMQ_CUDA(cudaMemcpyAsync(hd, y.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
        k_lincomb<<<kRedBlocks, kRedThreads, 0, s>>>(V, n, k, hd, u);
        IMQ_LAUNCH_CHECK();
        apply_M(u, zb);
        k_axpby<<<g, 256, 0, s>>>(w.xb.as<double>(), zb, 1.0, 1.0, n);
        IMQ_LAUNCH_CHECK();
        IMQ_CUDA(cudaStreamSynchronize(s));   // y lives on the host stack
        return state;
    };

    // ---- capture kIterPerGraph PCG iterations on a private stream
    GraphCapture cap;
    cudaStream_t cs = cap.begin();
    for (int it = 0; it < kIterPerGraph; ++it) {
        if (op == IMQ_OPERATOR_FAST_F32) {   // u32 = (float) p, written by the previous k_update_p
            fmm_apply<float>(P, w.u32.as<float>(), w.b32.as<float>(), 1, cs);
            k_q_dot<<<gr, kRedThreads, 0, cs>>>(w.b32.as<float>(), p, q, n, w.part.as<double>(), S);
        } else {
            if (op == IMQ_OPERATOR_FAST_F64) fmm_apply<double>(P, p, q, 1, cs);
            else dense_f64_async(P.pos.as<double>(), n, P.c, p, q, cs);
            k_dot_part<<<gr, kRedThreads, 0, cs>>>(p, q, n, w.part.as<double>(), S);
        }
        k_finish_alpha<<<1, kRedThreads, 0, cs>>>(w.part.as<double>(), S);
        k_update_xr<<<gr, kRedThreads, 0, cs>>>(x, r, p, q, n, w.part.as<double>(), S);
        k_finish_rr<<<1, kRedThreads, 0, cs>>>(w.part.as<double>(), S);
        k_copy_best<<<gr, kRedThreads, 0, cs>>>(x, w.xb.as<double>(), n, S);
        if (pre) {
            precond_apply(S, cs);
            k_dot_part<<<gr, kRedThreads, 0, cs>>>(r, z, n, w.part.as<double>(), S);
            k_finish_beta<<<1, kRedThreads, 0, cs>>>(w.part.as<double>(), S, 0);
        } else {
            k_finish_beta<<<1, kRedThreads, 0, cs>>>(w.part.as<double>(), S, 1);
        }
        k_update_p<<<gr, kRedThreads, 0, cs>>>(p, z, op == IMQ_OPERATOR_FAST_F32 ? w.u32.as<float>() : nullptr, n,
                                               S);
    }
    cudaGraphExec_t exec = cap.instantiate();
    const auto t0 = std::chrono::steady_clock::now();
    int total_iter = 0, outer_done = 0, final_status = kConverged;
    double worst_rel = 0;
    {
        for (int rhs = 0; rhs < nrhs; ++rhs) {
            const double *f = f_dev + (size_t)rhs * n;
            double *xo = x_dev + (size_t)rhs * n;
            k_gather_f64<<<g, 256, 0, s>>>(f, P.perm.as<int32_t>(), n, fs.as<double>());
            if (o.x0_given) k_gather_f64<<<g, 256, 0, s>>>(xo, P.perm.as<int32_t>(), n, xs.as<double>());
            else IMQ_CUDA(cudaMemsetAsync(xs.ptr, 0, 8 * n, s));
            IMQ_LAUNCH_CHECK();
            const double ff = read_dot(fs.as<double>(), fs.as<double>(), n, w.part, w.tmp, s);
            const double fn = std::sqrt(ff);
            double rel = 1.0;
            int status = kMaxIter;
            int iters = 0;
            const int max_outer = std::max(0, o.refine_steps);
            int restarts = 0;
            bool numerical = false;
            double prev_rel = 0;
            for (int outer = 0;; ++outer) {
                // residual r = f - A x (FP64 product unless x = 0)
                if (outer == 0 && !o.x0_given) {
                    IMQ_CUDA(cudaMemcpyAsync(r, fs.ptr, 8 * n, cudaMemcpyDeviceToDevice, s));
                } else {
                    residual_product(P, RP, o.residual == IMQ_RESIDUAL_DENSE_F64 ? 1 : 0, xs.as<double>(),
                                     ax.as<double>(), s);
                    k_sub<<<g, 256, 0, s>>>(r, fs.as<double>(), ax.as<double>(), n);
                    IMQ_LAUNCH_CHECK();
                }
                const double rr0 = read_dot(r, r, n, w.part, w.tmp, s);
                rel = fn > 0 ? std::sqrt(rr0) / fn : 0.0;
                if (!std::isfinite(rel)) {
                    status = kNumerical;
                    break;
                }
                if (rel <= o.rtol) {
                    status = kConverged;
                    break;
                }
                status = kMaxIter;
                if (iters >= o.maxit) break;
                // GMRES cycles without refinement steps continue while each one lowers the true residual
                if (gmres && max_outer == 0 && outer > 0 && !(rel < 0.999 * prev_rel)) break;
                prev_rel = rel;
                if (max_outer > 0 ? outer >= max_outer : (!gmres && outer > restarts)) break;
                // inner PCG on A d = r from d = 0
                // the recursive residual of the inner operator drifts from the true one by about the
                // operator's rounding error, so a single pass aims at half the tolerance
                const double inner_rtol =
                    max_outer > 0 ? std::max(o.inner_rtol, std::min(0.5, 0.5 * o.rtol / rel)) : 0.5 * o.rtol / rel;
                IMQ_CUDA(cudaMemsetAsync(x, 0, 8 * n, s));
                IMQ_CUDA(cudaMemsetAsync(w.xb.ptr, 0, 8 * n, s));
                double rr_start = rr0;
                if (two_level) {   // start the pass from the coarse solution d = Q r, r -= A d
                    coarse_restrict(P, r, nullptr, nullptr, nullptr, s);
                    coarse_solve(P, nullptr, s);
                    coarse_prolong(P, nullptr, x, nullptr, s);
                    IMQ_CUDA(cudaMemcpyAsync(w.xb.ptr, x, 8 * n, cudaMemcpyDeviceToDevice, s));
                    const float *b32;
                    const double *b64;
                    op_product(x, s, nullptr, &b32, &b64);
                    if (b32) k_sub_f32<<<gr, kRedThreads, 0, s>>>(r, b32, n);
                    else k_sub_f64<<<gr, kRedThreads, 0, s>>>(r, b64, n);
                    IMQ_LAUNCH_CHECK();
                    rr_start = read_dot(r, r, n, w.part, w.tmp, s);
                }
                if (gmres) {
                    int its = 0;
                    const int gs = gmres_cycle(r, inner_rtol * std::sqrt(rr0), o.maxit - iters, its);
                    iters += its;
                    k_axpby<<<g, 256, 0, s>>>(xs.as<double>(), w.xb.as<double>(), 1.0, 1.0, n);
                    IMQ_LAUNCH_CHECK();
                    outer_done = std::max(outer_done, outer + 1);
                    if (gs == kNumerical) {
                        numerical = true;
                        break;
                    }
                    continue;
                }
                CGScalars h{};
                h.rr = rr_start;
                h.rr0 = rr0;
                h.rr_best = rr_start;
                h.rr_target = inner_rtol * inner_rtol * rr0;
                h.maxit = o.maxit - iters;
                if (pre) {
                    CGScalars hz = h;
                    IMQ_CUDA(cudaMemcpyAsync(S, &hz, sizeof(CGScalars), cudaMemcpyHostToDevice, s));
                    precond_apply(S, s);
                    h.rz = read_dot(r, z, n, w.part, w.tmp, s);
                } else {
                    h.rz = rr0;
                }
                if (!std::isfinite(h.rz)) {
                    status = kNumerical;
                    break;
                }
                if (!(h.rz > 0)) break;   // the preconditioner is not positive on r: keep x
                IMQ_CUDA(cudaMemcpyAsync(p, z, 8 * n, cudaMemcpyDeviceToDevice, s));
                IMQ_CUDA(cudaMemcpyAsync(S, &h, sizeof(CGScalars), cudaMemcpyHostToDevice, s));
                if (op == IMQ_OPERATOR_FAST_F32) {   // the first product's input; the graph writes the rest
                    k_p_to_f32<<<gr, kRedThreads, 0, s>>>(p, w.u32.as<float>(), n, S);
                    IMQ_LAUNCH_CHECK();
                }
                CGScalars hs{};
                for (;;) {
                    IMQ_CUDA(cudaGraphLaunch(exec, s));
                    IMQ_CUDA(cudaMemcpyAsync(&hs, S, sizeof(CGScalars), cudaMemcpyDeviceToHost, s));
                    IMQ_CUDA(cudaStreamSynchronize(s));
                    if (hs.done) break;
                }
                iters += hs.iter;
                // x += best inner iterate (the pass's x = 0 start if no iterate improved)
                k_axpby<<<g, 256, 0, s>>>(xs.as<double>(), w.xb.as<double>(), 1.0, 1.0, n);
                IMQ_LAUNCH_CHECK();
                outer_done = std::max(outer_done, outer + 1);
                if (hs.status == kNumerical) {
                    numerical = true;
                    break;
                }
                // without refinement steps, a pass that improved on its start and either broke down
                // or met its target on the recursive residual is restarted from the true residual of
                // its best iterate while iterations are left (the recursive residual of the FP32
                // operator can drift below the true one, so only the true residual certifies);
                // otherwise the next outer pass only computes the final true residual
                if (max_outer == 0) {
                    if ((hs.status == kBreakdown || hs.status == kConverged) && hs.rr_best < hs.rr0 &&
                        restarts < kMaxRestarts)
                        ++restarts;
                    else restarts = -1;
                }
            }
            if (numerical) {
                // report the true residual of the iterate that is returned
                residual_product(P, RP, o.residual == IMQ_RESIDUAL_DENSE_F64 ? 1 : 0, xs.as<double>(),
                                 ax.as<double>(), s);
                k_sub<<<g, 256, 0, s>>>(r, fs.as<double>(), ax.as<double>(), n);
                IMQ_LAUNCH_CHECK();
                rel = std::sqrt(read_dot(r, r, n, w.part, w.tmp, s)) / fn;
                status = kNumerical;
            }
            k_scatter_f64<<<g, 256, 0, s>>>(xs.as<double>(), P.perm.as<int32_t>(), n, xo);
            IMQ_LAUNCH_CHECK();
            check_device_errors(s);   // synchronises; a wait that ran out invalidates the solve
            total_iter += iters;
            worst_rel = std::max(worst_rel, rel);
            if (status != kConverged) final_status = status == kNumerical ? kNumerical : kMaxIter;
            if (info && rhs < IMQ_CG_MAX_RHS_INFO) info->rel_residual[rhs] = rel;
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        info->iterations = total_iter;
        info->outer_steps = outer_done;
        info->max_rel_residual = worst_rel;
        info->seconds = secs;
        info->status = final_status == kConverged ? IMQ_OK : (final_status == kNumerical ? IMQ_NUMERICAL : IMQ_NOT_CONVERGED);
    }
    if (final_status == kNumerical) fail(IMQ_NUMERICAL, "imq_cg_solve: non-finite value or breakdown in CG");
    if (final_status != kConverged)
        fail(IMQ_NOT_CONVERGED, "imq_cg_solve: tolerance not reached; coef holds the best iterate");
}

}  // namespace imq
