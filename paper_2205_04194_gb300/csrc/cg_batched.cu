// Conjugate gradients on a batched plan: nprob independent interpolation
// systems A_b coef_b = f_b (Section 2, Eq. (3)-(4), one per problem) solved
// together.  Every product is one fast product over the merged tree of all
// problems; every scalar of CG (alpha, beta, the residual norms, the
// convergence test) is per problem.
//
//  * points of problem b occupy the contiguous Morton-order range
//    [prob_off[b], prob_off[b+1]), so each per-problem dot is one thread
//    block over that range: a fixed stride and a fixed tree, hence
//    bit-reproducible; the block finishes the scalar update itself, so an
//    iteration needs no separate "finish" launches;
//  * a problem that has converged (or broken down) sets its own done flag and
//    its blocks skip the vector updates; the product still runs over the whole
//    merged tree (the other problems need it);
//  * kIterPerGraph iterations are captured into one CUDA graph; the host reads
//    the nprob state records once per graph launch and stops when all are done;
//  * refinement steps are taken together: r_b = f_b - A_b x_b in FP64 for all
//    problems, problems already within rtol stay done through the inner pass.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kThreads = 512;
constexpr int kIterPerGraph = 8;

// kBreakdown: a finite p.q <= 0 or r.z <= 0 (the FP32 product or the shifted
// patch factors are not exactly positive definite for a nearly singular A);
// the problem's pass ends and it is restarted from its true residual.
enum BState : int { kRunning = 0, kConverged = 1, kNumerical = 2, kMaxIter = 3, kBreakdown = 4 };
constexpr int kMaxRestarts = 16;   // restarts after a breakdown when no refinement steps are requested

struct BScalars {
    double rz, rr, alpha, rr_target, rr_best, rr0;
    int iter, done, status, maxit;
};

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kThreads];
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = kThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    const double t = sh[0];
    __syncthreads();
    return t;
}

__global__ void k_to_f32(const double *__restrict__ p, float *__restrict__ u, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        u[i] = (float)p[i];
}

// q = A p (from FP32 b32 or FP64 q64), alpha_b = rz_b / (p.q)_b
__global__ void __launch_bounds__(kThreads) k_alpha(const float *__restrict__ b32, const double *__restrict__ p,
                                                    double *__restrict__ q, const int64_t *__restrict__ off,
                                                    BScalars *S) {
    const int b = blockIdx.x;
    if (S[b].done) return;
    const int64_t lo = off[b], hi = off[b + 1];
    double acc = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        double qi;
        if (b32) {
            qi = (double)b32[i];
            q[i] = qi;
        } else {
            qi = q[i];
        }
        acc += p[i] * qi;
    }
    const double pq = block_sum(acc);
    if (threadIdx.x == 0) {
        if (!isfinite(pq)) {
            S[b].status = kNumerical;
            S[b].done = 1;
        } else if (!(pq > 0)) {
            S[b].status = kBreakdown;
            S[b].done = 1;
        } else {
            S[b].alpha = S[b].rz / pq;
        }
    }
}

// x += alpha p, r -= alpha q, rr = r.r, convergence test, keep the best iterate
__global__ void __launch_bounds__(kThreads) k_update(double *__restrict__ x, double *__restrict__ r,
                                                     const double *__restrict__ p, const double *__restrict__ q,
                                                     double *__restrict__ xb, const int64_t *__restrict__ off,
                                                     BScalars *S) {
    const int b = blockIdx.x;
    __shared__ int s_go, s_improved;
    if (threadIdx.x == 0) s_go = !S[b].done;
    __syncthreads();
    if (!s_go) return;
    const int64_t lo = off[b], hi = off[b + 1];
    const double a = S[b].alpha;
    double acc = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        x[i] += a * p[i];
        const double ri = r[i] - a * q[i];
        r[i] = ri;
        acc += ri * ri;
    }
    const double rr = block_sum(acc);
    if (threadIdx.x == 0) {
        BScalars &s = S[b];
        s.rr = rr;
        s.iter += 1;
        s_improved = 0;
        if (!isfinite(rr)) {
            s.status = kNumerical;
            s.done = 1;
        } else {
            if (rr < s.rr_best) {
                s.rr_best = rr;
                s_improved = 1;
            }
            if (rr <= s.rr_target) {
                s.status = kConverged;
                s.done = 1;
            } else if (s.iter >= s.maxit) {
                s.status = kMaxIter;
                s.done = 1;
            }
        }
    }
    __syncthreads();
    if (s_improved)
        for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) xb[i] = x[i];
}

// beta_b = (r.z)_b / rz_b, p = z + beta p, rz_b = (r.z)_b.  Run on problems
// that finished in this iteration too: their p is never used again.
__global__ void __launch_bounds__(kThreads) k_beta(const double *__restrict__ r, const double *__restrict__ z,
                                                   double *__restrict__ p, const int64_t *__restrict__ off,
                                                   BScalars *S) {
    const int b = blockIdx.x;
    __shared__ double s_beta;
    __shared__ int s_go;
    if (threadIdx.x == 0) s_go = !S[b].done;
    __syncthreads();
    if (!s_go) return;
    const int64_t lo = off[b], hi = off[b + 1];
    double acc = 0;
    if (z != r)
        for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) acc += r[i] * z[i];
    const double rzn = z != r ? block_sum(acc) : S[b].rr;
    if (threadIdx.x == 0) {
        BScalars &s = S[b];
        if (!isfinite(rzn)) {
            s.status = kNumerical;
            s.done = 1;
            s_beta = 0;
        } else if (!(rzn > 0)) {
            s.status = kBreakdown;
            s.done = 1;
            s_beta = 0;
        } else {
            s_beta = rzn / s.rz;
            s.rz = rzn;
        }
    }
    __syncthreads();
    const double bt = s_beta;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) p[i] = z[i] + bt * p[i];
}

// out_b = (a.c)_b for every problem
__global__ void __launch_bounds__(kThreads) k_seg_dot(const double *__restrict__ a, const double *__restrict__ c,
                                                      const int64_t *__restrict__ off, double *__restrict__ out) {
    const int b = blockIdx.x;
    const int64_t lo = off[b], hi = off[b + 1];
    double acc = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) acc += a[i] * c[i];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) out[b] = t;
}

__global__ void k_sub(double *__restrict__ r, const double *__restrict__ f, const double *__restrict__ ax, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] = f[i] - ax[i];
}

__global__ void k_sub_from(double *__restrict__ r, const double *__restrict__ ax, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        r[i] -= ax[i];
}

__global__ void k_add(double *__restrict__ y, const double *__restrict__ x, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}

__global__ void k_gather(const double *__restrict__ v, const int32_t *__restrict__ perm, int64_t n,
                         double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = v[perm[i]];
}

__global__ void k_scatter(const double *__restrict__ v, const int32_t *__restrict__ perm, int64_t n,
                          double *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = v[i];
}

// ---- per-problem GMRES (Arnoldi vectors over the flattened points, every scalar per problem)
// out[i * B + b] = (V_i . w) restricted to problem b; one block per (problem, vector)
__global__ void __launch_bounds__(kThreads) k_seg_multi_dot(const double *__restrict__ V, int64_t n,
                                                            const double *__restrict__ w,
                                                            const int64_t *__restrict__ off, int B,
                                                            double *__restrict__ out) {
    const int b = blockIdx.x, i = blockIdx.y;
    const int64_t lo = off[b], hi = off[b + 1];
    const double *vi = V + (size_t)i * n;
    double acc = 0;
    for (int64_t k = lo + threadIdx.x; k < hi; k += kThreads) acc += vi[k] * w[k];
    const double t = block_sum(acc);
    if (threadIdx.x == 0) out[(size_t)i * B + b] = t;
}
// w -= sum_i h[i][problem] V_i
__global__ void k_seg_multi_axpy(const double *__restrict__ V, int64_t n, int nv, const double *__restrict__ h,
                                 const int32_t *__restrict__ prob, int B, double *__restrict__ w) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = prob[k];
        double acc = 0;
        for (int i = 0; i < nv; ++i) acc += h[(size_t)i * B + b] * V[(size_t)i * n + k];
        w[k] -= acc;
    }
}
// u = sum_i y[i][problem] V_i (y = 0 past a problem's own cycle length)
__global__ void k_seg_lincomb(const double *__restrict__ V, int64_t n, int nv, const double *__restrict__ y,
                              const int32_t *__restrict__ prob, int B, double *__restrict__ u) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int b = prob[k];
        double acc = 0;
        for (int i = 0; i < nv; ++i) acc += y[(size_t)i * B + b] * V[(size_t)i * n + k];
        u[k] = acc;
    }
}
// v = a[problem] * w
__global__ void k_seg_scale(const double *__restrict__ w, const double *__restrict__ a,
                            const int32_t *__restrict__ prob, int64_t n, double *__restrict__ v) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        v[k] = a[prob[k]] * w[k];
}
__global__ void k_f32_to_f64(const float *__restrict__ b, double *__restrict__ q, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        q[k] = (double)b[k];
}

std::vector<double> read_seg_dots(const double *a, const double *c, const int64_t *off, int B, DevMem &tmp,
                                  cudaStream_t s) {
    k_seg_dot<<<B, kThreads, 0, s>>>(a, c, off, tmp.as<double>());
    IMQ_LAUNCH_CHECK();
    std::vector<double> h(B);
    IMQ_CUDA(cudaMemcpyAsync(h.data(), tmp.ptr, sizeof(double) * B, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    return h;
}

}  // namespace

void cg_solve_batched(Plan &P, const double *f_dev, double *x_dev, int nrhs, const imq_cg_options &o,
                      imq_cg_info *info, double *rel_out, int32_t *iters_out, cudaStream_t s) {
    const int64_t n = P.N;
    const int B = P.nprob;
    if (o.residual_plan) fail(IMQ_UNSUPPORTED, "imq_cg_solve: residual_plan is not supported on batched plans");
    // the dense FP64 products of a batched plan are block diagonal: each problem only with itself
    const bool dense_res = o.residual == IMQ_RESIDUAL_DENSE_F64;
    const bool dense_op = o.inner_operator == IMQ_OPERATOR_DENSE_F64;
    ensure_ops(P, false, s);
    if (!dense_res || o.inner_operator == IMQ_OPERATOR_FAST_F64) ensure_ops(P, true, s);   // FP64 fast product
    const bool two_level = o.precond == IMQ_PRECOND_SCHWARZ_2L;
    if (two_level && o.krylov != IMQ_KRYLOV_GMRES)
        fail(IMQ_UNSUPPORTED, "imq_cg_solve_batched: the two-level preconditioner runs with GMRES on batched plans");
    const bool pre = o.precond == IMQ_PRECOND_SCHWARZ || two_level;
    if (pre) schwarz_setup(P, schwarz_nmax_of(o), o.schwarz_shift, o.schwarz_fp64 != 0, s);
    if (two_level) coarse_setup(P, o.coarse_points > 0 ? o.coarse_points : P.leaf, o.coarse_gram, s);
    const bool f64op = o.inner_operator == IMQ_OPERATOR_FAST_F64;
    const double *dpos = P.pos.as<double>(), *dprob_c = P.prob_c.as<double>();

    DevMem x, xb, r, p, q, z, u32, b32, St, tmp, off, xs, fs, ax;
    for (DevMem *d : {&x, &xb, &r, &p, &q, &xs, &fs, &ax}) d->alloc(8 * n);
    if (pre) z.alloc(8 * n);
    u32.alloc(4 * n);
    b32.alloc(4 * n);
    St.alloc(sizeof(BScalars) * B);
    tmp.alloc(sizeof(double) * B);
    off.alloc(sizeof(int64_t) * (B + 1));
    IMQ_CUDA(cudaMemcpyAsync(off.ptr, P.prob_off.data(), sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
    BScalars *S = St.as<BScalars>();
    const int64_t *doff = off.as<int64_t>();
    double *zp = pre ? z.as<double>() : r.as<double>();
    const unsigned g = blocks_for(n, 256);
    const unsigned gs = std::min<unsigned>(g, 4 * 152);

    IMQ_CUDA(cudaMemsetAsync(u32.ptr, 0, 4 * n, s));
    IMQ_CUDA(cudaMemsetAsync(p.ptr, 0, 8 * n, s));
    if (f64op) fmm_apply<double>(P, p.as<double>(), q.as<double>(), 1, s);
    else if (!dense_op) fmm_apply<float>(P, u32.as<float>(), b32.as<float>(), 1, s);
    IMQ_CUDA(cudaStreamSynchronize(s));

    GraphCapture cap;
    cudaStream_t cs = cap.begin();
    {
        for (int it = 0; it < kIterPerGraph; ++it) {
            if (dense_op) {
                dense_f64_seg_async(dpos, doff, B, dprob_c, p.as<double>(), q.as<double>(), n, cs);
                k_alpha<<<B, kThreads, 0, cs>>>(nullptr, p.as<double>(), q.as<double>(), doff, S);
            } else if (f64op) {
                fmm_apply<double>(P, p.as<double>(), q.as<double>(), 1, cs);
                k_alpha<<<B, kThreads, 0, cs>>>(nullptr, p.as<double>(), q.as<double>(), doff, S);
            } else {
                k_to_f32<<<gs, 256, 0, cs>>>(p.as<double>(), u32.as<float>(), n);
                fmm_apply<float>(P, u32.as<float>(), b32.as<float>(), 1, cs);
                k_alpha<<<B, kThreads, 0, cs>>>(b32.as<float>(), p.as<double>(), q.as<double>(), doff, S);
            }
            k_update<<<B, kThreads, 0, cs>>>(x.as<double>(), r.as<double>(), p.as<double>(), q.as<double>(),
                                             xb.as<double>(), doff, S);
            if (pre) schwarz_apply(P, P.schwarz, r.as<double>(), zp, P.c, n, nullptr, cs);
            k_beta<<<B, kThreads, 0, cs>>>(r.as<double>(), zp, p.as<double>(), doff, S);
        }
    }
    cudaGraphExec_t exec = cap.instantiate();

    // ---- GMRES(m) per problem: one restart cycle on A d = r for every active problem at once
    // (right preconditioning, d = M u); the correction is added to xb
    const bool gmres = o.krylov == IMQ_KRYLOV_GMRES;
    const int gm = o.gmres_m > 0 ? o.gmres_m : 40;
    DevMem V, hdev, ydev, scdev, zb, wv, ub, ay;
    if (gmres) {
        V.alloc(sizeof(double) * (size_t)(gm + 1) * n);
        hdev.alloc(sizeof(double) * (size_t)(gm + 1) * B);
        ydev.alloc(sizeof(double) * (size_t)(gm + 1) * B);
        scdev.alloc(sizeof(double) * B);
        for (DevMem *d : {&zb, &wv, &ub, &ay}) d->alloc(8 * n);
    }
    const int32_t *prob = P.pt_prob.as<int32_t>();
    auto apply_A = [&](const double *in, double *out) {
        if (dense_op) {
            dense_f64_seg_async(dpos, doff, B, dprob_c, in, out, n, s);
        } else if (f64op) {
            fmm_apply<double>(P, in, out, 1, s);
        } else {
            k_to_f32<<<gs, 256, 0, s>>>(in, u32.as<float>(), n);
            fmm_apply<float>(P, u32.as<float>(), b32.as<float>(), 1, s);
            k_f32_to_f64<<<gs, 256, 0, s>>>(b32.as<float>(), out, n);
            IMQ_LAUNCH_CHECK();
        }
    };
    // z = M r: the patch solves y, and with the coarse level z = y + Q (r - A y)
    auto apply_M = [&](const double *in, double *out) {
        if (!pre) {
            IMQ_CUDA(cudaMemcpyAsync(out, in, 8 * n, cudaMemcpyDeviceToDevice, s));
            return;
        }
        schwarz_apply(P, P.schwarz, in, out, P.c, n, nullptr, s);
        if (!two_level) return;
        apply_A(out, ay.as<double>());
        coarse_restrict(P, in, nullptr, ay.as<double>(), nullptr, s);
        coarse_solve(P, nullptr, s);
        coarse_prolong(P, out, out, nullptr, s);
    };
    auto seg_scale = [&](const double *w, const std::vector<double> &a, double *v) {
        IMQ_CUDA(cudaMemcpyAsync(scdev.ptr, a.data(), sizeof(double) * B, cudaMemcpyHostToDevice, s));
        k_seg_scale<<<gs, 256, 0, s>>>(w, scdev.as<double>(), prob, n, v);
        IMQ_LAUNCH_CHECK();
    };
    // r holds each active problem's residual (zero on the others); returns per-problem iterations
    auto gmres_cycle = [&](const std::vector<double> &target, const std::vector<int> &budget,
                           std::vector<int> &its, std::vector<char> &bad) {
        double *Vp = V.as<double>();
        const std::vector<double> bb = read_seg_dots(r.as<double>(), r.as<double>(), doff, B, tmp, s);
        std::vector<double> beta(B), sc(B, 0.0);
        std::vector<char> live(B, 0);
        std::vector<int> kb(B, 0);
        bool any = false;
        for (int b = 0; b < B; ++b) {
            beta[b] = std::sqrt(bb[b]);
            if (!std::isfinite(beta[b])) {
                bad[b] = 1;
                continue;
            }
            live[b] = beta[b] > target[b] && budget[b] > 0;
            sc[b] = live[b] ? 1.0 / beta[b] : 0.0;
            any |= live[b] != 0;
        }
        if (!any) return;
        seg_scale(r.as<double>(), sc, Vp);
        const size_t HS = (size_t)(gm + 1) * gm;
        std::vector<double> H(HS * B, 0.0), cs((size_t)gm * B), sn((size_t)gm * B), gv((size_t)(gm + 1) * B, 0.0),
            hh((size_t)(gm + 1) * B);
        auto Hb = [&](int b, int i, int j) -> double & { return H[(size_t)b * HS + (size_t)j * (gm + 1) + i]; };
        for (int b = 0; b < B; ++b) gv[(size_t)b * (gm + 1)] = beta[b];
        int jmax = 0;
        for (int j = 0; j < gm && any; ++j) {
            apply_M(Vp + (size_t)j * n, zb.as<double>());
            apply_A(zb.as<double>(), wv.as<double>());
            for (int pass = 0; pass < 2; ++pass) {   // classical Gram-Schmidt, twice
                k_seg_multi_dot<<<dim3(B, j + 1), kThreads, 0, s>>>(Vp, n, wv.as<double>(), doff, B,
                                                                    hdev.as<double>());
                k_seg_multi_axpy<<<gs, 256, 0, s>>>(Vp, n, j + 1, hdev.as<double>(), prob, B, wv.as<double>());
                IMQ_LAUNCH_CHECK();
                IMQ_CUDA(cudaMemcpyAsync(hh.data(), hdev.ptr, sizeof(double) * (size_t)(j + 1) * B,
                                         cudaMemcpyDeviceToHost, s));
                IMQ_CUDA(cudaStreamSynchronize(s));
                for (int b = 0; b < B; ++b)
                    if (live[b])
                        for (int i = 0; i <= j; ++i) Hb(b, i, j) += hh[(size_t)i * B + b];
            }
            const std::vector<double> hn2 = read_seg_dots(wv.as<double>(), wv.as<double>(), doff, B, tmp, s);
            jmax = j + 1;
            any = false;
            for (int b = 0; b < B; ++b) {
                sc[b] = 0.0;
                if (!live[b]) continue;
                double *g = &gv[(size_t)b * (gm + 1)];
                double *c = &cs[(size_t)b * gm], *sv = &sn[(size_t)b * gm];
                const double hn = std::sqrt(hn2[b]);
                Hb(b, j + 1, j) = hn;
                ++its[b];
                kb[b] = j + 1;
                for (int i = 0; i < j; ++i) {   // earlier rotations on the new column
                    const double a = Hb(b, i, j), e = Hb(b, i + 1, j);
                    Hb(b, i, j) = c[i] * a + sv[i] * e;
                    Hb(b, i + 1, j) = -sv[i] * a + c[i] * e;
                }
                const double a = Hb(b, j, j), e = Hb(b, j + 1, j), rho = std::hypot(a, e);
                if (!std::isfinite(rho)) {
                    bad[b] = 1;
                    live[b] = 0;
                    kb[b] = 0;
                    continue;
                }
                c[j] = rho > 0 ? a / rho : 1.0;
                sv[j] = rho > 0 ? e / rho : 0.0;
                Hb(b, j, j) = rho;
                Hb(b, j + 1, j) = 0;
                g[j + 1] = -sv[j] * g[j];
                g[j] = c[j] * g[j];
                if (std::fabs(g[j + 1]) <= target[b] || hn == 0 || its[b] >= budget[b]) {
                    live[b] = 0;
                    continue;
                }
                sc[b] = 1.0 / hn;
                any = true;
            }
            seg_scale(wv.as<double>(), sc, Vp + (size_t)(j + 1) * n);
        }
        // y_b from H_b(0:k, 0:k) y_b = g_b(0:k), problem by problem
        std::vector<double> y((size_t)(gm + 1) * B, 0.0);
        for (int b = 0; b < B; ++b) {
            const int k = kb[b];
            const double *g = &gv[(size_t)b * (gm + 1)];
            for (int i = k - 1; i >= 0; --i) {
                double t = g[i];
                for (int l = i + 1; l < k; ++l) t -= Hb(b, i, l) * y[(size_t)l * B + b];
                const double d = Hb(b, i, i);
                y[(size_t)i * B + b] = d != 0 ? t / d : 0.0;
                if (!std::isfinite(y[(size_t)i * B + b])) {
                    bad[b] = 1;
                    for (int l = 0; l < k; ++l) y[(size_t)l * B + b] = 0.0;
                    break;
                }
            }
        }
        if (jmax == 0) return;
        IMQ_CUDA(cudaMemcpyAsync(ydev.ptr, y.data(), sizeof(double) * (size_t)jmax * B, cudaMemcpyHostToDevice, s));
        k_seg_lincomb<<<gs, 256, 0, s>>>(Vp, n, jmax, ydev.as<double>(), prob, B, ub.as<double>());
        IMQ_LAUNCH_CHECK();
        apply_M(ub.as<double>(), zb.as<double>());
        k_add<<<gs, 256, 0, s>>>(xb.as<double>(), zb.as<double>(), n);
        IMQ_LAUNCH_CHECK();
        IMQ_CUDA(cudaStreamSynchronize(s));   // y lives on the host
    };

    const auto t0 = std::chrono::steady_clock::now();
    int total_iter = 0, outer_done = 0, final_status = kConverged;
    double worst_rel = 0;
    std::vector<BScalars> h(B);
    {
        for (int rhs = 0; rhs < nrhs; ++rhs) {
            const double *f = f_dev + (size_t)rhs * n;
            double *xo = x_dev + (size_t)rhs * n;
            k_gather<<<g, 256, 0, s>>>(f, P.perm.as<int32_t>(), n, fs.as<double>());
            if (o.x0_given) k_gather<<<g, 256, 0, s>>>(xo, P.perm.as<int32_t>(), n, xs.as<double>());
            else IMQ_CUDA(cudaMemsetAsync(xs.ptr, 0, 8 * n, s));
            IMQ_LAUNCH_CHECK();
            const std::vector<double> ff = read_seg_dots(fs.as<double>(), fs.as<double>(), doff, B, tmp, s);
            std::vector<double> rel(B, 1.0);
            std::vector<int> status(B, kMaxIter), iters(B, 0);
            const int max_outer = std::max(0, o.refine_steps);
            int restarts = 0;
            std::vector<double> prev_rel(B, 0.0);
            std::vector<char> stalled(B, 0);
            auto true_residual = [&]() {
                if (dense_res) dense_f64_seg_async(dpos, doff, B, dprob_c, xs.as<double>(), ax.as<double>(), n, s);
                else fmm_apply<double>(P, xs.as<double>(), ax.as<double>(), 1, s);
                k_sub<<<gs, 256, 0, s>>>(r.as<double>(), fs.as<double>(), ax.as<double>(), n);
                IMQ_LAUNCH_CHECK();
                return read_seg_dots(r.as<double>(), r.as<double>(), doff, B, tmp, s);
            };
            for (int outer = 0;; ++outer) {
                std::vector<double> rr0;
                if (outer == 0 && !o.x0_given) {
                    IMQ_CUDA(cudaMemcpyAsync(r.ptr, fs.ptr, 8 * n, cudaMemcpyDeviceToDevice, s));
                    rr0 = ff;
                } else {
                    rr0 = true_residual();
                }
                bool any = false;
                for (int b = 0; b < B; ++b) {
                    const double fn = std::sqrt(ff[b]);
                    rel[b] = fn > 0 ? std::sqrt(rr0[b]) / fn : 0.0;
                    if (status[b] == kNumerical) continue;
                    if (!std::isfinite(rel[b])) status[b] = kNumerical;
                    else if (rel[b] <= o.rtol) status[b] = kConverged;
                    else {
                        status[b] = kMaxIter;
                        // GMRES cycles without refinement steps continue while each lowers the true residual
                        if (gmres && max_outer == 0 && outer > 0 && !(rel[b] < 0.999 * prev_rel[b])) stalled[b] = 1;
                        if (iters[b] < o.maxit && !stalled[b]) any = true;
                    }
                    prev_rel[b] = rel[b];
                }
                if (!any || (max_outer > 0 ? outer >= max_outer : (!gmres && outer > restarts))) break;
                if (gmres) {
                    // problems not in this cycle: zero residual segments (their correction is zero)
                    std::vector<double> keep(B), target(B);
                    std::vector<int> budget(B), its(B, 0);
                    std::vector<char> bad(B, 0);
                    for (int b = 0; b < B; ++b) {
                        const bool act = status[b] == kMaxIter && iters[b] < o.maxit && !stalled[b];
                        keep[b] = act ? 1.0 : 0.0;
                        const double inner_rtol =
                            max_outer > 0 ? std::max(o.inner_rtol, std::min(0.5, 0.5 * o.rtol / rel[b]))
                                          : 0.5 * o.rtol / rel[b];
                        target[b] = inner_rtol * std::sqrt(rr0[b]);
                        budget[b] = act ? o.maxit - iters[b] : 0;
                    }
                    seg_scale(r.as<double>(), keep, r.as<double>());
                    IMQ_CUDA(cudaMemsetAsync(xb.ptr, 0, 8 * n, s));
                    if (two_level) {   // start from the coarse solution d = Q r, r -= A d (zero off the cycle)
                        coarse_restrict(P, r.as<double>(), nullptr, nullptr, nullptr, s);
                        coarse_solve(P, nullptr, s);
                        coarse_prolong(P, nullptr, xb.as<double>(), nullptr, s);
                        apply_A(xb.as<double>(), ay.as<double>());
                        k_sub_from<<<gs, 256, 0, s>>>(r.as<double>(), ay.as<double>(), n);
                        IMQ_LAUNCH_CHECK();
                    }
                    gmres_cycle(target, budget, its, bad);
                    k_add<<<gs, 256, 0, s>>>(xs.as<double>(), xb.as<double>(), n);
                    IMQ_LAUNCH_CHECK();
                    outer_done = std::max(outer_done, outer + 1);
                    for (int b = 0; b < B; ++b) {
                        iters[b] += its[b];
                        if (bad[b]) status[b] = kNumerical;
                    }
                    continue;
                }
                IMQ_CUDA(cudaMemsetAsync(x.ptr, 0, 8 * n, s));
                IMQ_CUDA(cudaMemsetAsync(xb.ptr, 0, 8 * n, s));
                std::vector<double> rz = rr0;
                if (pre) {
                    schwarz_apply(P, P.schwarz, r.as<double>(), zp, P.c, n, nullptr, s);
                    rz = read_seg_dots(r.as<double>(), zp, doff, B, tmp, s);
                }
                IMQ_CUDA(cudaMemcpyAsync(p.ptr, zp, 8 * n, cudaMemcpyDeviceToDevice, s));
                for (int b = 0; b < B; ++b) {
                    BScalars &e = h[b];
                    e = BScalars{};
                    const bool active = status[b] == kMaxIter && iters[b] < o.maxit;
                    const double inner_rtol =
                        max_outer > 0 ? std::max(o.inner_rtol, std::min(0.5, 0.5 * o.rtol / rel[b]))
                                      : 0.5 * o.rtol / rel[b];
                    e.rz = rz[b];
                    e.rr = rr0[b];
                    e.rr0 = rr0[b];
                    e.rr_best = rr0[b];
                    e.rr_target = inner_rtol * inner_rtol * rr0[b];
                    e.maxit = o.maxit - iters[b];
                    e.done = active ? 0 : 1;
                    e.status = active ? kRunning : kConverged;
                }
                IMQ_CUDA(cudaMemcpyAsync(S, h.data(), sizeof(BScalars) * B, cudaMemcpyHostToDevice, s));
                for (;;) {
                    IMQ_CUDA(cudaGraphLaunch(exec, s));
                    IMQ_CUDA(cudaMemcpyAsync(h.data(), S, sizeof(BScalars) * B, cudaMemcpyDeviceToHost, s));
                    IMQ_CUDA(cudaStreamSynchronize(s));
                    bool all = true;
                    for (int b = 0; b < B && all; ++b) all = h[b].done != 0;
                    if (all) break;
                }
                k_add<<<gs, 256, 0, s>>>(xs.as<double>(), xb.as<double>(), n);
                IMQ_LAUNCH_CHECK();
                outer_done = std::max(outer_done, outer + 1);
                for (int b = 0; b < B; ++b) {
                    iters[b] += h[b].iter;
                    if (h[b].status == kNumerical) status[b] = kNumerical;
                }
                if (max_outer == 0) {
                    // restart the problems whose pass improved on its start and broke down or met
                    // its target on the recursive residual, from the true residual of their best
                    // iterate (only the true residual certifies); otherwise the next outer pass only
                    // computes the final true residuals
                    bool restart = false;
                    for (int b = 0; b < B; ++b)
                        restart |= status[b] != kNumerical &&
                                   (h[b].status == kBreakdown || h[b].status == kConverged) &&
                                   h[b].rr_best < h[b].rr0 && iters[b] < o.maxit;
                    if (restart && restarts < kMaxRestarts) ++restarts;
                    else restarts = -1;
                }
            }
            k_scatter<<<g, 256, 0, s>>>(xs.as<double>(), P.perm.as<int32_t>(), n, xo);
            IMQ_LAUNCH_CHECK();
            check_device_errors(s);   // synchronises; a wait that ran out invalidates the solve
            double rhs_worst = 0;
            int rhs_iter = 0;
            for (int b = 0; b < B; ++b) {
                rhs_worst = std::max(rhs_worst, rel[b]);
                rhs_iter = std::max(rhs_iter, iters[b]);
                if (status[b] != kConverged) final_status = status[b] == kNumerical ? kNumerical
                                                          : (final_status == kNumerical ? kNumerical : kMaxIter);
                if (rel_out) rel_out[(size_t)rhs * B + b] = rel[b];
                if (iters_out) iters_out[(size_t)rhs * B + b] = iters[b];
            }
            total_iter += rhs_iter;
            worst_rel = std::max(worst_rel, rhs_worst);
            if (info && rhs < IMQ_CG_MAX_RHS_INFO) info->rel_residual[rhs] = rhs_worst;
        }
    }
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        info->iterations = total_iter;
        info->outer_steps = outer_done;
        info->max_rel_residual = worst_rel;
        info->seconds = secs;
        info->status = final_status == kConverged ? IMQ_OK
                                                  : (final_status == kNumerical ? IMQ_NUMERICAL : IMQ_NOT_CONVERGED);
    }
    if (final_status == kNumerical) fail(IMQ_NUMERICAL, "imq_cg_solve: non-finite value or breakdown in CG");
    if (final_status != kConverged)
        fail(IMQ_NOT_CONVERGED, "imq_cg_solve: tolerance not reached; coef holds the best iterate");
}

}  // namespace imq
