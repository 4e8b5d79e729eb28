// Gradient of a held-out validation loss of the IMQ interpolant.
//
// The interpolant of the paper's Eq. (2), P(t) = sum_j coef_j phi_c(|t - x_j|),
// has coefficients solving A(c) coef = f (Eq. (4)).  For validation points
// t_k with values y_k, L = mean_k (P(t_k) - y_k)^2, P = E(c) coef.  With
// g = (2/N_v)(P - y) and, A being symmetric, lambda = A^{-1} E^T g:
//     dL/df = lambda,   dL/dc = g . (dE/dc coef) - lambda . (dA/dc coef).
// Every product runs on the library's kernels: two CG solves on the training
// plan, evaluation / transpose / c-derivative on the evaluation plan (nodes
// and validation targets in one tree), the c-derivative product on the
// training plan, and deterministic dots.
#include <cmath>
#include <cstring>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

__global__ void k_loss_terms(const double *__restrict__ P, const double *__restrict__ y, int64_t n, double scale,
                             double *__restrict__ diff, double *__restrict__ g) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const double d = P[i] - y[i];
        diff[i] = d;
        g[i] = scale * d;
    }
}

__global__ void k_cast_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (float)a[i];
}

__global__ void k_cast_f64(const float *__restrict__ a, double *__restrict__ b, int64_t n) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = (double)a[i];
}

}  // namespace
}  // namespace imq

struct imq_plan_s {
    imq::Plan P;
};

using namespace imq;

extern "C" imq_status imq_evaluate(imq_plan_t, const void *, void *, int, imq_dtype, void *);
extern "C" imq_status imq_evaluate_transpose(imq_plan_t, const void *, void *, int, imq_dtype, void *);
extern "C" imq_status imq_evaluate_dc(imq_plan_t, const void *, void *, int, imq_dtype, void *);
extern "C" imq_status imq_matvec_dc(imq_plan_t, const void *, void *, int, imq_dtype, void *);
extern "C" imq_status imq_cg_solve(imq_plan_t, const double *, double *, int, const imq_cg_options *,
                                   imq_cg_info *, void *);
extern "C" const char *imq_last_error(void);

static void ok_or_throw(imq_status st) {
    if (st != IMQ_OK) fail(st, imq_last_error());
}

// a solve that stops at the iteration cap still leaves its best iterate: carry on, report at the end
static void solve_or_flag(imq_status st, bool &not_converged) {
    if (st == IMQ_NOT_CONVERGED || st == IMQ_NUMERICAL) not_converged = true;
    else ok_or_throw(st);
}

extern "C" imq_status imq_interp_loss_grad(imq_plan_t train, imq_plan_t eval, const double *f, const double *y,
                                           const imq_cg_options *opt, imq_dtype dt, double *loss,
                                           double *dloss_dc, double *dloss_df, double *coef_out,
                                           imq_cg_info *info, void *stream) {
    return guarded_call([&] {
        if (!train || !eval || !f || !y || !loss || !dloss_dc) fail(IMQ_INVALID_ARG, "imq_interp_loss_grad: NULL pointer");
        if (dt != IMQ_F32 && dt != IMQ_F64) fail(IMQ_INVALID_ARG, "imq_interp_loss_grad: unknown dtype");
        Plan &T = train->P, &E = eval->P;
        if (E.n_nodes != T.N) fail(IMQ_INVALID_ARG, "imq_interp_loss_grad: eval plan nodes != training points");
        if (E.c != T.c) fail(IMQ_INVALID_ARG, "imq_interp_loss_grad: plans have different c");
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int64_t n = T.N, nv = E.N - E.n_nodes;
        DevMem df, dy, coef, P, diff, g, etg, lam, dec, dac, P32, tmp32;
        df.alloc(8 * n); dy.alloc(8 * nv); coef.alloc(8 * n); P.alloc(8 * nv); diff.alloc(8 * nv); g.alloc(8 * nv);
        etg.alloc(8 * n); lam.alloc(8 * n); dec.alloc(8 * nv); dac.alloc(8 * n);
        IMQ_CUDA(cudaMemcpyAsync(df.ptr, f, 8 * n, cudaMemcpyDefault, s));
        IMQ_CUDA(cudaMemcpyAsync(dy.ptr, y, 8 * nv, cudaMemcpyDefault, s));
        imq_cg_info i1{}, i2{};
        // forward: coef = A^{-1} f, P = E coef
        bool unconverged = false;
        solve_or_flag(imq_cg_solve(train, df.as<double>(), coef.as<double>(), 1, opt, &i1, s), unconverged);
        // products in the requested precision (FP32 products take FP32 vectors)
        auto product = [&](auto fn, imq_plan_t pl, const double *in, int64_t nin, double *out, int64_t nout) {
            if (dt == IMQ_F64) {
                ok_or_throw(fn(pl, in, out, 1, IMQ_F64, s));
            } else {
                DevMem fi, fo;
                fi.alloc(4 * nin);
                fo.alloc(4 * nout);
                k_cast_f32<<<blocks_for(nin, 256), 256, 0, s>>>(in, fi.as<float>(), nin);
                IMQ_LAUNCH_CHECK();
                ok_or_throw(fn(pl, fi.ptr, fo.ptr, 1, IMQ_F32, s));
                k_cast_f64<<<blocks_for(nout, 256), 256, 0, s>>>(fo.as<float>(), out, nout);
                IMQ_LAUNCH_CHECK();
                IMQ_CUDA(cudaStreamSynchronize(s));
            }
        };
        product(imq_evaluate, eval, coef.as<double>(), n, P.as<double>(), nv);
        k_loss_terms<<<blocks_for(nv, 256), 256, 0, s>>>(P.as<double>(), dy.as<double>(), nv, 2.0 / (double)nv,
                                                         diff.as<double>(), g.as<double>());
        IMQ_LAUNCH_CHECK();
        *loss = device_dot(diff.as<double>(), diff.as<double>(), nv, s) / (double)nv;
        // adjoint: lambda = A^{-1} E^T g
        product(imq_evaluate_transpose, eval, g.as<double>(), nv, etg.as<double>(), n);
        solve_or_flag(imq_cg_solve(train, etg.as<double>(), lam.as<double>(), 1, opt, &i2, s), unconverged);
        // dL/dc = g . (dE/dc coef) - lambda . (dA/dc coef)
        product(imq_evaluate_dc, eval, coef.as<double>(), n, dec.as<double>(), nv);
        product(imq_matvec_dc, train, coef.as<double>(), n, dac.as<double>(), n);
        *dloss_dc = device_dot(g.as<double>(), dec.as<double>(), nv, s) -
                    device_dot(lam.as<double>(), dac.as<double>(), n, s);
        if (dloss_df) IMQ_CUDA(cudaMemcpyAsync(dloss_df, lam.ptr, 8 * n, cudaMemcpyDefault, s));
        if (coef_out) IMQ_CUDA(cudaMemcpyAsync(coef_out, coef.ptr, 8 * n, cudaMemcpyDefault, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        if (info) {
            *info = i1;
            info->iterations = i1.iterations + i2.iterations;
            info->max_rel_residual = std::max(i1.max_rel_residual, i2.max_rel_residual);
            info->seconds = i1.seconds + i2.seconds;
        }
        if (unconverged)
            fail(IMQ_NOT_CONVERGED, "imq_interp_loss_grad: a CG solve stopped at its cap; outputs use its best iterate");
    });
}
