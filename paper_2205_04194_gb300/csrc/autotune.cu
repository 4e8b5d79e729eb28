// Autotuner: choose the truncation order p, the leaf size, the precision of
// the translations and the tile shapes of the FP32 product for a point set.
//
// The paper fixes M (= p) from its a-priori bound (Theorem 2.1 and the worked
// example of Section 2.2) and picks the number of levels L by balancing the
// far-field count against the near-field count (Section 2.3).  On the adaptive
// tree the leaf size plays the role of L, and the bound is pessimistic for the
// M2L-based product, so both are chosen here by measurement: for each leaf
// size the smallest p whose FP32 product meets the target relative 2-norm
// error on a sample of exactly computed rows, then the fastest of those (with
// FP64 translations when no FP32 configuration meets the target); finally the
// tile shapes (P2P warps and target chunk, M2L pipeline depth) of the choice,
// with the paper's cost split (Section 2.3: near field against far field) as
// the reason the leaf size and the P2P tile come first.
//
// Everything runs through the public entry points (imq_plan, imq_plan_batched,
// imq_matvec, imq_plan_destroy); the exact rows are an FP64 direct sum over
// every source of the row's problem.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kRowThreads = 256;
constexpr int kRowsSingle = 2048;   // sampled rows of a single problem
constexpr int kRowsPerProblem = 32; // sampled rows per problem of a batch
constexpr int kTimedReps = 3;

// SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014), mapped to a float in [-1, 1).
__device__ __forceinline__ float splitmix_pm1(uint64_t i) {
    uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0);
}

__global__ void k_fill_pm1(float *__restrict__ v, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = splitmix_pm1((uint64_t)i);
}

// exact[r * S + s] = sum_{j in [lo_s, hi_s)} v[r * N + j] / sqrt(|x_i - x_j|^2 + c_s^2), FP64,
// for sampled row s (point i = row[s]); a fixed reduction tree per block.
__global__ void __launch_bounds__(kRowThreads) k_exact_rows(const double2 *__restrict__ pts, int64_t N,
                                                           const float *__restrict__ v, int nrhs,
                                                           const int64_t *__restrict__ row, const int64_t *__restrict__ lo,
                                                           const int64_t *__restrict__ hi, const double *__restrict__ cs,
                                                           int S, double *__restrict__ exact) {
    __shared__ double sh[kRowThreads];
    const int s = blockIdx.x;
    const double2 xi = pts[row[s]];
    const double c2 = cs[s] * cs[s];
    for (int r = 0; r < nrhs; ++r) {
        const float *vr = v + (int64_t)r * N;
        double acc = 0;
        for (int64_t j = lo[s] + threadIdx.x; j < hi[s]; j += kRowThreads) {
            const double dx = xi.x - pts[j].x, dy = xi.y - pts[j].y;
            acc += (double)vr[j] * rsqrt(dx * dx + dy * dy + c2);
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int off = kRowThreads / 2; off > 0; off >>= 1) {
            if (threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
            __syncthreads();
        }
        if (threadIdx.x == 0) exact[(int64_t)r * S + s] = sh[0];
        __syncthreads();
    }
}

__global__ void k_pick_rows(const float *__restrict__ b, int64_t N, int nrhs, const int64_t *__restrict__ row, int S,
                            float *__restrict__ out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < (int64_t)nrhs * S) {
        const int r = (int)(e / S), s = (int)(e - (int64_t)r * S);
        out[e] = b[(int64_t)r * N + row[s]];
    }
}

void check(imq_status st) {
    if (st != IMQ_OK) fail(st, std::string("imq_autotune: ") + imq_last_error());
}

struct PlanHolder {
    imq_plan_t h = nullptr;
    ~PlanHolder() { imq_plan_destroy(h); }
};

}  // namespace

void autotune(const double *points, const int64_t *offsets, int nprob, const double *cvals, double target,
              const int32_t *p_cand, int n_p, const int32_t *leaf_cand, int n_leaf, int nrhs, const float *v,
              const imq_options *opt, cudaStream_t s, imq_tune_result *out) {
    const int64_t N = offsets ? offsets[nprob] : 0;
    // ---- sampled rows: evenly spaced within each problem, in the caller's order
    std::vector<int64_t> row, lo, hi;
    std::vector<double> cs;
    std::vector<int> prob_of;
    for (int q = 0; q < nprob; ++q) {
        const int64_t a = offsets[q], n = offsets[q + 1] - offsets[q];
        const int64_t m = std::min<int64_t>(n, nprob == 1 ? kRowsSingle : kRowsPerProblem);
        for (int64_t k = 0; k < m; ++k) {
            row.push_back(a + (k * n) / m);
            lo.push_back(a);
            hi.push_back(a + n);
            cs.push_back(cvals[q]);
            prob_of.push_back(q);
        }
    }
    const int S = (int)row.size();
    AsyncMem d_pts(sizeof(double) * 2 * (size_t)N, s), d_v(sizeof(float) * (size_t)nrhs * N, s),
        d_b(sizeof(float) * (size_t)nrhs * N, s), d_row(8 * (size_t)S, s), d_lo(8 * (size_t)S, s),
        d_hi(8 * (size_t)S, s), d_c(8 * (size_t)S, s), d_exact(8 * (size_t)S * nrhs, s),
        d_pick(4 * (size_t)S * nrhs, s);
    IMQ_CUDA(cudaMemcpyAsync(d_pts.ptr, points, sizeof(double) * 2 * (size_t)N, cudaMemcpyDefault, s));
    IMQ_CUDA(cudaMemcpyAsync(d_row.ptr, row.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyAsync(d_lo.ptr, lo.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyAsync(d_hi.ptr, hi.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyAsync(d_c.ptr, cs.data(), 8 * (size_t)S, cudaMemcpyHostToDevice, s));
    if (v) {   // the caller's vectors (host or device)
        IMQ_CUDA(cudaMemcpyAsync(d_v.ptr, v, sizeof(float) * (size_t)nrhs * N, cudaMemcpyDefault, s));
    } else {
        k_fill_pm1<<<blocks_for((int64_t)nrhs * N, 256), 256, 0, s>>>(d_v.as<float>(), (int64_t)nrhs * N);
        IMQ_LAUNCH_CHECK();
    }
    k_exact_rows<<<S, kRowThreads, 0, s>>>(d_pts.as<double2>(), N, d_v.as<float>(), nrhs, d_row.as<int64_t>(),
                                           d_lo.as<int64_t>(), d_hi.as<int64_t>(), d_c.as<double>(), S,
                                           d_exact.as<double>());
    IMQ_LAUNCH_CHECK();
    std::vector<double> exact((size_t)S * nrhs);
    IMQ_CUDA(cudaMemcpyAsync(exact.data(), d_exact.ptr, 8 * exact.size(), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));

    std::vector<int32_t> ps(p_cand, p_cand + n_p);
    std::sort(ps.begin(), ps.end());
    ps.erase(std::unique(ps.begin(), ps.end()), ps.end());
    cudaEvent_t e0, e1;
    IMQ_CUDA(cudaEventCreate(&e0));
    IMQ_CUDA(cudaEventCreate(&e1));
    struct Ev {
        cudaEvent_t a, b;
        ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } ev{e0, e1};
    std::vector<float> picked((size_t)S * nrhs);
    std::memset(out, 0, sizeof(*out));
    imq_options base{};
    if (opt) std::memcpy(&base, opt, std::min(sizeof(base), (size_t)std::max(0, opt->struct_size)));
    base.struct_size = sizeof(imq_options);
    // build one configuration, measure its sampled error and best-of-3 time, record it
    auto measure = [&](int p, int leaf, int trans, int warps, int chunk, int stages, int split) -> int {
        imq_options o = base;
        o.translations = trans;
        o.p2p_warps = warps;
        o.p2p_chunk = chunk;
        o.m2l_stages = stages;
        o.m2l_split = split;
        PlanHolder plan;
        if (nprob == 1)
            check(imq_plan(d_pts.as<double>(), N, cvals[0], p, leaf, &o, s, &plan.h));
        else
            check(imq_plan_batched(d_pts.as<double>(), offsets, nprob, cvals, p, leaf, &o, s, &plan.h));
        check(imq_matvec(plan.h, d_v.ptr, d_b.ptr, nrhs, IMQ_F32, s));   // warm-up, and the error sample
        k_pick_rows<<<blocks_for((int64_t)S * nrhs, 256), 256, 0, s>>>(d_b.as<float>(), N, nrhs,
                                                                       d_row.as<int64_t>(), S, d_pick.as<float>());
        IMQ_LAUNCH_CHECK();
        IMQ_CUDA(cudaMemcpyAsync(picked.data(), d_pick.ptr, 4 * picked.size(), cudaMemcpyDeviceToHost, s));
        float best_ms = INFINITY;
        for (int rep = 0; rep < kTimedReps; ++rep) {
            IMQ_CUDA(cudaEventRecord(e0, s));
            check(imq_matvec(plan.h, d_v.ptr, d_b.ptr, nrhs, IMQ_F32, s));
            IMQ_CUDA(cudaEventRecord(e1, s));
            IMQ_CUDA(cudaEventSynchronize(e1));
            float ms = 0;
            IMQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            best_ms = std::min(best_ms, ms);
        }
        // relative 2-norm error over the sampled rows, per problem and right-hand side; the worst
        std::vector<double> num((size_t)nprob * nrhs, 0.0), den((size_t)nprob * nrhs, 0.0);
        for (int r = 0; r < nrhs; ++r)
            for (int k = 0; k < S; ++k) {
                const double e = exact[(size_t)r * S + k], d = (double)picked[(size_t)r * S + k] - e;
                num[(size_t)r * nprob + prob_of[k]] += d * d;
                den[(size_t)r * nprob + prob_of[k]] += e * e;
            }
        double err = 0;
        for (size_t k = 0; k < num.size(); ++k)
            err = std::max(err, den[k] > 0 ? std::sqrt(num[k] / den[k]) : std::sqrt(num[k]));
        if (out->n_tried >= IMQ_TUNE_MAX_TRIED) return -1;
        imq_tune_entry &t = out->tried[out->n_tried];
        t = imq_tune_entry{};
        t.p = p;
        t.leaf = leaf;
        t.rel_err = err;
        t.matvec_ms = best_ms;
        t.translations = trans;
        t.p2p_warps = warps;
        t.p2p_chunk = chunk;
        t.m2l_stages = stages;
        t.m2l_split = split;
        return out->n_tried++;
    };
    // 1-2: the smallest p meeting the target per leaf size, FP32 translations first
    auto search = [&](int trans) {
        bool any = false;
        for (int li = 0; li < n_leaf; ++li)
            for (int p : ps) {
                if (trans != IMQ_TRANS_FP32 && p > 16) continue;
                const int k = measure(p, leaf_cand[li], trans, 0, 0, 0, 0);
                if (k < 0) return any;
                if (out->tried[k].rel_err <= target) {
                    any = true;
                    break;
                }
            }
        return any;
    };
    bool met = search(IMQ_TRANS_FP32);
    if (!met && ps.front() <= 16) met = search(IMQ_TRANS_MIXED);
    if (!met && ps.front() <= 16) met = search(IMQ_TRANS_FP64);
    // the fastest configuration that meets the target, else the most accurate one
    auto pick = [&](int from) {
        int best = -1;
        for (int k = from; k < out->n_tried; ++k) {
            const imq_tune_entry &t = out->tried[k];
            if (t.rel_err > target) continue;
            if (best < 0 || t.matvec_ms < out->tried[best].matvec_ms) best = k;
        }
        return best;
    };
    int best = pick(0);
    out->met = best >= 0 ? 1 : 0;
    if (best < 0)
        for (int k = 0; k < out->n_tried; ++k)
            if (best < 0 || out->tried[k].rel_err < out->tried[best].rel_err) best = k;
    // 3: tile shapes of the chosen configuration, P2P first, then the M2L pipeline depth
    const imq_tune_entry chosen = out->tried[best];
    const double err_cap = out->met ? target : chosen.rel_err * 1.01;
    auto better = [&](int k, int cur) {
        return k >= 0 && out->tried[k].rel_err <= err_cap && out->tried[k].matvec_ms < out->tried[cur].matvec_ms;
    };
    int cur = best;
    for (int warps : {2, 4, 8})
        for (int chunk : {8, 16, 32}) {
            const int k = measure(chosen.p, chosen.leaf, chosen.translations, warps, chunk, 0, 0);
            if (better(k, cur)) cur = k;
        }
    const int K = (chosen.p + 1) * (chosen.p + 2) / 2;   // reals of the parity-reduced expansion
    const bool tensor = chosen.translations != IMQ_TRANS_FP64 && (!opt || opt->m2l_kernel != IMQ_M2L_CUDA_CORES) &&
                        m2l_umma_supported(K, K);
    if (tensor) {
        const int smax = m2l_umma_max_stages(K, K);
        const imq_tune_entry tp = out->tried[cur];
        for (int stages = m2l_umma_min_stages(); stages <= smax; ++stages) {
            const int k =
                measure(chosen.p, chosen.leaf, chosen.translations, tp.p2p_warps, tp.p2p_chunk, stages, 0);
            if (better(k, cur)) cur = k;
        }
        const imq_tune_entry ts = out->tried[cur];
        for (int split = 1; split <= 4; ++split) {
            const int k = measure(chosen.p, chosen.leaf, chosen.translations, ts.p2p_warps, ts.p2p_chunk,
                                  ts.m2l_stages, split);
            if (better(k, cur)) cur = k;
        }
    }
    const imq_tune_entry &w = out->tried[cur];
    out->p = w.p;
    out->leaf = w.leaf;
    out->rel_err = w.rel_err;
    out->matvec_ms = w.matvec_ms;
    out->translations = w.translations;
    out->p2p_warps = w.p2p_warps;
    out->p2p_chunk = w.p2p_chunk;
    out->m2l_stages = w.m2l_stages;
    out->m2l_split = w.m2l_split;
    out->sampled_rows = S;
    check_device_errors(s);   // a bounded wait that ran out would invalidate the measured errors
}

}  // namespace imq
