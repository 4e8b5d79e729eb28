// Evaluation of the far field at the points of each leaf for a compile-time
// order P, FP32: the local expansion of the leaf (L2P) plus the multipoles of
// its W list (M2P), the two far-field parts of the paper's Algorithm 1
// evaluation (the sum over S_p, Section 3).
//
// L2P.  Lh_n^m(B) against the regular harmonics of w = (x - c_B)/h in the
// plane z = 0: only n + m even survive and R_n^m(w) = norm * |w|^{n-m} conj(w)^m,
// so column m is  Re( conj(w)^m * P_m(|w|^2) )  with a polynomial P_m whose
// complex coefficients are the leaf's local coefficients times eps_m and the
// regular normalisation.  The warp builds these complex coefficients once per
// leaf in its own shared-memory row (read back as broadcasts) and each lane
// evaluates P_m by Horner's rule with packed f32x2 FMAs (real and imaginary
// part in one instruction).
//
// M2P.  For a source S of the W list, G_n^m(x - c_S) with vertical component c
// is G_m^m times a real sequence g_n (g_m = 1) that obeys the normalised
// three-term recurrence in n; column m contributes Re( G_m^m * sum_n g_n Mh_n^m ).
// The recurrence coefficients live in __constant__ memory, so with P fixed
// every coefficient is an operand of the FMA that uses it.  The M2P terms run
// first, one warp per (W entry, 32 points), into per-entry partial sums that
// the L2P kernel adds in W-list order.
#include <cmath>
#include <mutex>
#include <vector>

#include "f32x2.cuh"
#include "fixed_order.cuh"
#include "fmm_common.cuh"
#include <algorithm>

#include "imq_internal.h"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kMaxP = IMQ_MAX_P;
// g_n = A[n][m] * (t a) * g_{n-1} - B[n][m] * a^2 * g_{n-2};  f[m] = sqrt((2m-1)/(2m))
__constant__ float c_rec_a[(kMaxP + 1) * (kMaxP + 1)];
__constant__ float c_rec_b[(kMaxP + 1) * (kMaxP + 1)];
__constant__ float c_fm[kMaxP + 2];

constexpr int kFarWarps = 4;

// M2P of one W-list source S at up to 32 points of a leaf (one lane per point):
// the value of Mh(S) at x, column by column.
template <int P>
__device__ __forceinline__ float m2p_value(const u64 *cm, float vx, float vy, float c2, float c, float hs) {
    const float inv = rsqrtf(vx * vx + vy * vy + c2);
    const float a = hs * inv, t = c * inv;
    const float ta = t * a, a2 = a * a;
    const float zr0 = vx * inv * a, zi0 = vy * inv * a;
    float gr = inv, gi = 0.f;   // G_m^m, from G_0^0
    float acc = 0.f;
#pragma unroll
    for (int m = 0; m <= P; ++m) {
        if (m > 0) {
            const float f = c_fm[m];
            const float nr = (gr * zr0 - gi * zi0) * f;
            gi = (gr * zi0 + gi * zr0) * f;
            gr = nr;
        }
        const int k0 = cbase(P, m);
        u64 sm = cm[k0];   // g_m = 1
        float g1 = 1.f, g2 = 0.f;
#pragma unroll
        for (int n = m + 1; n <= P; ++n) {
            const float g = c_rec_a[n * (kMaxP + 1) + m] * ta * g1 - c_rec_b[n * (kMaxP + 1) + m] * a2 * g2;
            g2 = g1;
            g1 = g;
            if (((n + m) & 1) == 0) sm = fma2(pk2(g, g), cm[k0 + (n - m) / 2], sm);
        }
        float sr, si;
        up2(sm, sr, si);
        const float eps = m ? 2.f : 1.f;
        acc = fmaf(eps, gr * sr - gi * si, acc);
    }
    return acc;
}

// M2P work items, one warp each: item = (target leaf b, W source s, first point i0,
// offset of its 32 partial sums).  Splitting the W lists over warps keeps a leaf
// with a long W list from becoming the kernel's critical path.
template <int P>
__global__ void __launch_bounds__(32 * kFarWarps, 8) k_m2p_t(
    int nitems, const int4 *__restrict__ items, const int32_t *__restrict__ end, const int32_t *__restrict__ level,
    const double2 *__restrict__ centre, const float2 *__restrict__ loc, const float *__restrict__ M, int K, double S,
    ShapeC shape, float *__restrict__ wpart) {
    constexpr int NC = ncplx(P);
    __shared__ __align__(8) u64 s_cm[kFarWarps][NC];
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kFarWarps + wib;
    if (warp >= nitems) return;
    u64 *cm = s_cm[wib];
    const int4 it = items[warp];
    const int b = it.x, s = it.y, i = it.z + lane;
    const float *Ms = M + (int64_t)s * K;
    for (int k = lane; k < NC; k += 32) {
        int m, slot;
        decode_term<P>(k, m, slot);
        cm[k] = pk2(Ms[slot], m ? Ms[slot + 1] : 0.f);
    }
    __syncwarp();
    const float2 lp = i < end[b] ? loc[i] : make_float2(0.f, 0.f);
    const double2 cb = centre[b], cs = centre[s];
    const float c = (float)shape.of(b);
    const float vx = lp.x + (float)(cb.x - cs.x), vy = lp.y + (float)(cb.y - cs.y);
    const float hs = (float)(S / (double)(1 << level[s]));
    wpart[it.w + lane] = m2p_value<P>(cm, vx, vy, c * c, c, hs);
}

// (At most 4 CTAs of 4 warps per SM, 2 from P = 13 on: the unrolled evaluation keeps the leaf's
// coefficients in registers, and a tighter bound spills them to local memory.)
// L2P at the points of each leaf, then the leaf's M2P partial sums added in W-list
// order (the order of a serial loop over the list, so the sum is deterministic),
// then (if given) the point's near-field sum.
template <int P>
__global__ void __launch_bounds__(32 * kFarWarps, (P <= 12 ? 4 : 2)) k_l2p_t(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
    const int32_t *__restrict__ level, const float2 *__restrict__ loc, const int32_t *__restrict__ woff,
    const int32_t *__restrict__ wbase, const float *__restrict__ L, const float *__restrict__ coef, int K, double S,
    const float *__restrict__ wpart, const float *__restrict__ near, float *__restrict__ bs) {
    constexpr int NC = ncplx(P);
    __shared__ __align__(8) u64 s_cl[kFarWarps][NC];   // per-warp L2P coefficients
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int warp = blockIdx.x * kFarWarps + wib;
    if (warp >= nleaf) return;
    u64 *cl = s_cl[wib];
    const int b = leaves[warp];
    const float inv_h = 1.f / (float)(S / (double)(1 << level[b]));
    const float *Lb = L + (int64_t)b * K;

    // complex L2P coefficients of column m, term j: eps_m * norm * (Lr, Li)
    for (int k = lane; k < NC; k += 32) {
        int m, slot;
        decode_term<P>(k, m, slot);
        const float e = (m ? 2.f : 1.f) * coef[slot];
        cl[k] = pk2(e * Lb[slot], m ? e * Lb[slot + 1] : 0.f);
    }
    __syncwarp();

    const int i0 = begin[b], i1 = end[b];
    const int nw = woff[b + 1] - woff[b], nch = (i1 - i0 + 31) >> 5;
    const float *wp = wpart + wbase[warp];
    for (int base = i0, ch = 0; base < i1; base += 32, ++ch) {
        const int i = base + lane;
        const bool act = i < i1;
        const float2 lp = act ? loc[i] : make_float2(0.f, 0.f);
        float phi = 0.f;
        const float ux = lp.x * inv_h, uy = lp.y * inv_h;
        const float r2 = ux * ux + uy * uy;
        const u64 R2 = pk2(r2, r2);
        float zr = 1.f, zi = 0.f;
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            const int k0 = cbase(P, m), J = cnt_col(P, m);
            u64 pm = cl[k0 + J - 1];
#pragma unroll
            for (int j = J - 2; j >= 0; --j) pm = fma2(pm, R2, cl[k0 + j]);
            float pr, pi;
            up2(pm, pr, pi);
            phi = fmaf(zr, pr, fmaf(-zi, pi, phi));
            const float nr = zr * ux + zi * uy;
            zi = zi * ux - zr * uy;
            zr = nr;
        }
        for (int e = 0; e < nw; ++e) phi += wp[((int64_t)e * nch + ch) * 32 + lane];
        if (act) bs[i] = near ? phi + near[i] : phi;
    }
}

}  // namespace

// Host: the M2P item table and each leaf's offset into the partial sums (once per plan).
void ensure_m2p_items(Plan &P, cudaStream_t s) {
    if (P.n_m2p_items >= 0) return;
    const int nl = P.nleaf;
    std::vector<int32_t> leaves(nl), beg(P.nbox), en(P.nbox), woff(P.nbox + 1), witems(std::max<int64_t>(1, P.W.total)),
        utot(P.nbox);
    IMQ_CUDA(cudaMemcpyAsync(utot.data(), P.utot.ptr, 4 * (size_t)P.nbox, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(leaves.data(), P.leaves.ptr, 4 * (size_t)nl, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(beg.data(), P.begin.ptr, 4 * (size_t)P.nbox, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(en.data(), P.end.ptr, 4 * (size_t)P.nbox, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaMemcpyAsync(woff.data(), P.W.off.ptr, 4 * (size_t)(P.nbox + 1), cudaMemcpyDeviceToHost, s));
    if (P.W.total > 0)
        IMQ_CUDA(cudaMemcpyAsync(witems.data(), P.W.items.ptr, 4 * (size_t)P.W.total, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> wbase(nl);
    std::vector<int4> items;
    int64_t off = 0;
    for (int w = 0; w < nl; ++w) {
        const int b = leaves[w];
        const int nch = (en[b] - beg[b] + 31) / 32;
        wbase[w] = (int32_t)off;
        for (int e = woff[b]; e < woff[b + 1]; ++e)
            for (int k = 0; k < nch; ++k) {
                items.push_back(make_int4(b, witems[e], beg[b] + 32 * k, (int32_t)off));
                off += 32;
            }
    }
    if (off > 0x7FFFFFFF) fail(IMQ_UNSUPPORTED, "far field: too many M2P partial sums");
    // the persistent P2P kernel pulls leaves in this order: most pairs first, so the last ones
    // to start are short
    std::vector<int32_t> ord(nl);
    for (int k = 0; k < nl; ++k) ord[k] = k;
    auto pairs = [&](int k) { return (int64_t)(en[leaves[k]] - beg[leaves[k]]) * utot[leaves[k]]; };
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return pairs(a) > pairs(b); });
    P.p2p_order.alloc(4 * (size_t)std::max(1, nl));
    P.p2p_counter.alloc(sizeof(int32_t));
    if (nl > 0) IMQ_CUDA(cudaMemcpyAsync(P.p2p_order.ptr, ord.data(), 4 * (size_t)nl, cudaMemcpyHostToDevice, s));
    P.m2p_items.alloc(sizeof(int4) * std::max<size_t>(1, items.size()));
    P.wbase.alloc(4 * (size_t)std::max(1, nl));
    P.wpart.alloc(4 * (size_t)std::max<int64_t>(32, off));
    if (!items.empty())
        IMQ_CUDA(cudaMemcpyAsync(P.m2p_items.ptr, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, s));
    if (nl > 0) IMQ_CUDA(cudaMemcpyAsync(P.wbase.ptr, wbase.data(), 4 * (size_t)nl, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    P.n_m2p_items = (int)items.size();
}

namespace {

std::vector<int> g_tables_ready;   // per device
std::mutex g_tables_mu;            // plans may be built from several host threads

void upload_tables(cudaStream_t s) {
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_tables_mu);
    if ((int)g_tables_ready.size() <= dev) g_tables_ready.resize(dev + 1, 0);
    if (g_tables_ready[dev]) return;
    std::vector<float> A((kMaxP + 1) * (kMaxP + 1), 0.f), B(A.size(), 0.f), F(kMaxP + 2, 0.f);
    for (int n = 0; n <= kMaxP; ++n)
        for (int m = 0; m <= n; ++m) {
            const double b2 = (double)n * n - (double)m * m;
            if (b2 <= 0) continue;
            const double iv = 1.0 / std::sqrt(b2);
            const double a2 = (double)(n - 1) * (n - 1) - (double)m * m;
            A[n * (kMaxP + 1) + m] = (float)((2 * n - 1) * iv);
            B[n * (kMaxP + 1) + m] = (float)(a2 > 0 ? std::sqrt(a2) * iv : 0.0);
        }
    for (int m = 1; m <= kMaxP; ++m) F[m] = (float)std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_rec_a, A.data(), sizeof(float) * A.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_rec_b, B.data(), sizeof(float) * B.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_fm, F.data(), sizeof(float) * F.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    g_tables_ready[dev] = 1;
}

}  // namespace

bool far_fixed_p_supported(int p) { return p >= 1 && p <= 16; }

void far_fixed_p_prepare(cudaStream_t s) { upload_tables(s); }

void far_m2p_launch(Plan &P, const float *M, cudaStream_t s) {
    ensure_m2p_items(P, s);
    const unsigned gi = (unsigned)((P.n_m2p_items + kFarWarps - 1) / kFarWarps);
    if (gi == 0) return;
#define IMQ_M2P_CASE(PP)                                                                                      \
    case PP:                                                                                                 \
        k_m2p_t<PP><<<gi, 32 * kFarWarps, 0, s>>>(P.n_m2p_items, P.m2p_items.as<int4>(), P.end.as<int32_t>(), \
                                                  P.level.as<int32_t>(), P.centre.as<double2>(),             \
                                                  P.loc.as<float2>(), M, P.layout.K, P.side, P.shape(),      \
                                                  P.wpart.as<float>());                                      \
        break;
    switch (P.p) {
        IMQ_M2P_CASE(1) IMQ_M2P_CASE(2) IMQ_M2P_CASE(3) IMQ_M2P_CASE(4) IMQ_M2P_CASE(5) IMQ_M2P_CASE(6)
        IMQ_M2P_CASE(7) IMQ_M2P_CASE(8) IMQ_M2P_CASE(9) IMQ_M2P_CASE(10) IMQ_M2P_CASE(11) IMQ_M2P_CASE(12)
        IMQ_M2P_CASE(13) IMQ_M2P_CASE(14) IMQ_M2P_CASE(15) IMQ_M2P_CASE(16)
        default: fail(IMQ_UNSUPPORTED, "far field: no fixed-order kernel for this p");
    }
#undef IMQ_M2P_CASE
    IMQ_LAUNCH_CHECK();
}

void far_l2p_launch(Plan &P, const float *L, const float *coef, const float *near, float *b, cudaStream_t s) {
    const unsigned gl = (unsigned)((P.nleaf + kFarWarps - 1) / kFarWarps);
    if (gl == 0) return;
#define IMQ_L2P_CASE(PP)                                                                                        \
    case PP:                                                                                                   \
        k_l2p_t<PP><<<gl, 32 * kFarWarps, 0, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(),      \
                                                  P.end.as<int32_t>(), P.level.as<int32_t>(), P.loc.as<float2>(), \
                                                  P.W.off.as<int32_t>(), P.wbase.as<int32_t>(), L, coef,          \
                                                  P.layout.K, P.side, P.wpart.as<float>(), near, b);             \
        break;
    switch (P.p) {
        IMQ_L2P_CASE(1) IMQ_L2P_CASE(2) IMQ_L2P_CASE(3) IMQ_L2P_CASE(4) IMQ_L2P_CASE(5) IMQ_L2P_CASE(6)
        IMQ_L2P_CASE(7) IMQ_L2P_CASE(8) IMQ_L2P_CASE(9) IMQ_L2P_CASE(10) IMQ_L2P_CASE(11) IMQ_L2P_CASE(12)
        IMQ_L2P_CASE(13) IMQ_L2P_CASE(14) IMQ_L2P_CASE(15) IMQ_L2P_CASE(16)
        default: fail(IMQ_UNSUPPORTED, "far field: no fixed-order kernel for this p");
    }
#undef IMQ_L2P_CASE
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq
