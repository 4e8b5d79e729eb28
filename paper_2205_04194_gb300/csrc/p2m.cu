// P2M and P2L for a compile-time order P, FP32.
//
// P2M: the multipole moments of each leaf
// (the paper's moments v_k, w_k of a block, Section 3, Algorithm 1, in the
// solid-harmonic form of Eq. (8)): with w = (y_j - c_B)/h in the plane,
//   Mh_n^m(B) = norm_n^m * sum_j u_j conj(w_j)^m |w_j|^{n-m},   n + m even.
// One warp per leaf, one lane per point: each lane forms the complex moments
// of its points in registers (conj(w)^m by repeated multiplication, |w|^2 powers
// down each column, packed f32x2 arithmetic), and a butterfly transpose-
// reduction over the 32 lanes leaves lane L with the sums of complex terms
// q L .. q L + q - 1 (q = padded terms / 32), which it scales and stores.
// The summation order is fixed, so the result is deterministic.
//
// P2L (X list): the local coefficients of a box B from the points of the small
// leaves of its X list,  Lh_n^m(B) += sum_j u_j G_n^m(y_j - c_B)  with vertical
// component -c.  G_n^m = g_n G_m^m with the real three-term recurrence of the
// M2P evaluation, so each term costs one packed FMA on u_j G_m^m; lanes take
// the concatenated source points of the X entries and the same butterfly
// reduction closes the warp.
#include <cmath>
#include <mutex>
#include <vector>

#include "f32x2.cuh"
#include "fixed_order.cuh"
#include "fmm_common.cuh"
#include "imq_internal.h"
#include "umma.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kP2MWarps = 4;

template <int N>
__device__ __forceinline__ void butterfly_reduce(u64 (&v)[N], int lane) {
    static_assert(N % 32 == 0, "padded to a multiple of the warp");
    // stage with xor offset o keeps the lower or upper half of the live values
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int o = 16 >> st;
        const int live = N >> st, half = live >> 1;
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const u64 keep = up ? v[k + half] : v[k];
            const u64 send = up ? v[k] : v[k + half];
            v[k] = add2(keep, __shfl_xor_sync(0xFFFFFFFFu, send, o));
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32 * kP2MWarps) k_p2m_t(int nleaf, const int32_t *__restrict__ leaves,
                                                          const int32_t *__restrict__ begin,
                                                          const int32_t *__restrict__ end,
                                                          const int32_t *__restrict__ level,
                                                          const float2 *__restrict__ loc, const float *__restrict__ u,
                                                          float *__restrict__ M, int K,
                                                          const float *__restrict__ coef, double S,
                                                          float *__restrict__ Mpk, int KP) {
    constexpr int NC = ncplx(P);
    constexpr int NP = (NC + 31) / 32 * 32;
    constexpr int Q = NP / 32;
    const int warp = blockIdx.x * kP2MWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (warp >= nleaf) return;
    const int b = leaves[warp];
    const float inv_h = 1.f / (float)(S / (double)(1 << level[b]));
    u64 acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0ull;
    const int i0 = begin[b], i1 = end[b];
    for (int base = i0; base < i1; base += 32) {
        const int i = base + lane;
        const bool act = i < i1;
        const float2 lp = act ? loc[i] : make_float2(0.f, 0.f);
        const float uj = act ? u[i] : 0.f;
        const float wx = lp.x * inv_h, wy = lp.y * inv_h;
        const float r2 = wx * wx + wy * wy;
        const u64 R2 = pk2(r2, r2);
        float zr = uj, zi = 0.f;   // u conj(w)^m
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            u64 q = pk2(zr, zi);
#pragma unroll
            for (int j = 0; j < cnt_col(P, m); ++j) {
                acc[cbase(P, m) + j] = add2(acc[cbase(P, m) + j], q);
                if (j + 1 < cnt_col(P, m)) q = mul2(q, R2);
            }
            const float nr = zr * wx + zi * wy;
            zi = zi * wx - zr * wy;
            zr = nr;
        }
    }
    butterfly_reduce<NP>(acc, lane);
    float *Mb = M + (int64_t)b * K;
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int idx = Q * lane + k;
        if (idx >= NC) continue;
        int m, slot;
        decode_term<P>(idx, m, slot);
        float re, im;
        up2(acc[k], re, im);
        const float cc = coef[slot];
        const float vr = cc * re, vi = cc * im;
        Mb[slot] = vr;
        if (m > 0) Mb[slot + 1] = vi;
        mx = fmaxf(mx, fmaxf(fabsf(vr), m > 0 ? fabsf(vi) : 0.f));
    }
    if (!Mpk) return;
    // the scaled fp16 hi / lo rows the tensor-core M2L gathers, scale from the box's largest term
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    const int e = m2l_pow2_exp(mx);
    const float sc = pow2f(e);
    __half *pk = reinterpret_cast<__half *>(Mpk) + (int64_t)b * 2 * KP;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int idx = Q * lane + k;
        if (idx >= NC) continue;
        int m, slot;
        decode_term<P>(idx, m, slot);
        float re, im;
        up2(acc[k], re, im);
        const float cc = coef[slot];
        __half hi, lo;
        f16_split(cc * re * sc, hi, lo);
        pk[slot] = hi;
        pk[KP + slot] = lo;
        if (m > 0) {
            f16_split(cc * im * sc, hi, lo);
            pk[slot + 1] = hi;
            pk[KP + slot + 1] = lo;
        }
    }
    if (lane == 0) *reinterpret_cast<float *>(pk + m2l_scale_slot(K)) = pow2f(-e);
}

constexpr int kP2LWarps = 4;
constexpr int kMaxPT = IMQ_MAX_P;
__constant__ float c_p2l_a[(kMaxPT + 1) * (kMaxPT + 1)];   // (2n-1)/sqrt(n^2-m^2)
__constant__ float c_p2l_b[(kMaxPT + 1) * (kMaxPT + 1)];   // sqrt((n-1)^2-m^2)/sqrt(n^2-m^2)
__constant__ float c_p2l_f[kMaxPT + 2];                    // sqrt((2m-1)/(2m))

template <int P>
__global__ void __launch_bounds__(32 * kP2LWarps) k_p2l_t(
    int nxb, const int32_t *__restrict__ xboxes, const int32_t *__restrict__ xoff, const int32_t *__restrict__ xitems,
    const int32_t *__restrict__ xcum, const int32_t *__restrict__ xtot, const int32_t *__restrict__ begin,
    const int32_t *__restrict__ level, const double2 *__restrict__ centre, const float2 *__restrict__ loc,
    const float *__restrict__ u, float *__restrict__ L, int K, double S, ShapeC shape) {
    constexpr int NC = ncplx(P);
    constexpr int NP = (NC + 31) / 32 * 32;
    constexpr int Q = NP / 32;
    const int warp = blockIdx.x * kP2LWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (warp >= nxb) return;
    const int b = xboxes[warp];
    const float h = (float)(S / (double)(1 << level[b]));
    const double2 cb = centre[b];
    const float c = (float)shape.of(b);
    const int x0 = xoff[b], x1 = xoff[b + 1], St = xtot[b];
    u64 acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0ull;
    int r = x0;
    for (int base = 0; base < St; base += 32) {
        const int q = base + lane;
        const bool act = q < St;
        float vx = 0.f, vy = 1.f, uj = 0.f;
        if (act) {
            while (r + 1 < x1 && xcum[r + 1] <= q) ++r;
            const int sb = xitems[r];
            const int j = begin[sb] + (q - xcum[r]);
            const double2 cs = centre[sb];
            const float2 lp = loc[j];
            vx = lp.x + (float)(cs.x - cb.x);
            vy = lp.y + (float)(cs.y - cb.y);
            uj = u[j];
        }
        const float inv = rsqrtf(vx * vx + vy * vy + c * c);
        const float a = h * inv, t = -c * inv;
        const float ta = t * a, a2 = a * a;
        const float zr0 = vx * inv * a, zi0 = vy * inv * a;
        float gr = inv * uj, gi = 0.f;   // u_j G_m^m, from u_j G_0^0
#pragma unroll
        for (int m = 0; m <= P; ++m) {
            if (m > 0) {
                const float f = c_p2l_f[m];
                const float nr = (gr * zr0 - gi * zi0) * f;
                gi = (gr * zi0 + gi * zr0) * f;
                gr = nr;
            }
            const u64 G = pk2(gr, gi);
            acc[cbase(P, m)] = add2(acc[cbase(P, m)], G);
            float g1 = 1.f, g2 = 0.f;
#pragma unroll
            for (int n = m + 1; n <= P; ++n) {
                const float g = c_p2l_a[n * (kMaxPT + 1) + m] * ta * g1 - c_p2l_b[n * (kMaxPT + 1) + m] * a2 * g2;
                g2 = g1;
                g1 = g;
                if (((n - m) & 1) == 0) acc[cbase(P, m) + (n - m) / 2] = fma2(pk2(g, g), G, acc[cbase(P, m) + (n - m) / 2]);
            }
        }
    }
    butterfly_reduce<NP>(acc, lane);
    float *Lb = L + (int64_t)b * K;
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        const int idx = Q * lane + k;
        if (idx >= NC) continue;
        int m, slot;
        decode_term<P>(idx, m, slot);
        float re, im;
        up2(acc[k], re, im);
        Lb[slot] += re;
        if (m > 0) Lb[slot + 1] += im;
    }
}

std::vector<int> g_p2l_tables;   // per device
std::mutex g_p2l_mu;             // plans may be built from several host threads

}  // namespace

bool p2m_fixed_p_supported(int p) { return p >= 1 && p <= 16; }

void p2l_fixed_p_prepare(cudaStream_t s) {
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_p2l_mu);
    if ((int)g_p2l_tables.size() <= dev) g_p2l_tables.resize(dev + 1, 0);
    if (g_p2l_tables[dev]) return;
    std::vector<float> A((kMaxPT + 1) * (kMaxPT + 1), 0.f), B(A.size(), 0.f), F(kMaxPT + 2, 0.f);
    for (int n = 0; n <= kMaxPT; ++n)
        for (int m = 0; m <= n; ++m) {
            const double b2 = (double)n * n - (double)m * m;
            if (b2 <= 0) continue;
            const double iv = 1.0 / std::sqrt(b2);
            const double a2 = (double)(n - 1) * (n - 1) - (double)m * m;
            A[n * (kMaxPT + 1) + m] = (float)((2 * n - 1) * iv);
            B[n * (kMaxPT + 1) + m] = (float)(a2 > 0 ? std::sqrt(a2) * iv : 0.0);
        }
    for (int m = 1; m <= kMaxPT; ++m) F[m] = (float)std::sqrt((2.0 * m - 1.0) / (2.0 * m));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_p2l_a, A.data(), sizeof(float) * A.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_p2l_b, B.data(), sizeof(float) * B.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaMemcpyToSymbolAsync(c_p2l_f, F.data(), sizeof(float) * F.size(), 0, cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    g_p2l_tables[dev] = 1;
}

void p2l_fixed_p_launch(const Plan &P, const float *u, float *L, cudaStream_t s) {
    const unsigned grid = (unsigned)((P.nxbox + kP2LWarps - 1) / kP2LWarps);
    if (grid == 0 || P.X.total == 0) return;
#define IMQ_P2L_CASE(PP)                                                                                           \
    case PP:                                                                                                      \
        k_p2l_t<PP><<<grid, 32 * kP2LWarps, 0, s>>>(P.nxbox, P.xboxes.as<int32_t>(), P.X.off.as<int32_t>(),       \
                                                    P.X.items.as<int32_t>(), P.xcum.as<int32_t>(),                \
                                                    P.xtot.as<int32_t>(), P.begin.as<int32_t>(),                  \
                                                    P.level.as<int32_t>(), P.centre.as<double2>(),                \
                                                    P.loc.as<float2>(), u, L, P.layout.K, P.side, P.shape());    \
        break;
    switch (P.p) {
        IMQ_P2L_CASE(1)
        IMQ_P2L_CASE(2)
        IMQ_P2L_CASE(3)
        IMQ_P2L_CASE(4)
        IMQ_P2L_CASE(5)
        IMQ_P2L_CASE(6)
        IMQ_P2L_CASE(7)
        IMQ_P2L_CASE(8)
        IMQ_P2L_CASE(9)
        IMQ_P2L_CASE(10)
        IMQ_P2L_CASE(11)
        IMQ_P2L_CASE(12)
        IMQ_P2L_CASE(13)
        IMQ_P2L_CASE(14)
        IMQ_P2L_CASE(15)
        IMQ_P2L_CASE(16)
        default: fail(IMQ_UNSUPPORTED, "P2L: no fixed-order kernel for this p");
    }
#undef IMQ_P2L_CASE
    IMQ_LAUNCH_CHECK();
}

void p2m_fixed_p_launch(const Plan &P, const float *u, float *M, const float *coef, cudaStream_t s, float *Mpk,
                        int KP) {
    const unsigned grid = (unsigned)((P.nleaf + kP2MWarps - 1) / kP2MWarps);
    if (grid == 0) return;
#define IMQ_P2M_CASE(PP)                                                                                          \
    case PP:                                                                                                     \
        k_p2m_t<PP><<<grid, 32 * kP2MWarps, 0, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(),      \
                                                    P.end.as<int32_t>(), P.level.as<int32_t>(),                  \
                                                    P.loc.as<float2>(), u, M, P.layout.K, coef, P.side, Mpk, KP); \
        break;
    switch (P.p) {
        IMQ_P2M_CASE(1)
        IMQ_P2M_CASE(2)
        IMQ_P2M_CASE(3)
        IMQ_P2M_CASE(4)
        IMQ_P2M_CASE(5)
        IMQ_P2M_CASE(6)
        IMQ_P2M_CASE(7)
        IMQ_P2M_CASE(8)
        IMQ_P2M_CASE(9)
        IMQ_P2M_CASE(10)
        IMQ_P2M_CASE(11)
        IMQ_P2M_CASE(12)
        IMQ_P2M_CASE(13)
        IMQ_P2M_CASE(14)
        IMQ_P2M_CASE(15)
        IMQ_P2M_CASE(16)
        default: fail(IMQ_UNSUPPORTED, "P2M: no fixed-order kernel for this p");
    }
#undef IMQ_P2M_CASE
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq
