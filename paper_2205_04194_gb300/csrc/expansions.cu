// FMM kernels of the fast IMQ product on the adaptive quadtree.
//
// Paper Section 2.2 (Eq. (11)-(13), Algorithm 1): the moments v_k, w_k of a
// block about its centre are the multipole coefficients (P2M); the far-field
// evaluation d h [sin v + cos w] at the points of S_p is the multipole
// evaluated at a target (M2P); the near field on NS_p is the direct sum (P2P,
// p2p.cu).  The fast-multipole translations (M2M, M2L, L2L, L2P, P2L) move
// the same expansions between boxes so that each target evaluates one local
// expansion instead of one multipole per well-separated box.
//
// Coefficient layout and scaling: see imq_internal.h.  Every kernel is a
// template over the arithmetic type (float: the FP32 path, with point
// coordinates stored as FP32 offsets from their leaf centre; double: the FP64
// path on absolute FP64 coordinates).
#include <algorithm>
#include <type_traits>

#include "fmm_common.cuh"
#include "imq_internal.h"
#include "ptx.cuh"
#include "umma.cuh"
#include "util.cuh"

namespace imq {
namespace {

// ------------------------------------------------------------------ gather / scatter
template <class Tin, class T>
__global__ void k_gather(const Tin *__restrict__ v, const int32_t *__restrict__ perm, int64_t n, T *__restrict__ us) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) us[i] = (T)v[perm[i]];
}

template <class T, class Tout>
__global__ void k_scatter(const T *__restrict__ bs, const int32_t *__restrict__ perm, int64_t n, Tout *__restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[perm[i]] = (Tout)bs[i];
}

// ------------------------------------------------------------------ FP32 <-> FP64 expansion copies
// (the FP32 product with FP64 translations: P2M / P2L / L2P in FP32, M2M / M2L / L2L in FP64)
__global__ void k_widen(const float *__restrict__ a, double *__restrict__ b, int64_t n, int add) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = add ? b[i] + (double)a[i] : (double)a[i];
}
__global__ void k_narrow(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

// ------------------------------------------------------------------ P2M
// Mh_n^m = Ptilde_n^m(0) sum_j u_j conj(w_j)^m |w_j|^{n-m},  w_j = (y_j - z_B)/h_B.
template <class T>
__global__ void k_p2m(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin,
                      const int32_t *__restrict__ end, const int32_t *__restrict__ level,
                      const double2 *__restrict__ centre, const float2 *__restrict__ loc,
                      const double2 *__restrict__ pos, const T *__restrict__ u, T *__restrict__ M, int K, int p,
                      const T *__restrict__ coef, double S) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nleaf || lane > p) return;
    const int b = leaves[warp];
    const int m = lane;
    const T inv_h = (T)1 / box_side<T>(S, level[b]);
    const double2 cb = centre[b];
    T ar[kMaxCol], ai[kMaxCol];
#pragma unroll
    for (int k = 0; k < kMaxCol; ++k) ar[k] = ai[k] = 0;
    for (int j = begin[b]; j < end[b]; ++j) {
        T wx, wy;
        point_offset<T>(j, loc, pos, cb, cb, wx, wy);
        wx *= inv_h;
        wy *= inv_h;
        const T uj = u[j];
        T zr = uj, zi = 0;
        for (int t = 0; t < m; ++t) {   // u * conj(w)^m
            const T nr = zr * wx + zi * wy;
            zi = zi * wx - zr * wy;
            zr = nr;
        }
        const T r2 = wx * wx + wy * wy;
#pragma unroll
        for (int k = 0; k < kMaxCol; ++k) {
            if (m + 2 * k <= p) {
                ar[k] += zr;
                ai[k] += zi;
                zr *= r2;
                zi *= r2;
            }
        }
    }
    int slot = col_base(m, p);
    T *Mb = M + (int64_t)b * K;
#pragma unroll
    for (int k = 0; k < kMaxCol; ++k) {
        if (m + 2 * k <= p) {
            const T cc = coef[slot];
            Mb[slot] = cc * ar[k];
            if (m > 0) Mb[slot + 1] = cc * ai[k];
            slot += m ? 2 : 1;
        }
    }
}

// ------------------------------------------------------------------ M2M / L2L
// M2M and L2L (in-plane translations between a box and its four children,
// level-independent operators [q][i][o] in the scaled layout), over the
// internal boxes of one level.  A CTA takes 8 parents; warp q owns child
// quadrant q, and lane t owns outputs t + 32 r (r < RC) for all 8 boxes, so per
// input row a lane loads RC operator values (coalesced, reused for 8 boxes)
// and 8 staged inputs (two vector shared loads) for 8 RC FMAs, and the
// reduction chain is K rows long.  Operator rows are fetched kTransUnroll at a
// time with every load issued before the FMAs.  M2M sums the four quadrant
// partials in a fixed order; L2L adds warp q's result into child q.
constexpr int kTransG = 8;        // parents per CTA
constexpr int kTransUnroll = 4;   // operator rows in flight per step

template <class T>
__device__ __forceinline__ void lds8(const T *p, T (&v)[8]) {
    if constexpr (sizeof(T) == 4) {
        const float4 a = reinterpret_cast<const float4 *>(p)[0], b = reinterpret_cast<const float4 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const double2 a = reinterpret_cast<const double2 *>(p)[k];
            v[2 * k] = a.x;
            v[2 * k + 1] = a.y;
        }
    }
}

// acc[g][r] = sum_{i < K} A[i][lane + 32 r] * X[i][g]   (A: K x K row-major, X: K x 8)
template <class T, int RC>
__device__ __forceinline__ void trans_rows(const T *__restrict__ A, const T *X, int K, int lane, T (&acc)[8][RC]) {
#pragma unroll
    for (int g = 0; g < 8; ++g)
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[g][r] = 0;
    bool okr[RC];
#pragma unroll
    for (int r = 0; r < RC; ++r) okr[r] = lane + 32 * r < K;
    for (int i0 = 0; i0 < K; i0 += kTransUnroll) {
        T wv[kTransUnroll][RC];
#pragma unroll
        for (int u = 0; u < kTransUnroll; ++u)
#pragma unroll
            for (int r = 0; r < RC; ++r)
                wv[u][r] = (okr[r] && i0 + u < K) ? __ldg(A + (int64_t)(i0 + u) * K + lane + 32 * r) : (T)0;
#pragma unroll
        for (int u = 0; u < kTransUnroll; ++u) {
            if (i0 + u >= K) break;
            T mv[8];
            lds8<T>(X + (size_t)(i0 + u) * kTransG, mv);
#pragma unroll
            for (int g = 0; g < 8; ++g)
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[g][r] += wv[u][r] * mv[g];
        }
    }
}

// M(parent) = sum_q T_q M(child q)
template <class T, int RC>
__global__ void __launch_bounds__(128) k_m2m(const int32_t *__restrict__ parents, int n,
                                             const int32_t *__restrict__ child, T *__restrict__ M,
                                             const T *__restrict__ op, int K) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Mc = reinterpret_cast<T *>(smraw);          // [4][K][8]
    T *red = Mc + (size_t)4 * K * kTransG;           // [4][8][K]
    __shared__ int s_ch[kTransG * 4], s_par[kTransG];
    const int p0 = blockIdx.x * kTransG;
    const int ng = min(kTransG, n - p0);
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kTransG * 4) {
        const int g = threadIdx.x >> 2;
        const int pb = g < ng ? parents[p0 + g] : -1;
        s_ch[threadIdx.x] = pb >= 0 ? child[4 * pb + (threadIdx.x & 3)] : -1;
        if ((threadIdx.x & 3) == 0) s_par[g] = pb;
    }
    __syncthreads();
    {   // warp q stages child q of the 8 parents: all loads first, then the shared stores
        T v[kTransG][RC];
#pragma unroll
        for (int g = 0; g < kTransG; ++g) {
            const int ch = s_ch[4 * g + q];
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int i = lane + 32 * r;
                v[g][r] = (ch >= 0 && i < K) ? M[(int64_t)ch * K + i] : (T)0;
            }
        }
#pragma unroll
        for (int g = 0; g < kTransG; ++g)
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int i = lane + 32 * r;
                if (i < K) Mc[((size_t)q * K + i) * kTransG + g] = v[g][r];
            }
    }
    __syncwarp();
    T acc[8][RC];
    trans_rows<T, RC>(op + (int64_t)q * K * K, Mc + (size_t)q * K * kTransG, K, lane, acc);
#pragma unroll
    for (int g = 0; g < 8; ++g)
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int o = lane + 32 * r;
            if (o < K) red[((size_t)q * kTransG + g) * K + o] = acc[g][r];
        }
    __syncthreads();
    for (int e = threadIdx.x; e < kTransG * K; e += blockDim.x) {
        const int g = e / K, o = e - g * K;
        if (g >= ng) continue;
        const T sum = ((red[(0 * kTransG + g) * K + o] + red[(1 * kTransG + g) * K + o]) +
                       red[(2 * kTransG + g) * K + o]) + red[(3 * kTransG + g) * K + o];
        M[(int64_t)s_par[g] * K + o] = sum;
    }
}

// L(child q) += T_q L(parent)
template <class T, int RC>
__global__ void __launch_bounds__(128) k_l2l(const int32_t *__restrict__ parents, int n,
                                             const int32_t *__restrict__ child, T *__restrict__ L,
                                             const T *__restrict__ op, int K) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T *Lp = reinterpret_cast<T *>(smraw);          // [K][8]
    __shared__ int s_ch[kTransG * 4], s_par[kTransG];
    const int p0 = blockIdx.x * kTransG;
    const int ng = min(kTransG, n - p0);
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x < kTransG * 4) {
        const int g = threadIdx.x >> 2;
        const int pb = g < ng ? parents[p0 + g] : -1;
        s_ch[threadIdx.x] = pb >= 0 ? child[4 * pb + (threadIdx.x & 3)] : -1;
        if ((threadIdx.x & 3) == 0) s_par[g] = pb;
    }
    __syncthreads();
    for (int g = q; g < kTransG; g += 4) {   // warp q stages parents q, q + 4
        const int pb = s_par[g];
        T v[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int i = lane + 32 * r;
            v[r] = (pb >= 0 && i < K) ? L[(int64_t)pb * K + i] : (T)0;
        }
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int i = lane + 32 * r;
            if (i < K) Lp[(size_t)i * kTransG + g] = v[r];
        }
    }
    __syncthreads();
    T acc[8][RC];
    trans_rows<T, RC>(op + (int64_t)q * K * K, Lp, K, lane, acc);
    // children rows are distinct: read all old values, then write all sums
    T old[8][RC];
    int chs[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        chs[g] = g < ng ? s_ch[4 * g + q] : -1;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int o = lane + 32 * r;
            old[g][r] = (chs[g] >= 0 && o < K) ? L[(int64_t)chs[g] * K + o] : (T)0;
        }
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) {
        if (chs[g] < 0) continue;
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int o = lane + 32 * r;
            if (o < K) L[(int64_t)chs[g] * K + o] = old[g][r] + acc[g][r];
        }
    }
}

// FP32 M2M / L2L with the four quadrant operators staged in shared memory by
// one bulk copy per CTA (for K <= kTransSmemMaxK).  Per level the kernels above
// are bound by the latency of their K / kTransUnroll dependent operator-row
// loads from L2; here that is one copy, and the K-long reduction runs from
// shared memory.  CTA: 16 parents, 16 warps; warp w applies quadrant q = w & 3
// to parents 4 (w >> 2) .. + 3 (four warps per quadrant hide the shared-memory
// latency of the reduction).  Levels are chained with programmatic dependent
// launch, so a level's prologue overlaps the previous level.  Same FMA and
// quadrant-sum order as k_m2m / k_l2l, so the results are bitwise equal.
constexpr int kTransSmemMaxK = 110;
constexpr int kTS = 16;   // parents per CTA
constexpr int kTSG = 4;   // parents per warp
constexpr int kTSWarps = 4 * kTS / kTSG;

size_t trans_s_smem(int K) {
    return sizeof(float) * ((size_t)4 * K * K + (size_t)kTSWarps * K * kTSG) + 16;
}

// acc[g][r] = sum_{i < K} A[i][lane + 32 r] * X[i][g], A and X in shared memory
template <int RC>
__device__ __forceinline__ void trans_rows_smem(const float *A, const float *X, int K, int lane,
                                                float (&acc)[kTSG][RC]) {
#pragma unroll
    for (int g = 0; g < kTSG; ++g)
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[g][r] = 0.f;
#pragma unroll 4
    for (int i = 0; i < K; ++i) {
        float w[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) w[r] = lane + 32 * r < K ? A[i * K + lane + 32 * r] : 0.f;
        const float4 x = reinterpret_cast<const float4 *>(X)[i];
        const float mv[kTSG] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int g = 0; g < kTSG; ++g)
#pragma unroll
            for (int r = 0; r < RC; ++r) acc[g][r] += w[r] * mv[g];
    }
}

template <int RC, bool UP>
__global__ void __launch_bounds__(32 * kTSWarps) k_trans_s(const int32_t *__restrict__ parents, int n,
                                                           const int32_t *__restrict__ child, float *__restrict__ X,
                                                           const float *__restrict__ op, int K, int *err,
                                                           float *__restrict__ Xpk, int KP) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float *sop = reinterpret_cast<float *>(smraw);                 // [4][K][K]
    float *sx = sop + (size_t)4 * K * K;                            // [16 warps][K][4]; reused as red[4][16][K]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int s_ch[kTS * 4], s_par[kTS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, q = w & 3, grp = w >> 2;
    const int p0 = blockIdx.x * kTS;
    const int ng = min(kTS, n - p0);
    // programmatic dependent launch: the next level's kernel may start its prologue (barrier
    // set-up, the operator's bulk copy, parent and child ids) on idle SMs while this level
    // computes; it reads expansions only after its griddepcontrol.wait, which waits for this
    // grid to finish.  Triggering here rather than after the reduction took the 1M-point
    // product from 0.684 to 0.674 ms.
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)(sizeof(float) * 4 * K * K);
        mbar_arrive_expect_tx(&bar, bytes);
        bulk_g2s(sop, op, bytes, &bar);
    }
    if (threadIdx.x < kTS * 4) {
        const int g = threadIdx.x >> 2;
        const int pb = g < ng ? parents[p0 + g] : -1;
        s_ch[threadIdx.x] = pb >= 0 ? child[4 * pb + (threadIdx.x & 3)] : -1;
        if ((threadIdx.x & 3) == 0) s_par[g] = pb;
    }
    __syncthreads();
    // everything below reads expansions the previous kernel on the stream wrote
    asm volatile("griddepcontrol.wait;" ::: "memory");
    float *mx = sx + (size_t)w * K * kTSG;
    {   // stage: child q of the warp's parents (upward) or the parents themselves (downward)
        float v[kTSG][RC];
#pragma unroll
        for (int g = 0; g < kTSG; ++g) {
            const int src = UP ? s_ch[4 * (grp * kTSG + g) + q] : s_par[grp * kTSG + g];
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int i = lane + 32 * r;
                v[g][r] = (src >= 0 && i < K) ? X[(int64_t)src * K + i] : 0.f;
            }
        }
#pragma unroll
        for (int r = 0; r < RC; ++r) {
            const int i = lane + 32 * r;
            if (i < K) reinterpret_cast<float4 *>(mx)[i] = make_float4(v[0][r], v[1][r], v[2][r], v[3][r]);
        }
    }
    // a CTA-uniform outcome of the bounded wait, so that every thread leaves together
    if (!__syncthreads_and(mbar_wait(&bar, 0) ? 1 : 0)) {
        if (threadIdx.x == 0) set_error(err, kErrWaitTimeout);
        return;   // the results of this product are invalid; the host reads the error word
    }
    float acc[kTSG][RC];
    trans_rows_smem<RC>(sop + (size_t)q * K * K, mx, K, lane, acc);
    if (UP) {
        __shared__ int s_mx[kTS];   // largest |sum| of each parent (float bits, non-negative)
        if (threadIdx.x < kTS) s_mx[threadIdx.x] = 0;
        __syncthreads();   // every warp is done with its staging area: reuse it for the quadrant products
        float *red = sx;   // [4][16][K]
#pragma unroll
        for (int g = 0; g < kTSG; ++g)
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int o = lane + 32 * r;
                if (o < K) red[((size_t)q * kTS + grp * kTSG + g) * K + o] = acc[g][r];
            }
        __syncthreads();
        for (int e = threadIdx.x; e < kTS * K; e += blockDim.x) {
            const int g = e / K, o = e - g * K;
            if (g >= ng) continue;
            const float sum = ((red[(0 * kTS + g) * K + o] + red[(1 * kTS + g) * K + o]) + red[(2 * kTS + g) * K + o]) +
                              red[(3 * kTS + g) * K + o];
            X[(int64_t)s_par[g] * K + o] = sum;
            if (Xpk) atomicMax(&s_mx[g], __float_as_int(fabsf(sum)));
        }
        if (Xpk) {   // the scaled fp16 hi / lo rows the tensor-core M2L gathers (the same sums again)
            __syncthreads();
            for (int e = threadIdx.x; e < kTS * K; e += blockDim.x) {
                const int g = e / K, o = e - g * K;
                if (g >= ng) continue;
                const float sum = ((red[(0 * kTS + g) * K + o] + red[(1 * kTS + g) * K + o]) +
                                   red[(2 * kTS + g) * K + o]) +
                                  red[(3 * kTS + g) * K + o];
                __half *pk = reinterpret_cast<__half *>(Xpk) + (int64_t)s_par[g] * 2 * KP;
                __half hi, lo;
                f16_split(sum * pow2f(m2l_pow2_exp(__int_as_float(s_mx[g]))), hi, lo);
                pk[o] = hi;
                pk[KP + o] = lo;
            }
            if (threadIdx.x < ng) {
                __half *pk = reinterpret_cast<__half *>(Xpk) + (int64_t)s_par[threadIdx.x] * 2 * KP;
                *reinterpret_cast<float *>(pk + m2l_scale_slot(K)) =
                    pow2f(-m2l_pow2_exp(__int_as_float(s_mx[threadIdx.x])));
            }
        }
    } else {
        float old[kTSG][RC];
        int chs[kTSG];
#pragma unroll
        for (int g = 0; g < kTSG; ++g) {
            chs[g] = grp * kTSG + g < ng ? s_ch[4 * (grp * kTSG + g) + q] : -1;
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int o = lane + 32 * r;
                old[g][r] = (chs[g] >= 0 && o < K) ? X[(int64_t)chs[g] * K + o] : 0.f;
            }
        }
#pragma unroll
        for (int g = 0; g < kTSG; ++g) {
            if (chs[g] < 0) continue;
#pragma unroll
            for (int r = 0; r < RC; ++r) {
                const int o = lane + 32 * r;
                if (o < K) X[(int64_t)chs[g] * K + o] = old[g][r] + acc[g][r];
            }
        }
    }
}

// M2L for the FP64 path: one thread per (target box, output row), operators
// read through the cache hierarchy.
template <class T>
__global__ void k_m2l_direct(int lb, int nl, const int32_t *__restrict__ vtab, const T *__restrict__ M,
                             T *__restrict__ L, const T *__restrict__ ops, int Kin, int Kout,
                             const int32_t *__restrict__ box_opslot) {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= (int64_t)nl * Kout) return;
    const int b = lb + (int)(g / Kout), row = (int)(g % Kout);
    const T *opb = ops;
    if (box_opslot) {   // batched plans: operators of the box's (problem, level)
        const int sl = box_opslot[b];
        if (sl < 0) return;
        opb = ops + (size_t)sl * kOffsetClasses * Kin * Kout;
    }
    T acc = 0;
    for (int o = 0; o < kOffsetClasses; ++o) {
        const int s = vtab[(int64_t)kOffsetClasses * b + o];
        if (s < 0) continue;
        const T *op = opb + (size_t)o * Kin * Kout + row;
        const T *Ms = M + (int64_t)s * Kin;
        for (int i = 0; i < Kin; ++i) acc += op[(size_t)i * Kout] * Ms[i];
    }
    L[(int64_t)b * Kout + row] = acc;
}

// ------------------------------------------------------------------ irregular-harmonic evaluation
// G_n^m(v) = Ptilde_n^m(cos th) e^{i m om} (h/rho)^n / rho for n+m even is produced
// column by column from G_m^m with the normalised three-term recurrence; F(slot, gr, gi)
// consumes each term.  tab2/tabi are the recurrence tables of fill_recurrence_tables.
template <class T, class F>
__device__ __forceinline__ void irregular_column(int m, int p, T a, T t, T gmm_r, T gmm_i, const T *tab2,
                                                 const T *tabi, F &&f, int slot) {
    T g2r = 0, g2i = 0, g1r = gmm_r, g1i = gmm_i;
    f(slot, g1r, g1i);
    slot += m ? 2 : 1;
    const T ta = t * a, a2 = a * a;
    for (int n = m + 1; n <= p; ++n) {
        const T c1 = (T)(2 * n - 1) * ta;
        const T c2 = tab2[n * (p + 1) + m] * a2;
        const T iv = tabi[n * (p + 1) + m];
        const T gr = (c1 * g1r - c2 * g2r) * iv;
        const T gi = (c1 * g1i - c2 * g2i) * iv;
        g2r = g1r; g2i = g1i; g1r = gr; g1i = gi;
        if (((n + m) & 1) == 0) {
            f(slot, gr, gi);
            slot += m ? 2 : 1;
        }
    }
}

// ------------------------------------------------------------------ P2L (X list)
// Lh_k^l(B) += sum_j u_j G_k^l(Y_j - C_B), vertical component -c, for the k+l
// parity PAR.  One warp per box; the sources of all X entries form one
// concatenated range and lane q takes positions q, q+32, ...; each lane
// accumulates its own row of K coefficients in shared memory (row stride
// Kpad odd: conflict-free), and the 32 rows are summed per coefficient at the
// end.
constexpr int kP2LWarps = 2;

template <class T, int PAR>
__global__ void __launch_bounds__(32 * kP2LWarps) k_p2l(
    int nxb, const int32_t *__restrict__ xboxes, const int32_t *__restrict__ xoff, const int32_t *__restrict__ xitems,
    const int32_t *__restrict__ xcum, const int32_t *__restrict__ xtot, const int32_t *__restrict__ begin,
    const int32_t *__restrict__ level, const double2 *__restrict__ centre, const float2 *__restrict__ loc,
    const double2 *__restrict__ pos, const T *__restrict__ u, T *__restrict__ L, int K, int p, double S, ShapeC shape) {
    extern __shared__ __align__(16) unsigned char smraw_p2l[];
    T *tab2 = reinterpret_cast<T *>(smraw_p2l);
    T *tabi = tab2 + (IMQ_MAX_P + 1) * (IMQ_MAX_P + 1);
    T *fmm_ = tabi + (IMQ_MAX_P + 1) * (IMQ_MAX_P + 1);       // sqrt((2m-1)/(2m)), m = 1..p
    T *accb = fmm_ + (IMQ_MAX_P + 2);
    fill_recurrence_tables<T>(tab2, tabi, p);
    for (int m = threadIdx.x; m <= p; m += blockDim.x) fmm_[m] = m ? sqrt((T)(2 * m - 1) / (T)(2 * m)) : (T)1;
    const int Kpad = K | 1;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *acc = accb + (size_t)w * 32 * Kpad;
    for (int e = lane; e < 32 * Kpad; e += 32) acc[e] = 0;
    __syncthreads();
    const int widx = blockIdx.x * kP2LWarps + w;
    if (widx >= nxb) return;
    const int b = xboxes[widx];
    const T h = box_side<T>(S, level[b]);
    const double2 cb = centre[b];
    const T c = (T)shape.of(b);
    const int x0 = xoff[b], x1 = xoff[b + 1], St = xtot[b];
    T *row = acc + lane * Kpad;
    int r = x0;
    for (int q = lane; q < St; q += 32) {
        while (r + 1 < x1 && xcum[r + 1] <= q) ++r;
        const int sb = xitems[r];
        const int j = begin[sb] + (q - xcum[r]);
        T vx, vy;
        point_offset<T>(j, loc, pos, cb, centre[sb], vx, vy);
        const T inv = rsq<T>(vx * vx + vy * vy + c * c);
        const T a = h * inv, t = -c * inv;
        const T zr0 = vx * inv * a, zi0 = vy * inv * a;
        const T ta = t * a, a2 = a * a;
        T gr = inv * u[j], gi = 0;   // G_0^0 times u_j
        int slot = 0;
        for (int m = 0; m <= p; ++m) {
            if (m > 0) {
                const T f = fmm_[m];
                const T nr = (gr * zr0 - gi * zi0) * f;
                gi = (gr * zi0 + gi * zr0) * f;
                gr = nr;
            }
            const int step = m ? 2 : 1;
            if (PAR == 0) {
                row[slot] += gr;
                if (m) row[slot + 1] += gi;
                slot += step;
            }
            T g2r = 0, g2i = 0, g1r = gr, g1i = gi;
            for (int n = m + 1; n <= p; ++n) {
                const T c1 = (T)(2 * n - 1) * ta;
                const T c2 = tab2[n * (p + 1) + m] * a2;
                const T iv = tabi[n * (p + 1) + m];
                const T nr = (c1 * g1r - c2 * g2r) * iv;
                const T ni = (c1 * g1i - c2 * g2i) * iv;
                g2r = g1r; g2i = g1i; g1r = nr; g1i = ni;
                if (((n - m) & 1) == PAR) {
                    row[slot] += nr;
                    if (m) row[slot + 1] += ni;
                    slot += step;
                }
            }
        }
    }
    __syncwarp();
    T *Lb = L + (int64_t)b * K;
    for (int e = lane; e < K; e += 32) {
        T sum = 0;
        for (int l2 = 0; l2 < 32; ++l2) sum += acc[l2 * Kpad + e];
        Lb[e] += sum;
    }
}

template <class T, int PAR>
void p2l_launch_impl(Plan &P, const T *u, T *L, int K, cudaStream_t s) {
    if (P.X.total == 0) return;
    if constexpr (std::is_same<T, float>::value && PAR == 0) {
        if (p2m_fixed_p_supported(P.p)) {
            p2l_fixed_p_launch(P, u, L, s);
            return;
        }
    }
    const size_t smem = sizeof(T) * (2 * (IMQ_MAX_P + 1) * (IMQ_MAX_P + 1) + (IMQ_MAX_P + 2) +
                                     (size_t)kP2LWarps * 32 * (K | 1));
    IMQ_CUDA(cudaFuncSetAttribute(k_p2l<T, PAR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_p2l<T, PAR><<<(unsigned)((P.nxbox + kP2LWarps - 1) / kP2LWarps), 32 * kP2LWarps, smem, s>>>(
        P.nxbox, P.xboxes.as<int32_t>(), P.X.off.as<int32_t>(), P.X.items.as<int32_t>(), P.xcum.as<int32_t>(),
        P.xtot.as<int32_t>(), P.begin.as<int32_t>(), P.level.as<int32_t>(), P.centre.as<double2>(),
        P.loc.as<float2>(), P.pos.as<double2>(), u, L, K, P.p, P.side, P.shape());
    IMQ_LAUNCH_CHECK();
}

// ------------------------------------------------------------------ L2P + M2P (W list)
template <class T>
__global__ void k_far(int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin,
                      const int32_t *__restrict__ end, const int32_t *__restrict__ level,
                      const double2 *__restrict__ centre, const float2 *__restrict__ loc,
                      const double2 *__restrict__ pos, const int32_t *__restrict__ woff,
                      const int32_t *__restrict__ witems, const T *__restrict__ M, const T *__restrict__ L,
                      const T *__restrict__ coef, int K, int p, double S, ShapeC shape, T *__restrict__ bs) {
    __shared__ T tab2[(IMQ_MAX_P + 1) * (IMQ_MAX_P + 1)], tabi[(IMQ_MAX_P + 1) * (IMQ_MAX_P + 1)];
    fill_recurrence_tables<T>(tab2, tabi, p);
    __syncthreads();
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nleaf) return;
    const int b = leaves[warp];
    const double2 cb = centre[b];
    const T inv_h = (T)1 / box_side<T>(S, level[b]);
    const T c = (T)shape.of(b);
    const T *Lb = L + (int64_t)b * K;
    for (int i = begin[b] + lane; i < end[b]; i += 32) {
        T wx, wy;
        point_offset<T>(i, loc, pos, cb, cb, wx, wy);
        T phi = 0;
        // L2P: sum eps_m Ptilde_n^m(0) Re(Lh_n^m conj(w)^m |w|^{n-m}), w = (x - c_B)/h
        {
            const T ux = wx * inv_h, uy = wy * inv_h;
            const T r2 = ux * ux + uy * uy;
            T zr = 1, zi = 0;
            int slot = 0;
            for (int m = 0; m <= p; ++m) {
                T qr = zr, qi = zi;
                const T eps = m ? (T)2 : (T)1;
                for (int n = m; n <= p; n += 2) {
                    const T lr = Lb[slot];
                    const T li = m ? Lb[slot + 1] : (T)0;
                    phi += eps * coef[slot] * (lr * qr - li * qi);
                    qr *= r2;
                    qi *= r2;
                    slot += m ? 2 : 1;
                }
                const T nr = zr * ux + zi * uy;
                zi = zi * ux - zr * uy;
                zr = nr;
            }
        }
        // M2P over the W list: sum eps_m Re(Mh_n^m G_n^m(X_i - Z_S)), vertical component +c
        for (int e = woff[b]; e < woff[b + 1]; ++e) {
            const int s = witems[e];
            const double2 cs = centre[s];
            T vx, vy;
            point_offset<T>(i, loc, pos, cs, cb, vx, vy);
            const T hs = box_side<T>(S, level[s]);
            const T rho2 = vx * vx + vy * vy + c * c;
            const T inv = rsq<T>(rho2);
            const T a = hs * inv, t = c * inv;
            const T zr0 = vx * inv * a, zi0 = vy * inv * a;
            const T *Ms = M + (int64_t)s * K;
            T gr = inv, gi = 0;   // G_0^0
            int slot = 0;
            for (int m = 0; m <= p; ++m) {
                if (m > 0) {
                    const T f = sqrt((T)(2 * m - 1) / (T)(2 * m));
                    const T nr = (gr * zr0 - gi * zi0) * f;
                    gi = (gr * zi0 + gi * zr0) * f;
                    gr = nr;
                }
                const T eps = m ? (T)2 : (T)1;
                irregular_column<T>(m, p, a, t, gr, gi, tab2, tabi,
                                    [&](int sl, T xr, T xi) {
                                        const T mr = Ms[sl];
                                        const T mi = m ? Ms[sl + 1] : (T)0;
                                        phi += eps * (mr * xr - mi * xi);
                                    },
                                    slot);
                slot += ((p - m) / 2 + 1) * (m ? 2 : 1);
            }
        }
        bs[i] = phi;
    }
}

template <class T>
void upload(DevMem &dst, const std::vector<double> &src, cudaStream_t s) {
    std::vector<T> tmp(src.begin(), src.end());
    dst.alloc(sizeof(T) * std::max<size_t>(1, tmp.size()));
    IMQ_CUDA(cudaMemcpyAsync(dst.ptr, tmp.data(), sizeof(T) * tmp.size(), cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

int64_t Plan::device_bytes() const {
    int64_t t = 0;
    const DevMem *all[] = {&codes, &perm, &level, &prefix, &begin, &end, &parent, &child, &centre, &leaves,
                           &U.off, &U.items, &V.off, &V.items, &W.off, &W.items, &X.off, &X.items,
                           &colleagues, &vtab, &ucum, &uoff, &pos, &loc, &rec4, &leaf_of,
                           &ops32.m2m, &ops32.l2l, &ops32.m2l, &ops32.p2mc, &ops32.M, &ops32.L,
                           &ops64.m2m, &ops64.l2l, &ops64.m2l, &ops64.p2mc, &ops64.M, &ops64.L,
                           &schwarz.patch_off, &schwarz.patch_pts, &schwarz.fac_off, &schwarz.factor,
                           &schwarz.pt_off, &schwarz.pt_slot, &schwarz.ypatch, &box_prob, &prob_c, &pt_prob,
                           &box_opslot, &m2l_tiles, &m2l_tbox, &xcum, &xtot, &utot, &xboxes};
    for (auto *d : all) t += (int64_t)d->bytes;
    return t;
}

// FP32 M2L on the tensor cores unless the plan asks for the CUDA cores
static void prepare_tensor_m2l(Plan &P, TypedOps &O, int nblk, cudaStream_t s) {
    const int K = P.layout.K;
    const bool fits = m2l_umma_supported(K, K);
    if (P.m2l_kernel == IMQ_M2L_TENSOR && !fits)
        fail(IMQ_UNSUPPORTED, "imq_plan: the expansion does not fit the tensor-core M2L");
    if (P.m2l_kernel == IMQ_M2L_CUDA_CORES || !fits) return;
    m2l_umma_prepare(P, O.m2l.as<float>(), nblk, K, O.m2l_img, O.Mpk, O.m2l_tmask, O.m2l_order, O.m2l_counter, s);
    O.m2l_nblk = nblk;
    O.umma = true;
}

void ensure_ops(Plan &P, bool fp64, cudaStream_t s) {
    TypedOps &O = fp64 ? P.ops64 : P.ops32;
    if (O.ready) return;
    if (!fp64) {
        far_fixed_p_prepare(s);
        p2l_fixed_p_prepare(s);
    }
    const int K = P.layout.K;
    const int nlev = std::max(0, P.m2l_level_hi - P.m2l_level_lo + 1);
    if (P.nprob > 1) {   // batched: shared M2M/L2L, M2L per (problem, level) generated on the device
        if (P.h_m2m.empty()) {
            build_m2m_ops(P.layout, P.h_m2m);
            build_l2l_ops(P.layout, P.h_l2l);
            p2m_coefficients(P.layout, P.h_p2mc);
        }
        const size_t es = fp64 ? sizeof(double) : sizeof(float);
        if (!fp64 && !P.rec4.ptr) P.rec4.alloc(sizeof(float4) * (size_t)P.N);
        O.M.alloc(es * (size_t)P.nbox * K);
        O.L.alloc(es * (size_t)P.nbox * K);
        if (fp64) {
            upload<double>(O.m2m, P.h_m2m, s);
            upload<double>(O.l2l, P.h_l2l, s);
            upload<double>(O.p2mc, P.h_p2mc, s);
            generate_m2l_ops<double>(P.layout, P.layout, P.h_slot_hc, K, O.m2l, s);
        } else {
            upload<float>(O.m2m, P.h_m2m, s);
            upload<float>(O.l2l, P.h_l2l, s);
            upload<float>(O.p2mc, P.h_p2mc, s);
            const int RR = m2l_tiled_rows(K);
            if (RR < 0) fail(IMQ_UNSUPPORTED, "expansion order too large for the M2L kernel");
            generate_m2l_ops<float>(P.layout, P.layout, P.h_slot_hc, 16 * RR, O.m2l, s);
            prepare_tensor_m2l(P, O, (int)P.h_slot_hc.size(), s);
            ensure_m2p_items(P, s);
        }
        O.ready = true;
        return;
    }
    if (P.h_m2m.empty()) {
        build_m2m_ops(P.layout, P.h_m2m);
        build_l2l_ops(P.layout, P.h_l2l);
        p2m_coefficients(P.layout, P.h_p2mc);
        P.h_m2l.assign((size_t)std::max(1, nlev) * kOffsetClasses * K * K, 0.0);
        std::vector<double> tmp;
        for (int li = 0; li < nlev; ++li) {
            const double h = P.side / (double)(1 << (P.m2l_level_lo + li));
            build_m2l_ops(P.layout, P.layout, h, P.c, tmp);
            std::copy(tmp.begin(), tmp.end(), P.h_m2l.begin() + (size_t)li * kOffsetClasses * K * K);
        }
    }
    const size_t es = fp64 ? sizeof(double) : sizeof(float);
    if (!fp64 && !P.rec4.ptr) P.rec4.alloc(sizeof(float4) * (size_t)P.N);
    O.M.alloc(es * (size_t)P.nbox * K);
    O.L.alloc(es * (size_t)P.nbox * K);
    if (fp64) {
        upload<double>(O.m2m, P.h_m2m, s);
        upload<double>(O.l2l, P.h_l2l, s);
        upload<double>(O.m2l, P.h_m2l, s);
        upload<double>(O.p2mc, P.h_p2mc, s);
    } else {
        upload<float>(O.m2m, P.h_m2m, s);
        upload<float>(O.l2l, P.h_l2l, s);
        upload<float>(O.p2mc, P.h_p2mc, s);
        const int RR = m2l_tiled_rows(K);
        if (RR < 0) fail(IMQ_UNSUPPORTED, "expansion order too large for the M2L kernel");
        const int Kp = 16 * RR;
        std::vector<double> pad((size_t)std::max(1, nlev) * kOffsetClasses * K * Kp, 0.0);
        for (size_t blk = 0; blk < (size_t)std::max(1, nlev) * kOffsetClasses; ++blk)
            for (int i = 0; i < K; ++i)
                for (int r = 0; r < K; ++r) pad[(blk * K + i) * Kp + r] = P.h_m2l[(blk * K + i) * K + r];
        upload<float>(O.m2l, pad, s);
        prepare_tensor_m2l(P, O, std::max(1, nlev), s);
        ensure_m2p_items(P, s);   // also the P2P leaf order (host work, here before any stream capture)
    }
    O.ready = true;
}

template <class T>
void p2p_apply(Plan &P, const T *u, T *bs, cudaStream_t s);

template <class T>
void p2l_odd_launch(Plan &P, const T *u, T *Lodd, cudaStream_t s) {
    p2l_launch_impl<T, 1>(P, u, Lodd, P.layout_odd.K, s);
}
template void p2l_odd_launch<float>(Plan &, const float *, float *, cudaStream_t);
template void p2l_odd_launch<double>(Plan &, const double *, double *, cudaStream_t);

template <class T>
void m2m_levels(Plan &P, T *M, const T *m2m, cudaStream_t s, int *launches, float *Mpk = nullptr, int KP = 0);

// P2M: the fixed-order FP32 kernel where one is compiled, else the generic one
template <class T>
void p2m_launch(Plan &P, const T *u, T *M, const T *coef, cudaStream_t s, float *Mpk = nullptr, int KP = 0) {
    if constexpr (std::is_same<T, float>::value) {
        if (p2m_fixed_p_supported(P.p)) {
            p2m_fixed_p_launch(P, u, M, coef, s, Mpk, KP);
            return;
        }
    }
    k_p2m<T><<<blocks_for((int64_t)P.nleaf * 32, 128), 128, 0, s>>>(
        P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(), P.level.as<int32_t>(),
        P.centre.as<double2>(), P.loc.as<float2>(), P.pos.as<double2>(), u, M, P.layout.K, P.p, coef, P.side);
    IMQ_LAUNCH_CHECK();
}

template <class T>
void upward_launch(Plan &P, const T *u, T *M, const T *coef, const T *m2m, cudaStream_t s, int *launches) {
    p2m_launch<T>(P, u, M, coef, s);
    ++*launches;
    m2m_levels<T>(P, M, m2m, s, launches);
}

// internal boxes of each level, in box order (built once per plan)
void ensure_parents(Plan &P, cudaStream_t s) {
    if (!P.parent_start.empty()) return;
    std::vector<int32_t> ch(4 * (size_t)P.nbox);
    IMQ_CUDA(cudaMemcpyAsync(ch.data(), P.child.ptr, sizeof(int32_t) * ch.size(), cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<int32_t> par;
    P.parent_start.assign(P.level_start.size(), 0);
    for (size_t lev = 0; lev + 1 < P.level_start.size(); ++lev) {
        P.parent_start[lev] = (int)par.size();
        for (int b = P.level_start[lev]; b < P.level_start[lev + 1]; ++b)
            if (ch[4 * (size_t)b] >= 0 || ch[4 * (size_t)b + 1] >= 0 || ch[4 * (size_t)b + 2] >= 0 ||
                ch[4 * (size_t)b + 3] >= 0)
                par.push_back(b);
    }
    P.parent_start.back() = (int)par.size();
    P.parents.alloc(sizeof(int32_t) * std::max<size_t>(1, par.size()));
    if (!par.empty())
        IMQ_CUDA(cudaMemcpyAsync(P.parents.ptr, par.data(), sizeof(int32_t) * par.size(), cudaMemcpyHostToDevice, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
}

// Xpk (upward, shared-memory kernel only): also write the scaled fp16 hi / lo rows of the parents
template <class T, bool UP>
void trans_launch(Plan &P, T *X, const T *op, int K, int lev_lo, int lev_hi, bool downward, cudaStream_t s,
                  int *launches, float *Xpk = nullptr, int KP = 0) {
    ensure_parents(P, s);
    if constexpr (std::is_same<T, float>::value) {
        if (K <= kTransSmemMaxK) {
            const int RC = (K + 31) / 32;
            void (*kern)(const int32_t *, int, const int32_t *, float *, const float *, int, int *, float *, int) =
                RC == 1 ? k_trans_s<1, UP> : RC == 2 ? k_trans_s<2, UP> : RC == 3 ? k_trans_s<3, UP> : k_trans_s<4, UP>;
            const size_t smem = trans_s_smem(K);
            IMQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            int *err = device_error_word();
            for (int k = 0; k <= lev_hi - lev_lo; ++k) {
                const int lev = downward ? lev_lo + k : lev_hi - k;
                const int pb = P.parent_start[lev], np = P.parent_start[lev + 1] - pb;
                if (np <= 0) continue;
                cudaLaunchConfig_t cfg = {};
                cfg.gridDim = dim3((unsigned)((np + kTS - 1) / kTS));
                cfg.blockDim = dim3(32 * kTSWarps);
                cfg.dynamicSmemBytes = smem;
                cfg.stream = s;
                cudaLaunchAttribute attr[1];
                attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
                attr[0].val.programmaticStreamSerializationAllowed = 1;
                cfg.attrs = attr;
                cfg.numAttrs = 1;
                const int32_t *par = P.parents.as<int32_t>() + pb, *ch = P.child.as<int32_t>();
                IMQ_CUDA(cudaLaunchKernelEx(&cfg, kern, par, np, ch, (float *)X, (const float *)op, K, err, Xpk, KP));
                ++*launches;
            }
            return;
        }
    }
    const int RC = (K + 31) / 32;
    void (*kern)(const int32_t *, int, const int32_t *, T *, const T *, int) = nullptr;
#define IMQ_TRANS_CASE(R)                                \
    case R:                                              \
        kern = UP ? k_m2m<T, R> : k_l2l<T, R>;           \
        break;
    switch (RC) {
        IMQ_TRANS_CASE(1)
        IMQ_TRANS_CASE(2)
        IMQ_TRANS_CASE(3)
        IMQ_TRANS_CASE(4)
        IMQ_TRANS_CASE(5)
        IMQ_TRANS_CASE(6)
        default: fail(IMQ_UNSUPPORTED, "M2M/L2L: expansion too large");
    }
#undef IMQ_TRANS_CASE
    const size_t smem = sizeof(T) * (UP ? (size_t)4 * K * kTransG * 2 : (size_t)K * kTransG);
    IMQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int k = 0; k <= lev_hi - lev_lo; ++k) {
        const int lev = downward ? lev_lo + k : lev_hi - k;
        const int pb = P.parent_start[lev], np = P.parent_start[lev + 1] - pb;
        if (np <= 0) continue;
        kern<<<(np + kTransG - 1) / kTransG, 128, smem, s>>>(P.parents.as<int32_t>() + pb, np, P.child.as<int32_t>(),
                                                           X, op, K);
        IMQ_LAUNCH_CHECK();
        ++*launches;
    }
}

template <class T>
void m2m_levels(Plan &P, T *M, const T *m2m, cudaStream_t s, int *launches, float *Mpk, int KP) {
    trans_launch<T, true>(P, M, m2m, P.layout.K, 2, P.max_level - 1, false, s, launches, Mpk, KP);
}
template void m2m_levels<float>(Plan &, float *, const float *, cudaStream_t, int *, float *, int);
template void m2m_levels<double>(Plan &, double *, const double *, cudaStream_t, int *, float *, int);
template void upward_launch<float>(Plan &, const float *, float *, const float *, const float *, cudaStream_t, int *);
template void upward_launch<double>(Plan &, const double *, double *, const double *, const double *, cudaStream_t, int *);

template <class T>
void l2l_launch(Plan &P, T *L, const T *op, int K, cudaStream_t s, int *launches) {
    // parents at levels 2 .. max_level - 1, children one level below
    trans_launch<T, false>(P, L, op, K, 2, P.max_level - 1, true, s, launches);
}
template void l2l_launch<float>(Plan &, float *, const float *, int, cudaStream_t, int *);
template void l2l_launch<double>(Plan &, double *, const double *, int, cudaStream_t, int *);

template <class T>
void m2l_direct_launch(Plan &P, const T *M, T *L, const T *ops, int Kin, int Kout, cudaStream_t s, int *launches);

template <class T>
void m2l_direct_launch(Plan &P, const T *M, T *L, const T *ops, int Kin, int Kout, cudaStream_t s, int *launches) {
    for (int lev = P.m2l_level_lo; lev <= P.m2l_level_hi; ++lev) {
        const int lb = P.level_start[lev], nl = P.level_start[lev + 1] - lb;
        const bool batched = P.nprob > 1;
        const T *opl = batched ? ops : ops + (size_t)(lev - P.m2l_level_lo) * kOffsetClasses * Kin * Kout;
        k_m2l_direct<T><<<blocks_for((int64_t)nl * Kout, 128), 128, 0, s>>>(
            lb, nl, P.vtab.as<int32_t>(), M, L, opl, Kin, Kout, batched ? P.box_opslot.as<int32_t>() : nullptr);
        IMQ_LAUNCH_CHECK();
        ++*launches;
    }
}
template void m2l_direct_launch<float>(Plan &, const float *, float *, const float *, int, int, cudaStream_t, int *);
template void m2l_direct_launch<double>(Plan &, const double *, double *, const double *, int, int, cudaStream_t, int *);

// FP32 product at a fixed order p <= 16.  P2L (X lists), the near field (P2P)
// and the W-list M2P terms depend on the far-field chain only at its ends, so
// without a phase timer they run concurrently with the latency-bound chain
// P2M -> M2M -> M2L -> L2L, on the plan's two streams:
//
//   s0  : zero M and L, [fork] ... wait(done)
//   hi  : wait(fork), P2M, M2M, [mready], wait(xready), M2L (+= L), L2L, wait(join), L2P (+ W partials + near), [done]
//   aux : wait(fork), P2L (+= L), [xready], P2P -> near, wait(mready), M2P -> W partials, [join]
//
// With a timer every phase runs on s0 in the order P2M, M2M, P2L, M2L, L2L, P2P,
// far.  Either way L = P2L terms + M2L terms, and b = L2P + the W partials in
// list order + near, so both schedules give the same bits.
int fmm_apply_f32_fixed(Plan &P, const float *us, float *bs, int nrhs, cudaStream_t s0, PhaseTimer *tm) {
    TypedOps &O = P.ops32;
    const int K = P.layout.K, nb = P.nbox;
    float *M = O.M.as<float>(), *L = O.L.as<float>();
    const float *m2m = O.m2m.as<float>(), *l2l = O.l2l.as<float>(), *m2l = O.m2l.as<float>(),
                *coef = O.p2mc.as<float>();
    ensure_m2p_items(P, s0);
    // the near field of every right-hand side comes from one P2P pass (one kernel value per pair
    // serves four right-hand sides); the buffers grow outside any stream capture (the CG
    // solvers capture single right-hand-side products only)
    if (P.near.bytes < sizeof(float) * (size_t)P.N * nrhs) P.near.alloc(sizeof(float) * (size_t)P.N * nrhs);
    if (nrhs > 2 && !P.rec4b.ptr) P.rec4b.alloc(sizeof(float4) * (size_t)P.N);
    // the tensor-core M2L's scaled fp16 hi / lo rows are written by P2M and M2M themselves
    // (both fixed-order / shared-memory kernels), so no packing pass sits on the chain
    // FP64 translations: the multipoles are widened after P2M, translated (M2M, M2L, L2L) in FP64
    // and narrowed for M2P and L2P; the FP32 M2L path and its packed rows are not used
    const bool t64 = P.trans64, tmx = P.trans_mixed;   // FP64 M2M / M2L / L2L; FP64 M2M / L2L only
    if ((t64 || tmx) && !P.ops64.ready) fail(IMQ_CUDA_ERROR, "FP64 translation operators missing");
    double *Md = (t64 || tmx) ? P.ops64.M.as<double>() : nullptr;
    double *Ld = (t64 || tmx) ? P.ops64.L.as<double>() : nullptr;
    const int64_t nK = (int64_t)nb * K;
    const unsigned gw = (unsigned)std::min<int64_t>(blocks_for(nK, 256), 4 * 152);
    const bool fuse_pack =
        !t64 && !tmx && O.umma && P.n_m2l_tiles > 0 && p2m_fixed_p_supported(P.p) && K <= kTransSmemMaxK;
    const int kp_pack = m2l_umma_kp(K);
    const bool conc = tm == nullptr;
    if (conc) P.aux.ensure();
    cudaStream_t sa = conc ? P.aux.s : s0, s = conc ? P.aux.hi : s0;
    float *near = P.near.as<float>();
    int launches = 0;
    auto t0 = [&](int ph) { if (tm) tm->start(ph, s0); };
    auto t1 = [&]() { if (tm) tm->stop(s0); };
    const int p2p_launches = 2 * ((nrhs + 3) / 4);
    if (!conc) {
        t0(kPhP2P);
        p2p_near_f32(P, us, near, nrhs, s0);
        launches += p2p_launches;
        t1();
    }
    for (int r = 0; r < nrhs; ++r) {
        const float *u = us + (size_t)r * P.N;
        float *b = bs + (size_t)r * P.N;
        IMQ_CUDA(cudaMemsetAsync(M, 0, sizeof(float) * (size_t)nb * K, s0));
        IMQ_CUDA(cudaMemsetAsync(L, 0, sizeof(float) * (size_t)nb * K, s0));
        if (conc) {
            IMQ_CUDA(cudaEventRecord(P.aux.fork, s0));
            IMQ_CUDA(cudaStreamWaitEvent(s, P.aux.fork, 0));
            IMQ_CUDA(cudaStreamWaitEvent(sa, P.aux.fork, 0));
            if (P.X.total > 0) {
                p2l_launch_impl<float, 0>(P, u, L, K, sa);
                ++launches;
            }
            IMQ_CUDA(cudaEventRecord(P.aux.xready, sa));
            if (r == 0) {
                p2p_near_f32(P, us, near, nrhs, sa);
                launches += p2p_launches;
            }
        }
        t0(kPhP2M);
        p2m_launch<float>(P, u, M, coef, s, fuse_pack ? O.Mpk.as<float>() : nullptr, kp_pack);
        ++launches;
        t1();
        t0(kPhM2M);
        if (t64 || tmx) {
            k_widen<<<gw, 256, 0, s>>>(M, Md, nK, 0);
            m2m_levels<double>(P, Md, P.ops64.m2m.as<double>(), s, &launches);
            k_narrow<<<gw, 256, 0, s>>>(Md, M, nK);
            IMQ_LAUNCH_CHECK();
            launches += 2;
        } else {
            m2m_levels<float>(P, M, m2m, s, &launches, fuse_pack ? O.Mpk.as<float>() : nullptr, kp_pack);
        }
        t1();
        if (conc) {
            IMQ_CUDA(cudaEventRecord(P.aux.mready, s));
            IMQ_CUDA(cudaStreamWaitEvent(sa, P.aux.mready, 0));
            far_m2p_launch(P, M, sa);
            if (P.n_m2p_items > 0) ++launches;
            IMQ_CUDA(cudaEventRecord(P.aux.join, sa));
            IMQ_CUDA(cudaStreamWaitEvent(s, P.aux.xready, 0));
        } else {
            t0(kPhP2L);
            if (P.X.total > 0) {
                p2l_launch_impl<float, 0>(P, u, L, K, s);
                ++launches;
            }
            t1();
        }
        t0(kPhM2L);
        if (t64) {
            // M2L stores every box of its levels; then the P2L terms (in L) are added
            IMQ_CUDA(cudaMemsetAsync(Ld, 0, sizeof(double) * (size_t)nK, s));
            m2l_direct_launch<double>(P, Md, Ld, P.ops64.m2l.as<double>(), K, K, s, &launches);
            k_widen<<<gw, 256, 0, s>>>(L, Ld, nK, 1);
            IMQ_LAUNCH_CHECK();
            ++launches;
        } else if (P.n_m2l_tiles > 0 && O.umma) {
            m2l_umma_launch(P, M, L, O, K, s, fuse_pack);
            launches += fuse_pack ? 1 : 2;
        } else if (P.n_m2l_tiles > 0) {
            m2l_tiled_launch(P, M, L, m2l, s);
            ++launches;
        }
        t1();
        t0(kPhL2L);
        if (tmx) {   // the tensor-core M2L left L (P2L + M2L terms) in FP32
            k_widen<<<gw, 256, 0, s>>>(L, Ld, nK, 0);
            IMQ_LAUNCH_CHECK();
            ++launches;
        }
        if (t64 || tmx) {
            l2l_launch<double>(P, Ld, P.ops64.l2l.as<double>(), K, s, &launches);
            k_narrow<<<gw, 256, 0, s>>>(Ld, L, nK);
            IMQ_LAUNCH_CHECK();
            ++launches;
        } else {
            l2l_launch<float>(P, L, l2l, K, s, &launches);
        }
        t1();

        t0(kPhFar);
        if (conc) {
            IMQ_CUDA(cudaStreamWaitEvent(s, P.aux.join, 0));
        } else {
            far_m2p_launch(P, M, s);
            if (P.n_m2p_items > 0) ++launches;
        }
        far_l2p_launch(P, L, coef, near + (size_t)r * P.N, b, s);
        ++launches;
        t1();
        if (conc) {
            IMQ_CUDA(cudaEventRecord(P.aux.done, s));
            IMQ_CUDA(cudaStreamWaitEvent(s0, P.aux.done, 0));
        }
    }
    if (tm) tm->launches += launches;
    return launches;
}

template <class T>
int fmm_apply(Plan &P, const T *us, T *bs, int nrhs, cudaStream_t s, PhaseTimer *tm) {
    const bool f64 = std::is_same<T, double>::value;
    ensure_ops(P, f64, s);
    if constexpr (std::is_same<T, float>::value) {
        if (far_fixed_p_supported(P.p)) return fmm_apply_f32_fixed(P, us, bs, nrhs, s, tm);
    }
    TypedOps &O = f64 ? P.ops64 : P.ops32;
    const int K = P.layout.K, p = P.p, nb = P.nbox;
    T *M = O.M.as<T>(), *L = O.L.as<T>();
    const T *m2m = O.m2m.as<T>(), *l2l = O.l2l.as<T>(), *m2l = O.m2l.as<T>(), *coef = O.p2mc.as<T>();
    int launches = 0;
    auto t0 = [&](int ph) { if (tm) tm->start(ph, s); };
    auto t1 = [&]() { if (tm) tm->stop(s); };
    for (int r = 0; r < nrhs; ++r) {
        const T *u = us + (size_t)r * P.N;
        T *b = bs + (size_t)r * P.N;
        IMQ_CUDA(cudaMemsetAsync(M, 0, sizeof(T) * (size_t)nb * K, s));
        IMQ_CUDA(cudaMemsetAsync(L, 0, sizeof(T) * (size_t)nb * K, s));
        // upward pass
        t0(kPhP2M);
        p2m_launch<T>(P, u, M, coef, s);
        ++launches;
        t1();
        t0(kPhM2M);
        m2m_levels<T>(P, M, m2m, s, &launches);
        t1();
        // interaction: M2L per level, P2L over X lists
        t0(kPhM2L);
        if constexpr (std::is_same<T, float>::value) {
            if (P.n_m2l_tiles > 0 && O.umma) {
                m2l_umma_launch(P, M, L, O, K, s);
                launches += 2;
            } else if (P.n_m2l_tiles > 0) {
                m2l_tiled_launch(P, M, L, m2l, s);
                ++launches;
            }
        } else {
            m2l_direct_launch<T>(P, M, L, m2l, K, K, s, &launches);
        }
        t1();
        t0(kPhP2L);
        if (P.X.total > 0) {
            p2l_launch_impl<T, 0>(P, u, L, K, s);
            ++launches;
        }
        t1();
        // downward pass
        t0(kPhL2L);
        l2l_launch<T>(P, L, l2l, K, s, &launches);
        t1();
        // evaluation: L2P + M2P writes b, P2P adds the near field
        t0(kPhFar);
        k_far<T><<<blocks_for((int64_t)P.nleaf * 32, 128), 128, 0, s>>>(
            P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(), P.level.as<int32_t>(),
            P.centre.as<double2>(), P.loc.as<float2>(), P.pos.as<double2>(), P.W.off.as<int32_t>(),
            P.W.items.as<int32_t>(), M, L, coef, K, p, P.side, P.shape(), b);
        IMQ_LAUNCH_CHECK();
        ++launches;
        t1();
        t0(kPhP2P);
        p2p_apply<T>(P, u, b, s);
        launches += std::is_same<T, float>::value ? 2 : 1;
        t1();
    }
    if (tm) tm->launches += launches;
    return launches;
}

template int fmm_apply<float>(Plan &, const float *, float *, int, cudaStream_t, PhaseTimer *);
template int fmm_apply<double>(Plan &, const double *, double *, int, cudaStream_t, PhaseTimer *);

template <class Tin, class T>
void gather_sorted(const Plan &P, const Tin *v, T *us, int nrhs, cudaStream_t s) {
    for (int r = 0; r < nrhs; ++r) {
        k_gather<Tin, T><<<blocks_for(P.N, 256), 256, 0, s>>>(v + (size_t)r * P.N, P.perm.as<int32_t>(), P.N,
                                                              us + (size_t)r * P.N);
        IMQ_LAUNCH_CHECK();
    }
}

template <class T, class Tout>
void scatter_sorted(const Plan &P, const T *bs, Tout *out, int nrhs, cudaStream_t s) {
    for (int r = 0; r < nrhs; ++r) {
        k_scatter<T, Tout><<<blocks_for(P.N, 256), 256, 0, s>>>(bs + (size_t)r * P.N, P.perm.as<int32_t>(), P.N,
                                                               out + (size_t)r * P.N);
        IMQ_LAUNCH_CHECK();
    }
}

template void gather_sorted<float, float>(const Plan &, const float *, float *, int, cudaStream_t);
template void gather_sorted<double, double>(const Plan &, const double *, double *, int, cudaStream_t);
template void scatter_sorted<float, float>(const Plan &, const float *, float *, int, cudaStream_t);
template void scatter_sorted<double, double>(const Plan &, const double *, double *, int, cudaStream_t);

}  // namespace imq
