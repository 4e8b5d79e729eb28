// Near-field direct sum (P2P) over the U lists.
//
// Paper Algorithm 1, final loop: for each block p of the finest level and each
// x_i in the not-well-separated blocks NS_p, b_i += A_ij u_j for y_j in p.  On
// the adaptive tree NS_p is the U list of a leaf (adjacent leaves of any
// level, the leaf itself included), and the kernel is Eq. (5):
//     b_i += sum_{j in U(leaf(i))} u_j / sqrt(|x_i - x_j|^2 + c^2).
//
// Mapping (source-parallel, one warp per target leaf): the sources of all U
// entries form one virtual concatenated range; lane l takes positions
// l, l+32, ... of it, so a warp's lanes stay busy whatever the leaf sizes.
// Each lane keeps one partial sum per target of the current 32-target chunk in
// registers (targets broadcast from a per-warp shared-memory slot), and a
// butterfly transpose-reduction over the 32 lanes leaves target t's total in
// lane t.  Per pair: 2 FADD + 2 FFMA + 1 MUFU rsqrt + 1 FFMA.
//
// FP32 coordinates are offsets from the target leaf's centre: a source
// x_j = loc_j + (c_s - c_t) becomes loc_j - delta with delta = c_t - c_s
// rounded once from FP64, so the pair difference carries O(eps * box side)
// error instead of O(eps * |x|).
#include <type_traits>

#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kP2PWarps = 4;

template <class T>
__device__ __forceinline__ T rsq_p2p(T v) {
    if constexpr (std::is_same<T, float>::value) return rsqrtf(v);
    else return 1.0 / sqrt(v);
}

// After the call, lane t holds sum over lanes of acc[t] (t < 32).
template <class T>
__device__ __forceinline__ T transpose_reduce32(T (&acc)[32], int lane) {
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) {
        const bool upper = (lane & k) != 0;
#pragma unroll
        for (int i = 0; i < k; ++i) {
            const T send = upper ? acc[i] : acc[i + k];
            const T keep = upper ? acc[i + k] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, k);
        }
    }
    return acc[0];
}

template <class T>
__global__ void __launch_bounds__(32 * kP2PWarps) k_p2p(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
    const int32_t *__restrict__ uoffs, const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
    const int32_t *__restrict__ utot, const float2 *__restrict__ udelta, const float2 *__restrict__ loc,
    const double2 *__restrict__ pos, const T *__restrict__ u, T c2, T *__restrict__ bs) {
    __shared__ T tgx[kP2PWarps][32], tgy[kP2PWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int widx = blockIdx.x * kP2PWarps + w;
    if (widx >= nleaf) return;
    const int b = leaves[widx];
    const int tb = begin[b], nt = end[b] - tb;
    const int u0 = uoffs[b], u1 = uoffs[b + 1];
    const int St = utot[b];
    for (int tc = 0; tc < nt; tc += 32) {
        const int ntc = min(32, nt - tc);
        if (lane < ntc) {
            const int i = tb + tc + lane;
            if constexpr (std::is_same<T, float>::value) {
                tgx[w][lane] = loc[i].x;
                tgy[w][lane] = loc[i].y;
            } else {
                tgx[w][lane] = pos[i].x;
                tgy[w][lane] = pos[i].y;
            }
        }
        __syncwarp();
        T acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0;
        int r = u0;   // U entry holding this lane's current source position
        for (int q0 = 0; q0 < St; q0 += 32) {
            const int q = q0 + lane;
            T xs = 0, ys = 0, us = 0;
            if (q < St) {
                while (r + 1 < u1 && ucum[r + 1] <= q) ++r;
                const int j = begin[uitems[r]] + (q - ucum[r]);
                if constexpr (std::is_same<T, float>::value) {
                    const float2 l = loc[j];
                    const float2 d = udelta[r];
                    xs = l.x - d.x;
                    ys = l.y - d.y;
                } else {
                    xs = pos[j].x;
                    ys = pos[j].y;
                }
                us = u[j];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i < ntc) {
                    const T dx = tgx[w][i] - xs;
                    const T dy = tgy[w][i] - ys;
                    const T d2 = dx * dx + (dy * dy + c2);
                    acc[i] += rsq_p2p<T>(d2) * us;
                }
            }
        }
        const T tot = transpose_reduce32<T>(acc, lane);
        if (lane < ntc) bs[tb + tc + lane] += tot;
        __syncwarp();
    }
}

}  // namespace

template <class T>
void p2p_apply(Plan &P, const T *u, T *bs, cudaStream_t s) {
    const unsigned grid = (unsigned)((P.nleaf + kP2PWarps - 1) / kP2PWarps);
    k_p2p<T><<<grid, 32 * kP2PWarps, 0, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(),
                                              P.end.as<int32_t>(), P.U.off.as<int32_t>(), P.U.items.as<int32_t>(),
                                              P.ucum.as<int32_t>(), P.utot.as<int32_t>(), P.uoff.as<float2>(),
                                              P.loc.as<float2>(), P.pos.as<double2>(), u, (T)(P.c * P.c), bs);
    IMQ_LAUNCH_CHECK();
}

template void p2p_apply<float>(Plan &, const float *, float *, cudaStream_t);
template void p2p_apply<double>(Plan &, const double *, double *, cudaStream_t);

}  // namespace imq
