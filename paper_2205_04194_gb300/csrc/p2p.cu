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
// l, l+32, ... of it, so the lanes stay busy whatever the leaf sizes.  The
// targets of a leaf are processed in chunks of TC = 8, 16 or 32 (the smallest
// that holds the chunk); every lane keeps the chunk's target coordinates and
// one partial sum per target in registers, so the inner loop has no loads and
// no guards (padding targets sit far away and their sums are discarded).  A
// butterfly transpose-reduction over the 32 lanes leaves target t's total in
// lane t.  FP32 pairs of targets share one packed f32x2 instruction:
// per two pairs 2 add.f32x2 + 2 fma.f32x2 + 2 MUFU rsqrt + 1 fma.f32x2.
//
// FP32 coordinates are offsets from the target leaf's centre: a source
// x_j = loc_j + (c_s - c_t) becomes loc_j - delta with delta = c_t - c_s
// rounded once from FP64, so the pair difference carries O(eps * box side)
// error instead of O(eps * |x|).
#include <type_traits>

#include "f32x2.cuh"
#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kP2PWarps = 4;
constexpr float kFar = 1.0e18f;   // coordinate of padding targets

// Sum over the 32 lanes of each acc[i], i < TC; lane L ends with the total of
// target L % TC.
template <class T, int TC>
__device__ __forceinline__ T lane_reduce(T (&acc)[TC], int lane) {
#pragma unroll
    for (int k = TC / 2; k >= 1; k >>= 1) {
        const bool upper = (lane & k) != 0;
#pragma unroll
        for (int i = 0; i < k; ++i) {
            const T send = upper ? acc[i] : acc[i + k];
            const T keep = upper ? acc[i + k] : acc[i];
            acc[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, k);
        }
    }
    T v = acc[0];
#pragma unroll
    for (int k = TC; k < 32; k <<= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, k);
    return v;
}

// Position q of the concatenated U-list source range -> sorted point index j, entry r.
__device__ __forceinline__ int source_index(int q, int &r, int u1, const int32_t *__restrict__ ucum,
                                            const int32_t *__restrict__ uitems, const int32_t *__restrict__ begin) {
    while (r + 1 < u1 && ucum[r + 1] <= q) ++r;
    return begin[uitems[r]] + (q - ucum[r]);
}

// Per product: one 16-byte record (x, y, u, 0) per sorted point, x and y the
// offset from the point's leaf centre.
__global__ void k_pack_records(const float2 *__restrict__ loc, const float *__restrict__ u, int64_t n,
                               float4 *__restrict__ rec) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 l = loc[i];
        rec[i] = make_float4(l.x, l.y, u[i], 0.f);
    }
}

constexpr int kStageCap = 512;    // source records staged per warp at a time (8 KB)

struct WarpStage {
    float4 rec[kStageCap];
    uint64_t bar;
};

// Stage concatenated positions [q0, q0 + len) of the U-list sources of one leaf
// into shared memory with 1-D TMA bulk copies, one per overlapping U entry, the
// entries spread over the lanes (lane e sets up entry u0 + e, u0 + e + 32, ...);
// wait for them (bounded), then shift each entry's records into the target
// leaf's frame, the entry bounds and offset broadcast from the lane that loaded
// them.  St: total source count of the leaf.  Returns false if the wait timed out.
__device__ __forceinline__ bool stage_sources(WarpStage &ws, uint32_t &phase, int q0, int len, int u0, int u1, int St,
                                              const int32_t *__restrict__ begin, const int32_t *__restrict__ uitems,
                                              const int32_t *__restrict__ ucum, const float2 *__restrict__ udelta,
                                              const float4 *__restrict__ rec, int lane, int *err) {
    if (lane == 0) {
        // earlier generic-proxy writes to ws.rec must be ordered before the async-proxy copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&ws.bar, (uint32_t)len * 16u);
    }
    __syncwarp();
    int my_lo = 0, my_hi = 0;
    float2 my_d = make_float2(0.f, 0.f);
    for (int r = u0 + lane; r < u1; r += 32) {
        const int lo = ucum[r];
        const int hi = r + 1 < u1 ? ucum[r + 1] : St;
        if (r - u0 < 32) {
            my_lo = lo;
            my_hi = hi;
            my_d = udelta[r];
        }
        const int a = max(lo, q0), bnd = min(hi, q0 + len);
        if (a < bnd) bulk_g2s(&ws.rec[a - q0], rec + begin[uitems[r]] + (a - lo), (uint32_t)(bnd - a) * 16u, &ws.bar);
    }
    const bool ok = mbar_wait(&ws.bar, phase & 1u);
    phase++;
    if (!__all_sync(0xFFFFFFFFu, ok)) {
        if (lane == 0) set_error(err, kErrWaitTimeout);
        return false;
    }
    const int ne = u1 - u0;
    for (int e = 0; e < ne; ++e) {
        int lo, hi;
        float2 d;
        if (e < 32) {
            lo = __shfl_sync(0xFFFFFFFFu, my_lo, e);
            hi = __shfl_sync(0xFFFFFFFFu, my_hi, e);
            d.x = __shfl_sync(0xFFFFFFFFu, my_d.x, e);
            d.y = __shfl_sync(0xFFFFFFFFu, my_d.y, e);
        } else {
            lo = ucum[u0 + e];
            hi = e + 1 < ne ? ucum[u0 + e + 1] : St;
            d = udelta[u0 + e];
        }
        const int a = max(lo, q0), bnd = min(hi, q0 + len);
        for (int q = a + lane; q < bnd; q += 32) {
            float4 v = ws.rec[q - q0];
            v.x -= d.x;
            v.y -= d.y;
            ws.rec[q - q0] = v;
        }
    }
    __syncwarp();
    return true;
}

template <int TC>
__device__ __forceinline__ void p2p_tile_f32(const float4 *__restrict__ srec, int len, int lane, const u64 (&tx)[TC / 2],
                                             const u64 (&ty)[TC / 2], u64 (&acc)[TC / 2], u64 cc) {
    for (int q0 = 0; q0 < len; q0 += 32) {
        const int q = q0 + lane;
        const float4 sr = q < len ? srec[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        const u64 nx = pk2(-sr.x, -sr.x), ny = pk2(-sr.y, -sr.y), uu = pk2(sr.z, sr.z);
#pragma unroll
        for (int k = 0; k < TC / 2; ++k) {
            const u64 dx = add2(tx[k], nx);
            const u64 dy = add2(ty[k], ny);
            const u64 d2 = fma2(dx, dx, fma2(dy, dy, cc));
            float a, b;
            up2(d2, a, b);
            acc[k] = fma2(pk2(rsqrtf(a), rsqrtf(b)), uu, acc[k]);
        }
    }
}

template <int TC>
__device__ __forceinline__ float p2p_chunk_staged(WarpStage &ws, uint32_t &phase, bool staged_all, int ti, int ntc,
                                                  int lane, int u0, int u1, int St, const int32_t *__restrict__ begin,
                                                  const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
                                                  const float2 *__restrict__ udelta, const float2 *__restrict__ loc,
                                                  const float4 *__restrict__ rec, float c2, int *err) {
    u64 tx[TC / 2], ty[TC / 2], acc[TC / 2];
#pragma unroll
    for (int q = 0; q < TC / 2; ++q) {
        const int i0 = 2 * q, i1 = 2 * q + 1;
        const float2 a = i0 < ntc ? loc[ti + i0] : make_float2(kFar, kFar);
        const float2 b = i1 < ntc ? loc[ti + i1] : make_float2(kFar, kFar);
        tx[q] = pk2(a.x, b.x);
        ty[q] = pk2(a.y, b.y);
        acc[q] = 0ull;
    }
    const u64 cc = pk2(c2, c2);
    if (staged_all) {
        p2p_tile_f32<TC>(ws.rec, St, lane, tx, ty, acc, cc);
    } else {
        for (int q0 = 0; q0 < St; q0 += kStageCap) {
            const int len = min(kStageCap, St - q0);
            if (!stage_sources(ws, phase, q0, len, u0, u1, St, begin, uitems, ucum, udelta, rec, lane, err)) break;
            p2p_tile_f32<TC>(ws.rec, len, lane, tx, ty, acc, cc);
            __syncwarp();
        }
    }
    float s[TC];
#pragma unroll
    for (int k = 0; k < TC / 2; ++k) up2(acc[k], s[2 * k], s[2 * k + 1]);
    return lane_reduce<float, TC>(s, lane);
}

// STORE: write the near-field sum (b_near = sum); otherwise add it to bs.
// W warps per CTA (one target leaf each); targets in chunks of at most TCMAX.
template <bool STORE, int W, int TCMAX>
__global__ void __launch_bounds__(32 * W) k_p2p_f32(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
    const int32_t *__restrict__ uoffs, const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
    const int32_t *__restrict__ utot, const float2 *__restrict__ udelta, const float2 *__restrict__ loc,
    const float4 *__restrict__ rec, ShapeC shape, float *__restrict__ bs, int *err) {
    extern __shared__ __align__(128) unsigned char smraw_p2p[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStage &ws = reinterpret_cast<WarpStage *>(smraw_p2p)[w];
    if (lane == 0) {
        mbar_init(&ws.bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    const int widx = blockIdx.x * W + w;
    if (widx >= nleaf) return;
    const int b = leaves[widx];
    const int tb = begin[b], nt = end[b] - tb;
    const int u0 = uoffs[b], u1 = uoffs[b + 1];
    const int St = utot[b];
    const double cb = shape.of(b);
    const float c2 = (float)(cb * cb);
    uint32_t phase = 0;
    const bool staged_all = St <= kStageCap;
    if (staged_all && !stage_sources(ws, phase, 0, St, u0, u1, St, begin, uitems, ucum, udelta, rec, lane, err)) return;
    for (int tc = 0; tc < nt; tc += TCMAX) {
        const int ntc = min(TCMAX, nt - tc);
        float tot;
        int tcap;
        if (ntc <= 8) {
            tot = p2p_chunk_staged<8>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St, begin, uitems, ucum,
                                      udelta, loc, rec, c2, err);
            tcap = 8;
        } else if (TCMAX == 16 || ntc <= 16) {
            tot = p2p_chunk_staged<16>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St, begin, uitems, ucum,
                                       udelta, loc, rec, c2, err);
            tcap = 16;
        } else {
            tot = p2p_chunk_staged<(TCMAX > 16 ? 32 : 16)>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St,
                                                           begin, uitems, ucum, udelta, loc, rec, c2, err);
            tcap = TCMAX > 16 ? 32 : 16;
        }
        if (lane < tcap && lane < ntc) {
            if (STORE) bs[tb + tc + lane] = tot;
            else bs[tb + tc + lane] += tot;
        }
    }
}

// FP64 form: same mapping, one target chunk of 32 at a time, absolute coordinates.
__global__ void __launch_bounds__(32 * kP2PWarps) k_p2p_f64(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ begin, const int32_t *__restrict__ end,
    const int32_t *__restrict__ uoffs, const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
    const int32_t *__restrict__ utot, const double2 *__restrict__ pos, const double *__restrict__ u, ShapeC shape,
    double *__restrict__ bs) {
    __shared__ double tgx[kP2PWarps][32], tgy[kP2PWarps][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int widx = blockIdx.x * kP2PWarps + w;
    if (widx >= nleaf) return;
    const int b = leaves[widx];
    const int tb = begin[b], nt = end[b] - tb;
    const int u0 = uoffs[b], u1 = uoffs[b + 1];
    const int St = utot[b];
    const double c2 = shape.of(b) * shape.of(b);
    for (int tc = 0; tc < nt; tc += 32) {
        const int ntc = min(32, nt - tc);
        if (lane < ntc) {
            tgx[w][lane] = pos[tb + tc + lane].x;
            tgy[w][lane] = pos[tb + tc + lane].y;
        }
        __syncwarp();
        double acc[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) acc[i] = 0;
        int r = u0;
        for (int q0 = 0; q0 < St; q0 += 32) {
            const int q = q0 + lane;
            double xs = 0, ys = 0, us = 0;
            if (q < St) {
                const int j = source_index(q, r, u1, ucum, uitems, begin);
                xs = pos[j].x;
                ys = pos[j].y;
                us = u[j];
            }
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                if (i < ntc) {
                    const double dx = tgx[w][i] - xs, dy = tgy[w][i] - ys;
                    acc[i] += us / sqrt(dx * dx + (dy * dy + c2));
                }
            }
        }
        const double tot = lane_reduce<double, 32>(acc, lane);
        if (lane < ntc) bs[tb + tc + lane] += tot;
        __syncwarp();
    }
}

}  // namespace

template <bool STORE, int W, int TCMAX>
void p2p_f32_launch_t(Plan &P, float *bs, cudaStream_t s) {
    const unsigned grid = (unsigned)((P.nleaf + W - 1) / W);
    const size_t smem = sizeof(WarpStage) * W;
    IMQ_CUDA(cudaFuncSetAttribute(k_p2p_f32<STORE, W, TCMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_p2p_f32<STORE, W, TCMAX><<<grid, 32 * W, smem, s>>>(
        P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(), P.end.as<int32_t>(), P.U.off.as<int32_t>(),
        P.U.items.as<int32_t>(), P.ucum.as<int32_t>(), P.utot.as<int32_t>(), P.uoff.as<float2>(), P.loc.as<float2>(),
        P.rec4.as<float4>(), P.shape(), bs, device_error_word());
    IMQ_LAUNCH_CHECK();
}

// The plan's P2P tile shape (warps per CTA, target chunk) selects the instance.
template <bool STORE, int W>
void p2p_f32_launch_w(Plan &P, float *bs, cudaStream_t s) {
    switch (P.p2p_chunk) {
        case 8: p2p_f32_launch_t<STORE, W, 8>(P, bs, s); break;
        case 32: p2p_f32_launch_t<STORE, W, 32>(P, bs, s); break;
        default: p2p_f32_launch_t<STORE, W, 16>(P, bs, s); break;
    }
}

template <bool STORE>
void p2p_f32_launch(Plan &P, const float *u, float *bs, cudaStream_t s) {
    if (!P.rec4.ptr) fail(IMQ_CUDA_ERROR, "P2P: record workspace missing");
    k_pack_records<<<blocks_for(P.N, 256), 256, 0, s>>>(P.loc.as<float2>(), u, P.N, P.rec4.as<float4>());
    IMQ_LAUNCH_CHECK();
    switch (P.p2p_warps) {
        case 2: p2p_f32_launch_w<STORE, 2>(P, bs, s); break;
        case 8: p2p_f32_launch_w<STORE, 8>(P, bs, s); break;
        default: p2p_f32_launch_w<STORE, 4>(P, bs, s); break;
    }
}

template <class T>
void p2p_apply(Plan &P, const T *u, T *bs, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        p2p_f32_launch<false>(P, u, bs, s);
    } else {
        const unsigned grid = (unsigned)((P.nleaf + kP2PWarps - 1) / kP2PWarps);
        k_p2p_f64<<<grid, 32 * kP2PWarps, 0, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(),
                                                  P.end.as<int32_t>(), P.U.off.as<int32_t>(), P.U.items.as<int32_t>(),
                                                  P.ucum.as<int32_t>(), P.utot.as<int32_t>(), P.pos.as<double2>(), u,
                                                  P.shape(), bs);
        IMQ_LAUNCH_CHECK();
    }
}

void p2p_near_f32(Plan &P, const float *u, float *near, cudaStream_t s) { p2p_f32_launch<true>(P, u, near, s); }

template void p2p_apply<float>(Plan &, const float *, float *, cudaStream_t);
template void p2p_apply<double>(Plan &, const double *, double *, cudaStream_t);

}  // namespace imq
