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
#include <algorithm>
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

// Per product: 16-byte records per sorted point, x and y the offset from the
// point's leaf centre: rec = (x, y, u0, u1) (u1 = 0 for one right-hand side) and,
// for up to four right-hand sides, recb = (u2, u3, 0, 0).
__global__ void k_pack_records(const float2 *__restrict__ loc, const float *__restrict__ u, int64_t n, int nr,
                               float4 *__restrict__ rec, float4 *__restrict__ recb) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const float2 l = loc[i];
        rec[i] = make_float4(l.x, l.y, u[i], nr > 1 ? u[n + i] : 0.f);
        if (nr > 2) recb[i] = make_float4(u[2 * n + i], nr > 3 ? u[3 * n + i] : 0.f, 0.f, 0.f);
    }
}

constexpr int kStageCap = 512;    // source records staged per warp at a time (8 KB per record array)

template <int NR>
struct WarpStage {
    float4 rec[kStageCap];
    float4 recb[NR > 2 ? kStageCap : 1];
    uint64_t bar;
};

// Stage concatenated positions [q0, q0 + len) of the U-list sources of one leaf
// into shared memory with 1-D TMA bulk copies, one per overlapping U entry and
// record array, the entries spread over the lanes (lane e sets up entry u0 + e,
// u0 + e + 32, ...); wait for them (bounded), then shift each entry's records
// into the target leaf's frame, the entry bounds and offset broadcast from the
// lane that loaded them.  St: total source count of the leaf.  Returns false if
// the wait timed out.
template <int NR>
__device__ __forceinline__ bool stage_sources(WarpStage<NR> &ws, uint32_t &phase, int q0, int len, int u0, int u1,
                                              int St, const int32_t *__restrict__ begin,
                                              const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
                                              const float2 *__restrict__ udelta, const float4 *__restrict__ rec,
                                              const float4 *__restrict__ recb, int lane, int *err) {
    if (lane == 0) {
        // earlier generic-proxy writes to ws.rec must be ordered before the async-proxy copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&ws.bar, (uint32_t)len * 16u * (NR > 2 ? 2u : 1u));
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
        if (a < bnd) {
            const int64_t src = begin[uitems[r]] + (a - lo);
            bulk_g2s(&ws.rec[a - q0], rec + src, (uint32_t)(bnd - a) * 16u, &ws.bar);
            if (NR > 2) bulk_g2s(&ws.recb[a - q0], recb + src, (uint32_t)(bnd - a) * 16u, &ws.bar);
        }
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

// One kernel value per (source, target) pair serves all NR right-hand sides.
template <int TC, int NR>
__device__ __forceinline__ void p2p_tile_f32(const WarpStage<NR> &ws, int len, int lane, const u64 (&tx)[TC / 2],
                                             const u64 (&ty)[TC / 2], u64 (&acc)[NR][TC / 2], u64 cc) {
    for (int q0 = 0; q0 < len; q0 += 32) {
        const int q = q0 + lane;
        const float4 sr = q < len ? ws.rec[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 sb = make_float4(0.f, 0.f, 0.f, 0.f);
        if (NR > 2 && q < len) sb = ws.recb[q];
        const u64 nx = pk2(-sr.x, -sr.x), ny = pk2(-sr.y, -sr.y);
        u64 uu[NR];
        uu[0] = pk2(sr.z, sr.z);
        if (NR > 1) uu[1] = pk2(sr.w, sr.w);
        if (NR > 2) uu[2] = pk2(sb.x, sb.x);
        if (NR > 3) uu[3] = pk2(sb.y, sb.y);
#pragma unroll
        for (int k = 0; k < TC / 2; ++k) {
            const u64 dx = add2(tx[k], nx);
            const u64 dy = add2(ty[k], ny);
            const u64 d2 = fma2(dx, dx, fma2(dy, dy, cc));
            float a, b;
            up2(d2, a, b);
            const u64 rr = pk2(rsqrtf(a), rsqrtf(b));
#pragma unroll
            for (int m = 0; m < NR; ++m) acc[m][k] = fma2(rr, uu[m], acc[m][k]);
        }
    }
}

// Sums of one chunk of up to TC targets for every right-hand side; lane L ends with
// target L % TC's total in tot[m].
template <int TC, int NR>
__device__ __forceinline__ void p2p_chunk_staged(WarpStage<NR> &ws, uint32_t &phase, bool staged_all, int ti, int ntc,
                                                 int lane, int u0, int u1, int St, const int32_t *__restrict__ begin,
                                                 const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum,
                                                 const float2 *__restrict__ udelta, const float2 *__restrict__ loc,
                                                 const float4 *__restrict__ rec, const float4 *__restrict__ recb,
                                                 float c2, int *err, float (&tot)[NR]) {
    u64 tx[TC / 2], ty[TC / 2], acc[NR][TC / 2];
#pragma unroll
    for (int q = 0; q < TC / 2; ++q) {
        const int i0 = 2 * q, i1 = 2 * q + 1;
        const float2 a = i0 < ntc ? loc[ti + i0] : make_float2(kFar, kFar);
        const float2 b = i1 < ntc ? loc[ti + i1] : make_float2(kFar, kFar);
        tx[q] = pk2(a.x, b.x);
        ty[q] = pk2(a.y, b.y);
#pragma unroll
        for (int m = 0; m < NR; ++m) acc[m][q] = 0ull;
    }
    const u64 cc = pk2(c2, c2);
    if (staged_all) {
        p2p_tile_f32<TC, NR>(ws, St, lane, tx, ty, acc, cc);
    } else {
        for (int q0 = 0; q0 < St; q0 += kStageCap) {
            const int len = min(kStageCap, St - q0);
            if (!stage_sources<NR>(ws, phase, q0, len, u0, u1, St, begin, uitems, ucum, udelta, rec, recb, lane, err))
                break;
            p2p_tile_f32<TC, NR>(ws, len, lane, tx, ty, acc, cc);
            __syncwarp();
        }
    }
#pragma unroll
    for (int m = 0; m < NR; ++m) {
        float sm[TC];
#pragma unroll
        for (int k = 0; k < TC / 2; ++k) up2(acc[m][k], sm[2 * k], sm[2 * k + 1]);
        tot[m] = lane_reduce<float, TC>(sm, lane);
    }
}

// STORE: write the near-field sums (b_near = sum); otherwise add them to bs.  W warps per
// CTA; each warp pulls target leaves from a device counter (the plan's order, most pairs
// first) until none is left; targets in chunks of at most TCMAX; NR right-hand sides.
template <bool STORE, int W, int TCMAX, int NR>
__global__ void __launch_bounds__(32 * W) k_p2p_f32(
    int nleaf, const int32_t *__restrict__ leaves, const int32_t *__restrict__ order, int *counter,
    const int32_t *__restrict__ begin, const int32_t *__restrict__ end, const int32_t *__restrict__ uoffs,
    const int32_t *__restrict__ uitems, const int32_t *__restrict__ ucum, const int32_t *__restrict__ utot,
    const float2 *__restrict__ udelta, const float2 *__restrict__ loc, const float4 *__restrict__ rec,
    const float4 *__restrict__ recb, ShapeC shape, int64_t n, float *__restrict__ bs, int *err) {
    extern __shared__ __align__(128) unsigned char smraw_p2p[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStage<NR> &ws = reinterpret_cast<WarpStage<NR> *>(smraw_p2p)[w];
    if (lane == 0) {
        mbar_init(&ws.bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    uint32_t phase = 0;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item >= nleaf) break;
        const int b = leaves[order[item]];
        const int tb = begin[b], nt = end[b] - tb;
        const int u0 = uoffs[b], u1 = uoffs[b + 1];
        const int St = utot[b];
        const double cb = shape.of(b);
        const float c2 = (float)(cb * cb);
        const bool staged_all = St <= kStageCap;
        if (staged_all &&
            !stage_sources<NR>(ws, phase, 0, St, u0, u1, St, begin, uitems, ucum, udelta, rec, recb, lane, err))
            break;
        for (int tc = 0; tc < nt; tc += TCMAX) {
            const int ntc = min(TCMAX, nt - tc);
            float tot[NR];
            int tcap;
            if (ntc <= 8) {
                p2p_chunk_staged<8, NR>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St, begin, uitems, ucum,
                                        udelta, loc, rec, recb, c2, err, tot);
                tcap = 8;
            } else if (TCMAX == 16 || ntc <= 16) {
                p2p_chunk_staged<16, NR>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St, begin, uitems,
                                         ucum, udelta, loc, rec, recb, c2, err, tot);
                tcap = 16;
            } else {
                p2p_chunk_staged<(TCMAX > 16 ? 32 : 16), NR>(ws, phase, staged_all, tb + tc, ntc, lane, u0, u1, St,
                                                             begin, uitems, ucum, udelta, loc, rec, recb, c2, err,
                                                             tot);
                tcap = TCMAX > 16 ? 32 : 16;
            }
            if (lane < tcap && lane < ntc) {
#pragma unroll
                for (int m = 0; m < NR; ++m) {
                    float *o = bs + (int64_t)m * n + tb + tc + lane;
                    if (STORE) *o = tot[m];
                    else *o += tot[m];
                }
            }
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

template <bool STORE, int W, int TCMAX, int NR>
void p2p_f32_launch_t(Plan &P, float *bs, cudaStream_t s) {
    const size_t smem = sizeof(WarpStage<NR>) * W;
    auto kern = k_p2p_f32<STORE, W, TCMAX, NR>;
    IMQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent: enough CTAs to fill every SM several times over, each warp pulling leaves
    static int n_sm[64] = {0}, per_sm[64][2][3][3] = {};
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) fail(IMQ_UNSUPPORTED, "P2P: device index out of range");
    if (n_sm[dev] == 0) IMQ_CUDA(cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev));
    int &occ = per_sm[dev][W == 2 ? 0 : W == 4 ? 1 : 2][NR == 1 ? 0 : NR == 2 ? 1 : 2][TCMAX == 8 ? 0 : TCMAX == 16 ? 1 : 2];
    if (occ == 0) IMQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * W, smem));
    const int64_t want = ((int64_t)P.nleaf + W - 1) / W;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)n_sm[dev] * std::max(1, occ)));
    IMQ_CUDA(cudaMemsetAsync(P.p2p_counter.ptr, 0, sizeof(int), s));
    kern<<<grid, 32 * W, smem, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.p2p_order.as<int32_t>(),
                                    P.p2p_counter.as<int>(), P.begin.as<int32_t>(), P.end.as<int32_t>(),
                                    P.U.off.as<int32_t>(), P.U.items.as<int32_t>(), P.ucum.as<int32_t>(),
                                    P.utot.as<int32_t>(), P.uoff.as<float2>(), P.loc.as<float2>(), P.rec4.as<float4>(),
                                    NR > 2 ? P.rec4b.as<float4>() : nullptr, P.shape(), P.N, bs, device_error_word());
    IMQ_LAUNCH_CHECK();
}

// The plan's P2P tile shape (warps per CTA, target chunk) selects the instance.
template <bool STORE, int W, int NR>
void p2p_f32_launch_w(Plan &P, float *bs, cudaStream_t s) {
    switch (P.p2p_chunk) {
        case 8: p2p_f32_launch_t<STORE, W, 8, NR>(P, bs, s); break;
        case 32: p2p_f32_launch_t<STORE, W, 32, NR>(P, bs, s); break;
        default: p2p_f32_launch_t<STORE, W, 16, NR>(P, bs, s); break;
    }
}

template <bool STORE, int NR>
void p2p_f32_launch_r(Plan &P, float *bs, cudaStream_t s) {
    switch (P.p2p_warps) {
        case 2: p2p_f32_launch_w<STORE, 2, NR>(P, bs, s); break;
        case 8: p2p_f32_launch_w<STORE, 8, NR>(P, bs, s); break;
        default: p2p_f32_launch_w<STORE, 4, NR>(P, bs, s); break;
    }
}

// u, bs: [nrhs][N]; the right-hand sides go through the kernel four at a time
template <bool STORE>
void p2p_f32_launch(Plan &P, const float *u, float *bs, int nrhs, cudaStream_t s) {
    if (!P.rec4.ptr || !P.p2p_order.ptr) fail(IMQ_CUDA_ERROR, "P2P: record workspace or leaf order missing");
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
        const int nr = std::min(4, nrhs - r0);
        if (nr > 2 && !P.rec4b.ptr) fail(IMQ_CUDA_ERROR, "P2P: second record workspace missing");
        k_pack_records<<<blocks_for(P.N, 256), 256, 0, s>>>(P.loc.as<float2>(), u + (size_t)r0 * P.N, P.N, nr,
                                                            P.rec4.as<float4>(), P.rec4b.as<float4>());
        IMQ_LAUNCH_CHECK();
        float *b = bs + (size_t)r0 * P.N;
        if (nr == 1) p2p_f32_launch_r<STORE, 1>(P, b, s);
        else if (nr == 2) p2p_f32_launch_r<STORE, 2>(P, b, s);
        else p2p_f32_launch_r<STORE, 4>(P, b, s);
    }
}

template <class T>
void p2p_apply(Plan &P, const T *u, T *bs, cudaStream_t s) {
    if constexpr (std::is_same<T, float>::value) {
        p2p_f32_launch<false>(P, u, bs, 1, s);
    } else {
        const unsigned grid = (unsigned)((P.nleaf + kP2PWarps - 1) / kP2PWarps);
        k_p2p_f64<<<grid, 32 * kP2PWarps, 0, s>>>(P.nleaf, P.leaves.as<int32_t>(), P.begin.as<int32_t>(),
                                                  P.end.as<int32_t>(), P.U.off.as<int32_t>(), P.U.items.as<int32_t>(),
                                                  P.ucum.as<int32_t>(), P.utot.as<int32_t>(), P.pos.as<double2>(), u,
                                                  P.shape(), bs);
        IMQ_LAUNCH_CHECK();
    }
}

void p2p_near_f32(Plan &P, const float *u, float *near, int nrhs, cudaStream_t s) {
    p2p_f32_launch<true>(P, u, near, nrhs, s);
}

template void p2p_apply<float>(Plan &, const float *, float *, cudaStream_t);
template void p2p_apply<double>(Plan &, const double *, double *, cudaStream_t);

}  // namespace imq
