// M2L on CUDA cores, batched by relative-offset class and register-tiled.
//
// For a box B and a source S of its V list (the paper's well-separated set
// S_p), the local coefficients of B receive T_{l,o} M_S, where the K x K real
// operator depends only on the level l and the integer offset o of S
// relative to B (40 classes).  One CTA owns a tile of up to kTB target boxes
// of one level and accumulates, in registers, the contributions of all 40
// classes:  L[:, tile] += sum_o T_{l,o} M[:, src(tile, o)]  (added to what P2L left there).
// Per class the operator (K x Kp, input-major, zero-padded rows) and the
// gathered source multipoles (kTB x Kpad, box-major, Kpad odd so that the
// column reads hit distinct banks) are staged in shared memory.  Thread
// (ty, tx) owns rows [ty*RR, ty*RR+RR) of columns {tx + 16 c : c < 8}: per
// input coefficient it loads RR operator values (broadcast, paired loads)
// and 8 multipole values and issues 8*RR FMAs.  All levels run in one launch
// from a host-built tile list, so small coarse levels overlap the fine ones.
#include "imq_internal.h"
#include "ptx.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kTB = 128;   // target boxes per tile
constexpr int kThreads = 256;

template <int RR>
__global__ void __launch_bounds__(kThreads) k_m2l_tiled(const int4 *__restrict__ tiles,
                                                        const int32_t *__restrict__ tbox,
                                                        const int32_t *__restrict__ vtab,
                                                        const float *__restrict__ M, float *__restrict__ L,
                                                        const float *__restrict__ ops, int K, int Kout, int Kpad) {
    // K: input (multipole) reals; Kout: output (local) reals, Kout <= 16*RR
    constexpr int Kp = 16 * RR;
    extern __shared__ __align__(16) unsigned char smraw[];
    float *Top = reinterpret_cast<float *>(smraw);        // [K][Kp]
    float *Ms = Top + (size_t)K * Kp;                     // [kTB][Kpad]  (Top: [K][Kp])
    __shared__ int srcs[kTB];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int4 tile = tiles[blockIdx.x];
    const int li = tile.x, b0 = tile.y, nbt = tile.z;   // boxes tbox[b0 .. b0+nbt)
    const float *opl = ops + (size_t)li * kOffsetClasses * K * Kp;
    float acc[RR][8];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;

    for (int o = 0; o < kOffsetClasses; ++o) {
        int s = -1;
        if (tid < kTB) {
            s = tid < nbt ? vtab[(int64_t)kOffsetClasses * tbox[b0 + tid] + o] : -1;
            srcs[tid] = s;
        }
        if (!__syncthreads_or(s >= 0)) continue;
        {
            const float4 *g = reinterpret_cast<const float4 *>(opl + (size_t)o * K * Kp);
            float4 *t4 = reinterpret_cast<float4 *>(Top);
            for (int e = tid; e < K * Kp / 4; e += kThreads) t4[e] = g[e];
        }
        for (int e = tid; e < kTB * K; e += kThreads) {
            const int col = e / K, i = e - col * K;
            const int sb = srcs[col];
            Ms[col * Kpad + i] = sb >= 0 ? M[(int64_t)sb * K + i] : 0.f;
        }
        __syncthreads();
        const float *trow = Top + ty * RR;
        const float *mcol = Ms + tx * Kpad;
#pragma unroll 2
        for (int i = 0; i < K; ++i) {
            float a[RR];
            if constexpr (RR % 2 == 0) {
#pragma unroll
                for (int r = 0; r < RR; r += 2) {
                    const float2 v = *reinterpret_cast<const float2 *>(trow + (size_t)i * Kp + r);
                    a[r] = v.x;
                    a[r + 1] = v.y;
                }
            } else {
#pragma unroll
                for (int r = 0; r < RR; ++r) a[r] = trow[(size_t)i * Kp + r];
            }
            float bv[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) bv[c] = mcol[c * 16 * Kpad + i];
#pragma unroll
            for (int r = 0; r < RR; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int col = tx + 16 * c;
        if (col >= nbt) continue;
        float *Lb = L + (int64_t)tbox[b0 + col] * Kout;
#pragma unroll
        for (int r = 0; r < RR; ++r) {
            const int row = ty * RR + r;
            if (row < Kout) atomicAdd(Lb + row, acc[r][c]);   // one add per element: a RED, no load
        }
    }
}

}  // namespace

int m2l_tiled_rows(int K) {
    const int rr = (K + 15) / 16;
    const int buckets[] = {3, 4, 5, 6, 8, 10, 12};
    for (int b : buckets)
        if (rr <= b) return b;
    return -1;
}

void m2l_tiled_launch(const Plan &P, const float *M, float *L, const float *ops, cudaStream_t s, int Kout) {
    const int K = P.layout.K;
    if (Kout <= 0) Kout = K;
    const int RR = m2l_tiled_rows(Kout);
    const int Kp = 16 * RR;
    const int Kpad = K | 1;
    const size_t smem = sizeof(float) * ((size_t)K * Kp + (size_t)kTB * Kpad);
    if (P.n_m2l_tiles == 0) return;
#define IMQ_M2L_T(R)                                                                                      \
    case R: {                                                                                             \
        auto kern = k_m2l_tiled<R>;                                                                       \
        IMQ_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));     \
        kern<<<P.n_m2l_tiles, kThreads, smem, s>>>(P.m2l_tiles.as<int4>(), P.m2l_tbox.as<int32_t>(),     \
                                                   P.vtab.as<int32_t>(), M, L,                            \
                                                   ops, K, Kout, Kpad);                                   \
        break;                                                                                            \
    }
    switch (RR) {
        IMQ_M2L_T(3)
        IMQ_M2L_T(4)
        IMQ_M2L_T(5)
        IMQ_M2L_T(6)
        IMQ_M2L_T(8)
        IMQ_M2L_T(10)
        IMQ_M2L_T(12)
        default: fail(IMQ_UNSUPPORTED, "M2L: expansion too large");
    }
#undef IMQ_M2L_T
    IMQ_LAUNCH_CHECK();
}

// Tiles hold boxes of one level and one quadrant within the parent: the V list
// of a box draws its offsets from the 27 classes fixed by its quadrant, so the
// other 13 class passes are skipped for the whole tile.
void build_m2l_tiles(Plan &P, cudaStream_t s) {
    std::vector<uint32_t> prefix(P.nbox);
    IMQ_CUDA(cudaMemcpyAsync(prefix.data(), P.prefix.ptr, sizeof(uint32_t) * P.nbox, cudaMemcpyDeviceToHost, s));
    IMQ_CUDA(cudaStreamSynchronize(s));
    std::vector<int4> t;
    std::vector<int32_t> order;
    for (int lev = P.m2l_level_lo; lev <= P.m2l_level_hi; ++lev) {
        const int lb = P.level_start[lev], le = P.level_start[lev + 1];
        for (int q = 0; q < 4; ++q) {
            const int start = (int)order.size();
            for (int b = lb; b < le; ++b)
                if ((int)(prefix[b] & 3u) == q) order.push_back(b);
            const int cnt = (int)order.size() - start;
            for (int k = 0; k < cnt; k += kTB)
                t.push_back(make_int4(lev - P.m2l_level_lo, start + k, std::min(kTB, cnt - k), 0));
        }
    }
    P.n_m2l_tiles = (int)t.size();
    P.m2l_tiles.alloc(sizeof(int4) * std::max<size_t>(1, t.size()));
    P.m2l_tbox.alloc(sizeof(int32_t) * std::max<size_t>(1, order.size()));
    if (!t.empty()) {
        IMQ_CUDA(cudaMemcpyAsync(P.m2l_tiles.ptr, t.data(), sizeof(int4) * t.size(), cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaMemcpyAsync(P.m2l_tbox.ptr, order.data(), sizeof(int32_t) * order.size(),
                                 cudaMemcpyHostToDevice, s));
    }
    IMQ_CUDA(cudaStreamSynchronize(s));
}

}  // namespace imq
