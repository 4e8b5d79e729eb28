// M2L on the tensor cores (tcgen05, kind::tf32 with a 3xTF32 split).
//
// The multipole-to-local translation of the value path (the far-field terms
// the paper sums over the well-separated set S_p, Section 3, Algorithm 1) is
// L_B = sum_{S in V(B)} T_{l,o(S,B)} M_S with a K x K real operator per level l
// and offset class o (40 classes).  A tile of up to 128 target boxes of one
// level and one quadrant (27 classes) is one GEMM chain:
//
//   D[128 x Kn] = sum_o  A_o[128 x K] * T_o^T[K x Kn]
//
// where row b of A_o is the multipole vector of the class-o source of target b
// (zero if it has none).  A_o is gathered by 16-byte cp.async from a packed
// copy of M (one padded row per box), T_o arrives as a pre-swizzled image, and
// the accumulator D lives in tensor memory (one TMEM lane per target box,
// one column per local coefficient).  Each operand is split into a tf32 head
// and a tf32 tail (x = hi + lo), and D accumulates hi*hi + hi*lo + lo*hi, so
// the products carry about 22 significant bits, close to FP32.
//
// Pipeline: the K dimension of each class is cut into 32-wide chunks; a
// chunk's A and T tiles form one shared-memory stage.  All threads gather the
// stage S-1 chunks ahead; one thread issues the 12 MMAs of a chunk and commits
// them to the stage's mbarrier, which releases the stage for reuse.  Every
// wait is bounded and reports kErrWaitTimeout through the device error word.
#include <algorithm>

#include "imq_internal.h"
#include "ptx.cuh"
#include "umma.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kTB = 128;         // target boxes per tile = MMA M
constexpr int kAStage = 16384;   // 128 rows x 128 bytes, one of hi / lo
constexpr size_t kStaticSmem = 1024;   // bound on the kernel's static shared memory

struct UmmaDims {
    int K, Kout, KP, NKC, Kn, tcols, stages;
    size_t stage_bytes() const { return 2 * (size_t)kAStage + 2 * (size_t)Kn * 128; }
    size_t smem() const { return (size_t)stages * stage_bytes() + 1024; }
};

UmmaDims umma_dims(int K, int Kout) {
    UmmaDims d{};
    d.K = K;
    d.Kout = Kout;
    d.NKC = (K + 31) / 32;
    d.KP = 32 * d.NKC;
    d.Kn = (Kout + 15) / 16 * 16;
    d.tcols = (d.Kn + 31) / 32;   // accumulator column groups (NC)
    d.stages = 4;
    while (d.stages > 2 && d.smem() + kStaticSmem > 227 * 1024) --d.stages;
    return d;
}

// Mpk[box] = [hi(M_box) | 0 pad to KP | lo(M_box) | 0 pad]
__global__ void k_pack_m(const float *__restrict__ M, int64_t nbox, int K, int KP, float *__restrict__ Mpk) {
    const int64_t total = nbox * KP;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / KP;
        const int k = (int)(e - b * KP);
        const float v = k < K ? M[b * K + k] : 0.f;
        const float hi = tf32_round(v);
        Mpk[b * 2 * KP + k] = hi;
        Mpk[b * 2 * KP + KP + k] = tf32_round(v - hi);
    }
}

// Operator images: for each (block, class, chunk) the hi and lo tiles of
// T_o restricted to inputs [32 kc, 32 kc + 32), rows = outputs 0..Kn-1, in the
// swizzled K-major layout.  ops: [nblk][40][K][Kp] input-major FP32.
__global__ void k_m2l_images(const float *__restrict__ ops, int64_t nblk, int K, int Kp, int Kout, int Kn, int NKC,
                             float *__restrict__ img) {
    const int64_t per = (int64_t)NKC * Kn * 8;   // 16-byte chunks per (block, class) and part
    const int64_t total = nblk * kOffsetClasses * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bo = e / per;                 // block * 40 + class
        int64_t r = e - bo * per;
        const int kc = (int)(r / (Kn * 8));
        r -= (int64_t)kc * Kn * 8;
        const int j = (int)(r / 8), jj = (int)(r - (int64_t)j * 8);
        float hi[4], lo[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = kc * 32 + 4 * jj + q;
            const float v = (k < K && j < Kout) ? ops[(bo * K + k) * Kp + j] : 0.f;
            hi[q] = tf32_round(v);
            lo[q] = tf32_round(v - hi[q]);
        }
        unsigned char *base = reinterpret_cast<unsigned char *>(img) + ((size_t)bo * NKC + kc) * (2 * (size_t)Kn * 128);
        *reinterpret_cast<float4 *>(base + sw128_offset(j, jj)) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(base + (size_t)Kn * 128 + sw128_offset(j, jj)) =
            make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

// Warp roles (416 threads):
//   warps 0-7  drain: warp w reads TMEM lane quarter w % 4 (thread b of the
//              quarter owns target row 32 (w % 4) + b) and column half w / 4 of
//              the accumulator; after each chunk it loads its NC x 16 columns
//              with back-to-back tcgen05.ld and one wait, adds them to FP32
//              registers, and at the end adds them to the target's local
//              coefficients;
//   warps 8-11 producers: gather the 128 rows of A (hi and lo) by cp.async,
//              eight threads per 128-byte row, and arrive on the stage's
//              barrier through cp.async.mbarrier.arrive.noinc; the first
//              producer thread also issues the bulk copy of the operator image;
//   warp 12    lane 0 issues the 12 MMAs of each chunk into one of NA TMEM
//              accumulators and commits them to the stage's "empty" barrier and
//              the accumulator's "full" barrier.
// Barriers: full[S] (129 arrivals + image bytes), empty[S] (MMA commit),
// acc_full[NA] (MMA commit), acc_empty[NA] (8 drain warps); NA accumulators
// rotate so that the MMAs of chunk it wait only for the drain of chunk it - NA.
// A work item is (tile, part): a tile's offset classes are split over nsplit
// CTAs, which add their partial sums to L with one RED per element each.
constexpr int kDrainWarps = 8, kDrainThreads = 32 * kDrainWarps, kProdThreads = 128;
constexpr int kThreadsWS = kDrainThreads + kProdThreads + 32;

constexpr int kRing = 16;   // tile records in flight between the roles (a tile has >= 1 chunk)

// Persistent: one CTA per SM pulls work items (tile, part) in the plan's order
// (heaviest first) from a device counter until none is left.  The producer
// leader fetches an item, writes its record (tile, class list) into a ring
// slot and arrives on the slot's barrier; the MMA issuer and the drain read
// the record after waiting on that barrier.  Chunk counters run across tiles,
// so the pipeline never drains between tiles, and TMEM and the barriers are
// set up once per CTA.
template <int S, int NC>
__global__ void __launch_bounds__(kThreadsWS, 1)
    k_m2l_umma(const int4 *__restrict__ tiles, const uint64_t *__restrict__ tmask, const int32_t *__restrict__ order,
               const int32_t *__restrict__ tbox, const int32_t *__restrict__ vtab, const float *__restrict__ Mpk,
               float *__restrict__ L, const float *__restrict__ img, int Kout, int Kn, int NKC, int n_items,
               int nsplit, int *counter, int *err) {
    constexpr uint32_t kAccCols = NC <= 2 ? 64 : NC <= 4 ? 128 : 256;   // columns per accumulator
    constexpr int NA = NC <= 4 ? 4 : 2;                                   // accumulators in rotation
    constexpr uint32_t kTCols = NA * kAccCols;                            // <= 512
    extern __shared__ unsigned char smraw[];
    __shared__ int s_tix[kRing], s_ncls[kRing];
    __shared__ int8_t s_cls[kRing][kOffsetClasses];
    __shared__ volatile int s_abort;
    __shared__ __align__(8) uint64_t s_full[S], s_empty[S], s_accf[4], s_acce[4], s_ring[kRing];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t raw0 = smem_u32(smraw);
    const uint32_t sbase = (raw0 + 1023u) & ~1023u;
    const uint32_t img_bytes = 2u * (uint32_t)Kn * 128u;
    const uint32_t stage_bytes = 2u * kAStage + img_bytes;
    const int KP = 32 * NKC;

    if (w == 0) tmem_alloc(&s_tmem, kTCols);
    if (tid == 32) {
        s_abort = 0;
        for (int i = 0; i < S; ++i) {
            mbar_init(&s_full[i], kProdThreads + 1);
            mbar_init(&s_empty[i], 1);
        }
        for (int i = 0; i < NA; ++i) {
            mbar_init(&s_accf[i], 1);
            mbar_init(&s_acce[i], kDrainWarps);
        }
        for (int i = 0; i < kRing; ++i) mbar_init(&s_ring[i], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    bool ok = true;

    if (w < kDrainWarps) {
        // ---------------------------------------------------------------- drain
        constexpr int H = NC * 16;                 // columns of this warp's half
        constexpr int BL = NC <= 3 ? NC : 2;       // 16-column loads in flight per wait
        const int quarter = w & 3, half = w >> 2;
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * H);
        int g = 0;   // chunk counter across tiles
        for (int t = 0;; ++t) {
            const int slot = t % kRing;
            if (!__all_sync(0xFFFFFFFFu, mbar_wait(&s_ring[slot], (uint32_t)(t / kRing) & 1u)) || s_abort) {
                ok = false;
                break;
            }
            const int ncls = s_ncls[slot];
            if (ncls < 0) break;
            const int4 tile = tiles[s_tix[slot]];
            float acc[H];
#pragma unroll
            for (int i = 0; i < H; ++i) acc[i] = 0.f;
            // every 32-wide K chunk is drained and summed in FP32 registers: fewer partial sums
            // accumulated inside the tensor core keep the tf32 products' precision
            const int nitems = ncls * NKC;
            for (int it = 0; it < nitems; ++it, ++g) {
                const bool got = mbar_wait(&s_accf[g % NA], (uint32_t)(g / NA) & 1u);
                if (!__all_sync(0xFFFFFFFFu, got) || s_abort) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a = tl + (uint32_t)(g % NA) * kAccCols;
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += BL) {
                    uint32_t v[BL * 16];
#pragma unroll
                    for (int c = 0; c < BL; ++c)
                        if (c0 + c < NC) tmem_ld16_issue(a + (uint32_t)((c0 + c) * 16), v + 16 * c);
                    tmem_ld_wait_regs<BL * 16>(v);
#pragma unroll
                    for (int c = 0; c < BL; ++c)
                        if (c0 + c < NC)
#pragma unroll
                            for (int i = 0; i < 16; ++i) acc[(c0 + c) * 16 + i] += __uint_as_float(v[16 * c + i]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_acce[g % NA]);
            }
            if (!ok) break;
            const int row = quarter * 32 + lane;
            if (row < tile.z) {
                float *Lb = L + (int64_t)tbox[tile.y + row] * Kout + half * H;
                const int ncol = min(H, Kout - half * H);
#pragma unroll
                for (int i = 0; i < H; ++i)
                    if (i < ncol) atomicAdd(Lb + i, acc[i]);   // onto the P2L terms in L: a RED, no load
            }
        }
    } else if (w < kDrainWarps + 4) {
        // ---------------------------------------------------------------- producers
        // No producer waits for its own copies: each chunk ends with an arrive
        // that the hardware performs once the thread's copies have landed, so
        // the producers run up to S chunks ahead of the MMAs.
        const int r = tid - kDrainThreads;
        const int j = r & 7;
        const unsigned char *imgb = reinterpret_cast<const unsigned char *>(img);
        int g = 0;
        for (int t = 0;; ++t) {
            const int slot = t % kRing;
            if (r == 0) {
                // next work item with at least one class (empty ones are skipped here)
                int ncls = -1, tix = 0;
                for (;;) {
                    const int item = s_abort ? n_items : atomicAdd(counter, 1);
                    if (item >= n_items) break;
                    tix = order[item / nsplit];
                    const int part = item - (item / nsplit) * nsplit;
                    const uint64_t mk = tmask[tix];
                    const int all = __popcll(mk);
                    const int c0 = (all * part) / nsplit, c1 = (all * (part + 1)) / nsplit;
                    int n = 0, k = 0;
                    for (int o = 0; o < kOffsetClasses; ++o)
                        if ((mk >> o) & 1ull) {
                            if (k >= c0 && k < c1) s_cls[slot][n++] = (int8_t)o;
                            ++k;
                        }
                    if (n > 0) {
                        ncls = n;
                        break;
                    }
                }
                s_tix[slot] = tix;
                s_ncls[slot] = ncls;
                mbar_arrive(&s_ring[slot]);   // release: the record is visible to whoever waits on it
            }
            asm volatile("bar.sync 1, %0;" ::"n"(kProdThreads) : "memory");   // producers only
            const int ncls = s_ncls[slot];
            if (ncls < 0) break;
            const int4 tile = tiles[s_tix[slot]];
            const int blk = tile.x, b0 = tile.y, nbt = tile.z;
            // producer thread r gathers chunk (r & 7) of rows (r >> 3) + 16 k, k < 8
            int tgt[8], src[8], nxt[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int row = (r >> 3) + 16 * k;
                tgt[k] = row < nbt ? tbox[b0 + row] : -1;
                src[k] = -1;
                nxt[k] = tgt[k] >= 0 ? __ldg(vtab + (int64_t)kOffsetClasses * tgt[k] + s_cls[slot][0]) : -1;
            }
            const int nitems = ncls * NKC;
            for (int it = 0; it < nitems; ++it, ++g) {
                const int st = g % S;
                if (s_abort || (g >= S && !mbar_wait(&s_empty[st], (uint32_t)((g / S) + 1) & 1u))) {
                    ok = false;
                    break;
                }
                const int ci = it / NKC, o = s_cls[slot][ci], kc = it - ci * NKC;
                if (kc == 0) {   // the next class's sources are loaded while this class is gathered
#pragma unroll
                    for (int k = 0; k < 8; ++k) src[k] = nxt[k];
                    if (ci + 1 < ncls) {
                        const int o1 = s_cls[slot][ci + 1];
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            nxt[k] = tgt[k] >= 0 ? __ldg(vtab + (int64_t)kOffsetClasses * tgt[k] + o1) : -1;
                    }
                }
                const uint32_t sa = sbase + (uint32_t)st * stage_bytes;
                if (r == 0) {
                    mbar_arrive_expect_tx(&s_full[st], img_bytes);
                    bulk_g2s(smraw + (sa - raw0) + 2 * kAStage,
                             imgb + (((size_t)blk * kOffsetClasses + o) * NKC + kc) * (size_t)img_bytes, img_bytes,
                             &s_full[st]);
                }
                // 8 consecutive threads fetch the 8 16-byte chunks of one 128-byte row, so a
                // warp instruction reads 4 whole rows (full sectors) rather than 32 fragments
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int row = (r >> 3) + 16 * k;
                    const int sb = src[k];
                    const uint32_t off = sw128_offset((uint32_t)row, (uint32_t)j);
                    if (sb >= 0) {
                        const float *mh = Mpk + (int64_t)sb * 2 * KP + kc * 32 + 4 * j;
                        cp_async16(sa + off, mh);
                        cp_async16(sa + kAStage + off, mh + KP);
                    } else {
                        cp_async16_zero(sa + off, Mpk);
                        cp_async16_zero(sa + kAStage + off, Mpk);
                    }
                }
                cp_async_arrive_noinc(&s_full[st]);
            }
            // a failed wait sets s_abort (below) and the leader then hands out no more tiles: the
            // producers leave the loop together, right after the named barrier, so none of them
            // waits at that barrier for one that has left
            if (!ok) s_abort = 1;
        }
        cp_async_wait<0>();
    } else if (lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = umma_idesc_tf32(kTB, (uint32_t)Kn);
        int g = 0;
        for (int t = 0; ok; ++t) {
            const int slot = t % kRing;
            if (s_abort || !mbar_wait(&s_ring[slot], (uint32_t)(t / kRing) & 1u)) {
                ok = false;
                break;
            }
            const int ncls = s_ncls[slot];
            if (ncls < 0) break;
            const int nitems = ncls * NKC;
            for (int it = 0; it < nitems; ++it, ++g) {
                const int st = g % S;
                if (s_abort || !mbar_wait(&s_full[st], (uint32_t)(g / S) & 1u) ||
                    (g >= NA && !mbar_wait(&s_acce[g % NA], (uint32_t)((g / NA) + 1) & 1u))) {
                    ok = false;
                    break;
                }
                // the A rows were written by cp.async (generic proxy); the MMA reads them
                // through the async proxy
                fence_proxy_async_smem();
                tc_fence_after();
                const uint32_t sa = sbase + (uint32_t)st * stage_bytes;
                const uint32_t bh = sa + 2 * kAStage, bl = bh + (uint32_t)Kn * 128u;
                const uint32_t d = tmem + (uint32_t)(g % NA) * kAccCols;
#pragma unroll
                for (int ks = 0; ks < 4; ++ks) {
                    const uint64_t dah = umma_desc_sw128(sa + 32 * ks), dal = umma_desc_sw128(sa + kAStage + 32 * ks);
                    const uint64_t dbh = umma_desc_sw128(bh + 32 * ks), dbl = umma_desc_sw128(bl + 32 * ks);
                    umma_tf32(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                    umma_tf32(d, dah, dbl, idesc, 1u);
                    umma_tf32(d, dal, dbh, idesc, 1u);
                }
                umma_commit(&s_empty[st]);
                umma_commit(&s_accf[g % NA]);
            }
        }
        // the last commits must land before the CTA releases its TMEM
        if (ok && g > 0) {
            const int last = g - 1;
            if (!mbar_wait(&s_empty[last % S], (uint32_t)(last / S) & 1u)) ok = false;
        }
    }
    if (!ok) {
        s_abort = 1;
        set_error(err, kErrWaitTimeout);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_dealloc(tmem, kTCols);
}

// Bit o of mask[t] is set when some target box of tile t has a class-o V source.
// One warp per tile, lanes over its boxes.
__global__ void k_tile_masks(const int4 *__restrict__ tiles, int ntiles, const int32_t *__restrict__ tbox,
                             const int32_t *__restrict__ vtab, uint64_t *__restrict__ mask) {
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (t >= ntiles) return;
    const int4 tile = tiles[t];
    uint64_t m = 0;
    for (int row = lane; row < tile.z; row += 32) {
        const int b = tbox[tile.y + row];
        for (int o = 0; o < kOffsetClasses; ++o)
            if (vtab[(int64_t)kOffsetClasses * b + o] >= 0) m |= 1ull << o;
    }
#pragma unroll
    for (int k = 16; k >= 1; k >>= 1) m |= __shfl_xor_sync(0xFFFFFFFFu, m, k);
    if (lane == 0) mask[t] = m;
}

}  // namespace

bool m2l_umma_supported(int K, int Kout) {
    if (K < 1 || Kout < 1 || K > 256 || Kout > 256) return false;
    const UmmaDims d = umma_dims(K, Kout);
    return d.smem() + kStaticSmem <= 227 * 1024;
}

void m2l_umma_prepare(const Plan &P, const float *ops, int nblk, int Kout, DevMem &img, DevMem &Mpk, DevMem &tmask,
                      DevMem &order, DevMem &counter, cudaStream_t s) {
    const int K = P.layout.K;
    const UmmaDims d = umma_dims(K, Kout);
    const int Kp = 16 * m2l_tiled_rows(Kout);
    const size_t img_bytes = (size_t)nblk * kOffsetClasses * d.NKC * 2 * (size_t)d.Kn * 128;
    img.alloc(std::max<size_t>(16, img_bytes));
    const int64_t chunks = (int64_t)nblk * kOffsetClasses * d.NKC * d.Kn * 8;
    if (chunks > 0)
        k_m2l_images<<<blocks_for(chunks, 256), 256, 0, s>>>(ops, nblk, K, Kp, Kout, d.Kn, d.NKC, img.as<float>());
    IMQ_LAUNCH_CHECK();
    Mpk.alloc(sizeof(float) * (size_t)P.nbox * 2 * d.KP);
    // the pads past K stay zero: the fused writers (P2M, M2M) store only the first K of each half
    IMQ_CUDA(cudaMemsetAsync(Mpk.ptr, 0, sizeof(float) * (size_t)P.nbox * 2 * d.KP, s));
    const int nt = std::max(1, P.n_m2l_tiles);
    tmask.alloc(sizeof(uint64_t) * (size_t)nt);
    order.alloc(sizeof(int32_t) * (size_t)nt);
    counter.alloc(sizeof(int32_t));
    if (P.n_m2l_tiles > 0) {
        k_tile_masks<<<(P.n_m2l_tiles + 3) / 4, 128, 0, s>>>(P.m2l_tiles.as<int4>(), P.n_m2l_tiles,
                                                            P.m2l_tbox.as<int32_t>(), P.vtab.as<int32_t>(),
                                                            tmask.as<uint64_t>());
        IMQ_LAUNCH_CHECK();
        // the persistent kernel takes tiles heaviest first (classes x boxes), so the last
        // ones to start are the short ones
        std::vector<uint64_t> mk(P.n_m2l_tiles);
        std::vector<int4> tl(P.n_m2l_tiles);
        IMQ_CUDA(cudaMemcpyAsync(mk.data(), tmask.ptr, sizeof(uint64_t) * mk.size(), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaMemcpyAsync(tl.data(), P.m2l_tiles.ptr, sizeof(int4) * tl.size(), cudaMemcpyDeviceToHost, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
        std::vector<int32_t> ord(P.n_m2l_tiles);
        for (int t = 0; t < P.n_m2l_tiles; ++t) ord[t] = t;
        auto cost = [&](int t) { return (int64_t)__builtin_popcountll(mk[t]) * tl[t].z; };
        std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return cost(a) > cost(b); });
        IMQ_CUDA(cudaMemcpyAsync(order.ptr, ord.data(), sizeof(int32_t) * ord.size(), cudaMemcpyHostToDevice, s));
        IMQ_CUDA(cudaStreamSynchronize(s));
    }
}

int m2l_umma_kp(int K) { return 32 * ((K + 31) / 32); }

int m2l_default_split(int ntiles) {
    // measured at N = 1M clustered (384 tiles): splitting a tile's classes over more CTAs adds
    // per-CTA set-up and RED traffic faster than it evens out the last wave; the autotuner
    // measures other splits
    (void)ntiles;
    return 1;
}

int m2l_umma_max_stages(int K, int Kout) { return umma_dims(K, Kout).stages; }

void m2l_umma_launch(const Plan &P, const float *M, float *L, const TypedOps &O, int Kout, cudaStream_t s,
                     bool packed) {
    if (P.n_m2l_tiles == 0) return;
    const int K = P.layout.K;
    UmmaDims d = umma_dims(K, Kout);
    // the plan's tile choice: fewer pipeline stages than fit (never more)
    if (P.m2l_stages >= 2 && P.m2l_stages < d.stages) d.stages = P.m2l_stages;
    float *Mpk = O.Mpk.as<float>();
    if (!packed) {
        k_pack_m<<<blocks_for((int64_t)P.nbox * d.KP, 256), 256, 0, s>>>(M, P.nbox, K, d.KP, Mpk);
        IMQ_LAUNCH_CHECK();
    }
    const size_t smem = d.smem();
    int *err = device_error_word();
    // classes of a tile split over nsplit work items: the plan's choice, else one per tile
    const int nsplit = P.m2l_split > 0 ? P.m2l_split : m2l_default_split(P.n_m2l_tiles);
    const int n_items = P.n_m2l_tiles * nsplit;
    static int n_sm[64] = {0};
    int dev = 0;
    IMQ_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && n_sm[dev] == 0)
        IMQ_CUDA(cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev));
    const int grid = std::min(n_items, (dev >= 0 && dev < 64 && n_sm[dev] > 0) ? n_sm[dev] : 152);
    int *counter = O.m2l_counter.as<int>();
    IMQ_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), s));
    const float *img = O.m2l_img.as<float>();
    const uint64_t *tmask = O.m2l_tmask.as<uint64_t>();
    const int32_t *order = O.m2l_order.as<int32_t>();
#define IMQ_UMMA_CASE(SS, NCC)                                                                                    \
    if (d.stages == SS && d.tcols == NCC) {                                                                      \
        IMQ_CUDA(cudaFuncSetAttribute(k_m2l_umma<SS, NCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_m2l_umma<SS, NCC><<<grid, kThreadsWS, smem, s>>>(P.m2l_tiles.as<int4>(), tmask, order,                  \
                                                           P.m2l_tbox.as<int32_t>(), P.vtab.as<int32_t>(), Mpk, L,  \
                                                           img, Kout, d.Kn, d.NKC, n_items, nsplit, counter, err); \
        launched = true;                                                                                          \
    }
    bool launched = false;
    IMQ_UMMA_CASE(2, 1)
    IMQ_UMMA_CASE(2, 2)
    IMQ_UMMA_CASE(2, 3)
    IMQ_UMMA_CASE(2, 4)
    IMQ_UMMA_CASE(4, 1)
    IMQ_UMMA_CASE(4, 2)
    IMQ_UMMA_CASE(4, 3)
    IMQ_UMMA_CASE(3, 1)
    IMQ_UMMA_CASE(3, 2)
    IMQ_UMMA_CASE(3, 3)
    IMQ_UMMA_CASE(3, 4)
    IMQ_UMMA_CASE(2, 5)
    IMQ_UMMA_CASE(3, 5)
    IMQ_UMMA_CASE(2, 6)
    IMQ_UMMA_CASE(2, 7)
    IMQ_UMMA_CASE(2, 8)
#undef IMQ_UMMA_CASE
    if (!launched) fail(IMQ_UNSUPPORTED, "M2L: no tensor-core kernel for this expansion size");
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq
