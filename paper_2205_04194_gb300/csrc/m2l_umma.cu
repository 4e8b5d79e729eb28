// M2L on the tensor cores (tcgen05, kind::f16 with an fp16 hi/lo split).
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
// (zero if it has none).  A_o is gathered by 16-byte cp.async from packed rows
// of M (one padded row per box), T_o arrives as a pre-swizzled image, and the
// accumulator D lives in tensor memory (one TMEM lane per target box, one
// column per local coefficient).
//
// Precision: each operand is scaled by a power of two into the fp16 range (a
// row of M by its box's scale, a row of T_l by its output coefficient's scale,
// shared by the 40 classes of the level) and split into an fp16 head and tail
// (x = hi + lo, 11 significant bits each).  D accumulates hi*lo + lo*hi and then
// hi*hi in FP32 (small terms first), so the products carry about 22 significant
// bits, as a 3xTF32 split does, with half the operand bytes and twice the tensor
// rate.  The drain takes the box scale out of every chunk and the coefficient
// scale out of the sum.
//
// Pipeline: the K dimension of each class is cut into 32-wide chunks (64-byte
// rows, 64-byte swizzle); a chunk's A and T tiles form one shared-memory stage.
// One thread issues the 6 MMAs of a chunk and commits them to the stage's
// mbarrier, which releases the stage for reuse.  Every wait is bounded and
// reports kErrWaitTimeout through the device error word.
#include <algorithm>

#include "imq_internal.h"
#include "ptx.cuh"
#include "umma.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kTB = 128;               // target boxes per tile = MMA M
constexpr int kAStage = 8192;          // 128 rows x 64 bytes (32 fp16), one of hi / lo
constexpr int kMaxStages = 8;
// Four producer warps take the chunks in turn, and each waits on its stage's "empty" barrier by
// phase parity.  A warp at chunk g has seen chunk g - 4 - S committed (its previous wait), so with
// S >= 4 the barrier is at most one phase behind and the parity cannot alias; fewer stages are
// never used.
constexpr int kMinStages = 4;
constexpr size_t kStaticSmem = 2048;   // bound on the kernel's static shared memory
// one CTA per SM: the kernel allocates all 512 TMEM columns, so a second CTA on the same SM would
// wait in its allocation; asking for more than half of the SM's shared memory rules that out
constexpr size_t kMinSmem = 116 * 1024;

struct UmmaDims {
    int K, Kout, KP, NKC, Kn, tcols, stages;
    size_t stage_bytes() const { return 2 * (size_t)kAStage + 2 * (size_t)Kn * 64; }
    size_t smem() const { return std::max(kMinSmem, (size_t)stages * stage_bytes() + 1024); }
};

UmmaDims umma_dims(int K, int Kout) {
    UmmaDims d{};
    d.K = K;
    d.Kout = Kout;
    d.NKC = (K + 31) / 32;
    d.KP = 32 * d.NKC;
    d.Kn = (Kout + 15) / 16 * 16;
    d.tcols = (d.Kn + 31) / 32;   // accumulator column groups (NC)
    d.stages = 6;
    while (d.stages > kMinStages && d.smem() + kStaticSmem > 227 * 1024) --d.stages;
    return d;
}

// Packed row of box b (2 KP fp16 values): [hi(s_b M_b) | 0 pad to KP | lo(s_b M_b) | 0 pad],
// s_b = 2^e_b (m2l_pow2_exp of max |M_b|); 1 / s_b is stored as a float in two pad halfs of
// the hi part (m2l_scale_slot), where the operator image is zero.
__global__ void k_pack_m(const float *__restrict__ M, int64_t nbox, int K, int KP, float *__restrict__ Mpk) {
    const int64_t b = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nbox) return;
    const float *Mb = M + b * K;
    float mx = 0.f;
    for (int k = lane; k < K; k += 32) mx = fmaxf(mx, fabsf(Mb[k]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    const int e = m2l_pow2_exp(mx);
    const float sc = pow2f(e);
    __half *row = reinterpret_cast<__half *>(Mpk) + b * 2 * KP;
    for (int k = lane; k < KP; k += 32) {
        __half hi = __float2half_rn(0.f), lo = hi;
        if (k < K) f16_split(Mb[k] * sc, hi, lo);
        row[k] = hi;
        row[KP + k] = lo;
    }
    __syncwarp();
    if (lane == 0) *reinterpret_cast<float *>(row + m2l_scale_slot(K)) = pow2f(-e);
}

// Per (block, output coefficient j): t_inv[blk][j] = 2^-f with 2^f scaling max over the 40
// classes and the K inputs of |T_jk| into the fp16 range.  One warp per (blk, j).
__global__ void k_m2l_row_scales(const float *__restrict__ ops, int nblk, int K, int Kp, int Kout, int Kn,
                                 float *__restrict__ t_inv) {
    const int64_t w = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= (int64_t)nblk * Kn) return;
    const int blk = (int)(w / Kn), j = (int)(w - (int64_t)blk * Kn);
    float mx = 0.f;
    if (j < Kout)
        for (int e = lane; e < kOffsetClasses * K; e += 32)
            mx = fmaxf(mx, fabsf(ops[(((int64_t)blk * kOffsetClasses) * K + e) * Kp + j]));
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
    if (lane == 0) t_inv[w] = pow2f(-m2l_pow2_exp(mx));
}

// Operator images: for each (block, class, chunk) the hi and lo tiles of the scaled T_o
// restricted to inputs [32 kc, 32 kc + 32), rows = outputs 0..Kn-1, fp16 in the 64-byte-swizzled
// K-major layout.  ops: [nblk][40][K][Kp] input-major FP32.
__global__ void k_m2l_images(const float *__restrict__ ops, int64_t nblk, int K, int Kp, int Kout, int Kn, int NKC,
                             const float *__restrict__ t_inv, unsigned char *__restrict__ img) {
    const int64_t per = (int64_t)NKC * Kn * 4;   // 16-byte chunks per (block, class) and part
    const int64_t total = nblk * kOffsetClasses * per;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bo = e / per;                 // block * 40 + class
        int64_t r = e - bo * per;
        const int kc = (int)(r / (Kn * 4));
        r -= (int64_t)kc * Kn * 4;
        const int j = (int)(r / 4), jj = (int)(r - (int64_t)j * 4);
        const float sc = 1.f / t_inv[(bo / kOffsetClasses) * Kn + j];   // a power of two: exact
        __align__(16) __half hi[8], lo[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = kc * 32 + 8 * jj + q;
            const float v = (k < K && j < Kout) ? ops[(bo * K + k) * Kp + j] : 0.f;
            f16_split(v * sc, hi[q], lo[q]);
        }
        unsigned char *base = img + ((size_t)bo * NKC + kc) * (2 * (size_t)Kn * 64);
        *reinterpret_cast<uint4 *>(base + sw64_offset(j, jj)) = *reinterpret_cast<const uint4 *>(hi);
        *reinterpret_cast<uint4 *>(base + (size_t)Kn * 64 + sw64_offset(j, jj)) = *reinterpret_cast<const uint4 *>(lo);
    }
}

// Warp roles (416 threads):
//   warps 0-7  drain: warp w reads TMEM lane quarter w % 4 (thread b of the
//              quarter owns target row 32 (w % 4) + b) and column half w / 4 of
//              the accumulator; after each chunk it loads its NC x 16 columns
//              with back-to-back tcgen05.ld and one wait, multiplies them by the
//              inverse scale of the row's source box and adds them to FP32
//              registers; at the end it takes out the coefficient scales and
//              adds the sums to the target's local coefficients;
//   warps 8-11 producers: warp q gathers the 128 rows of A (hi and lo) of every
//              fourth chunk by cp.async, four lanes per 64-byte row, and its
//              lanes arrive on the stage's barrier through
//              cp.async.mbarrier.arrive.noinc; its lane 0 also issues the bulk
//              copy of the operator image;
//   warp 12    lane 0 issues the 6 MMAs of each chunk into one of NA TMEM
//              accumulators and commits them to the stage's "empty" barrier and
//              the accumulator's "full" barrier.
// Barriers: full[S] (33 arrivals + image bytes), empty[S] (MMA commit),
// acc_full[NA] (MMA commit), acc_empty[NA] (8 drain warps); NA accumulators
// rotate so that the MMAs of chunk it wait only for the drain of chunk it - NA.
// A work item is (tile, part): a tile's offset classes are split over nsplit
// CTAs, which add their partial sums to L with one RED per element each.
constexpr int kDrainWarps = 8, kDrainThreads = 32 * kDrainWarps, kProdWarps = 4, kProdThreads = 32 * kProdWarps;
constexpr int kThreadsWS = kDrainThreads + kProdThreads + 32;

constexpr int kRing = 16;   // tile records in flight between the roles (a tile has >= 1 chunk)

// inverse scale of a packed source row (0 for no source: its row is zero anyway)
__device__ __forceinline__ float row_inv_scale(const __half *Mpk, int src, int KP, int slot) {
    return src >= 0 ? __ldg(reinterpret_cast<const float *>(Mpk + (int64_t)src * 2 * KP + slot)) : 0.f;
}

// Persistent: one CTA per SM pulls work items (tile, part) in the plan's order
// (heaviest first) from a device counter until none is left.  The producer
// leader fetches an item, writes its record (tile, class list) into a ring
// slot and arrives on the slot's barrier; the MMA issuer and the drain read
// the record after waiting on that barrier.  Chunk counters run across tiles,
// so the pipeline never drains between tiles, and TMEM and the barriers are
// set up once per CTA.  S (pipeline stages, <= kMaxStages) is a launch argument.
template <int NC>
__global__ void __launch_bounds__(kThreadsWS, 1)
    k_m2l_umma(const int4 *__restrict__ tiles, const uint64_t *__restrict__ tmask, const int32_t *__restrict__ order,
               const int32_t *__restrict__ tbox, const int32_t *__restrict__ vtab, const __half *__restrict__ Mpk,
               float *__restrict__ L, const unsigned char *__restrict__ img, const float *__restrict__ t_inv,
               int K, int Kout, int Kn, int NKC, int S, int n_items, int nsplit, int *counter, int *err) {
    constexpr uint32_t kAccCols = NC <= 2 ? 64 : NC <= 4 ? 128 : 256;   // columns per accumulator
    constexpr int NA = NC <= 4 ? 4 : 2;                                   // accumulators in rotation
    constexpr uint32_t kTCols = NA * kAccCols;                            // <= 512
    extern __shared__ unsigned char smraw[];
    __shared__ int s_tix[kRing], s_ncls[kRing];
    __shared__ int8_t s_cls[kRing][kOffsetClasses];
    __shared__ volatile int s_abort;
    __shared__ __align__(8) uint64_t s_full[kMaxStages], s_empty[kMaxStages], s_accf[4], s_acce[4], s_ring[kRing];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const uint32_t raw0 = smem_u32(smraw);
    const uint32_t sbase = (raw0 + 1023u) & ~1023u;
    const uint32_t img_bytes = 2u * (uint32_t)Kn * 64u;
    const uint32_t stage_bytes = 2u * kAStage + img_bytes;
    const int KP = 32 * NKC;
    const int slot_sc = m2l_scale_slot(K);

    if (w == 0) tmem_alloc(&s_tmem, kTCols);
    if (tid == 32) {
        s_abort = 0;
        for (int i = 0; i < S; ++i) {
            mbar_init(&s_full[i], 32 + 1);   // one producer warp's lanes + the image bytes
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
        const int quarter = w & 3, half = w >> 2, row = quarter * 32 + lane;
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
            const int tgt = row < tile.z ? tbox[tile.y + row] : -1;
            // inverse scale of this row's source in the current class, and the next class's
            float isc = 0.f, isc_next =
                tgt >= 0 ? row_inv_scale(Mpk, __ldg(vtab + (int64_t)kOffsetClasses * tgt + s_cls[slot][0]), KP, slot_sc)
                         : 0.f;
            float acc[H];
#pragma unroll
            for (int i = 0; i < H; ++i) acc[i] = 0.f;
            // every 32-wide K chunk is drained and summed in FP32 registers: fewer partial sums
            // accumulated inside the tensor core keep the split products' precision
            const int nitems = ncls * NKC;
            for (int it = 0; it < nitems; ++it, ++g) {
                const int ci = it / NKC, kc = it - ci * NKC;
                if (kc == 0) {
                    isc = isc_next;
                    isc_next = (tgt >= 0 && ci + 1 < ncls)
                                   ? row_inv_scale(Mpk, __ldg(vtab + (int64_t)kOffsetClasses * tgt + s_cls[slot][ci + 1]),
                                                   KP, slot_sc)
                                   : 0.f;
                }
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
                            for (int i = 0; i < 16; ++i)
                                acc[(c0 + c) * 16 + i] = fmaf(__uint_as_float(v[16 * c + i]), isc, acc[(c0 + c) * 16 + i]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s_acce[g % NA]);
            }
            if (!ok) break;
            if (tgt >= 0) {
                float *Lb = L + (int64_t)tgt * Kout + half * H;
                const float *ti = t_inv + (int64_t)tile.x * Kn + half * H;
                const int ncol = min(H, Kout - half * H);
#pragma unroll
                for (int i = 0; i < H; ++i)
                    if (i < ncol) atomicAdd(Lb + i, acc[i] * __ldg(ti + i));   // onto the P2L terms: a RED
            }
        }
    } else if (w < kDrainWarps + kProdWarps) {
        // ---------------------------------------------------------------- producers
        // Producer warp q gathers every kProdWarps-th chunk (global chunk g with
        // g % kProdWarps == q) on its own, so the serial latency of one chunk's issue
        // overlaps with the other warps' chunks.  No lane waits for its copies: each
        // chunk ends with an arrive that the hardware performs once the lane's copies
        // have landed, so the producers run up to S chunks ahead of the MMAs.
        const int q = w - kDrainWarps;
        const int j = lane & 3;
        int g = 0;   // chunks of the tiles before this one (the same on every producer warp)
        for (int t = 0;; ++t) {
            const int slot = t % kRing;
            if (q == 0 && lane == 0) {
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
            // lane l copies 16-byte chunk (l & 3) of rows (l >> 2) + 8 k, k < 16
            int tgt[16], src[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int row = (lane >> 2) + 8 * k;
                tgt[k] = row < nbt ? tbox[b0 + row] : -1;
            }
            const int nitems = ncls * NKC;
            int cls = -1;   // class whose sources src[] holds
            for (int it = (q - g % kProdWarps + kProdWarps) % kProdWarps; it < nitems; it += kProdWarps) {
                const int gg = g + it, st = gg % S;
                const int ci = it / NKC, kc = it - ci * NKC, o = s_cls[slot][ci];
                if (ci != cls) {
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        src[k] = tgt[k] >= 0 ? __ldg(vtab + (int64_t)kOffsetClasses * tgt[k] + o) : -1;
                    cls = ci;
                }
                int okw = 1;
                if (lane == 0) okw = (!s_abort && (gg < S || mbar_wait(&s_empty[st], (uint32_t)((gg / S) + 1) & 1u)));
                if (!__shfl_sync(0xFFFFFFFFu, okw, 0)) {
                    ok = false;
                    break;
                }
                const uint32_t sa = sbase + (uint32_t)st * stage_bytes;
                if (lane == 0) {
                    mbar_arrive_expect_tx(&s_full[st], img_bytes);
                    bulk_g2s(smraw + (sa - raw0) + 2 * kAStage,
                             img + (((size_t)blk * kOffsetClasses + o) * NKC + kc) * (size_t)img_bytes, img_bytes,
                             &s_full[st]);
                }
                // 4 consecutive lanes fetch the 4 16-byte chunks of one 64-byte row
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    const int row = (lane >> 2) + 8 * k;
                    const int sb = src[k];
                    const uint32_t off = sw64_offset((uint32_t)row, (uint32_t)j);
                    if (sb >= 0) {
                        const __half *mh = Mpk + (int64_t)sb * 2 * KP + kc * 32 + 8 * j;
                        cp_async16(sa + off, mh);
                        cp_async16(sa + kAStage + off, mh + KP);
                    } else {
                        cp_async16_zero(sa + off, Mpk);
                        cp_async16_zero(sa + kAStage + off, Mpk);
                    }
                }
                cp_async_arrive_noinc(&s_full[st]);
            }
            g += nitems;
            // a failed wait sets s_abort (below) and the leader then hands out no more tiles: the
            // producers leave the loop together, right after the named barrier, so none of them
            // waits at that barrier for one that has left
            if (!ok) s_abort = 1;
        }
        cp_async_wait<0>();
    } else if (lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = umma_idesc_f16(kTB, (uint32_t)Kn);
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
                const uint32_t bh = sa + 2 * kAStage, bl = bh + (uint32_t)Kn * 64u;
                const uint32_t d = tmem + (uint32_t)(g % NA) * kAccCols;
                // the small products first (hi*lo, lo*hi over both K halves), then hi*hi: the
                // tensor core's FP32 sum then adds the large terms to a small partial sum instead
                // of the small terms to a large one
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint64_t dah = umma_desc_sw64(sa + 32 * ks), dal = umma_desc_sw64(sa + kAStage + 32 * ks);
                    const uint64_t dbh = umma_desc_sw64(bh + 32 * ks), dbl = umma_desc_sw64(bl + 32 * ks);
                    umma_f16(d, dah, dbl, idesc, ks > 0 ? 1u : 0u);
                    umma_f16(d, dal, dbh, idesc, 1u);
                }
#pragma unroll
                for (int ks = 0; ks < 2; ++ks)
                    umma_f16(d, umma_desc_sw64(sa + 32 * ks), umma_desc_sw64(bh + 32 * ks), idesc, 1u);
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
    if (K < 1 || Kout < 1 || K > 192 || Kout > 192) return false;   // up to 6 accumulator column groups
    const UmmaDims d = umma_dims(K, Kout);
    if (m2l_scale_slot(K) + 2 > d.KP) return false;   // room for the row's scale in its padding
    return d.stages >= kMinStages && d.smem() + kStaticSmem <= 227 * 1024;
}

void m2l_umma_prepare(const Plan &P, const float *ops, int nblk, int Kout, DevMem &img, DevMem &Mpk, DevMem &tmask,
                      DevMem &order, DevMem &counter, cudaStream_t s) {
    const int K = P.layout.K;
    const UmmaDims d = umma_dims(K, Kout);
    const int Kp = 16 * m2l_tiled_rows(Kout);
    // images, then the per-(block, coefficient) inverse scales
    const size_t img_bytes = (size_t)nblk * kOffsetClasses * d.NKC * 2 * (size_t)d.Kn * 64;
    img.alloc(img_bytes + sizeof(float) * (size_t)std::max(1, nblk) * d.Kn);
    unsigned char *ib = img.as<unsigned char>();
    float *t_inv = reinterpret_cast<float *>(ib + img_bytes);
    if (nblk > 0) {
        const int64_t rows = (int64_t)nblk * d.Kn;
        k_m2l_row_scales<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(ops, nblk, K, Kp, Kout, d.Kn, t_inv);
        IMQ_LAUNCH_CHECK();
        const int64_t chunks = (int64_t)nblk * kOffsetClasses * d.NKC * d.Kn * 4;
        k_m2l_images<<<blocks_for(chunks, 256), 256, 0, s>>>(ops, nblk, K, Kp, Kout, d.Kn, d.NKC, t_inv, ib);
        IMQ_LAUNCH_CHECK();
    }
    // packed fp16 rows: 2 KP halfs = KP floats per box
    Mpk.alloc(sizeof(float) * (size_t)P.nbox * d.KP);
    // the pads past K stay zero: the fused writers (P2M, M2M) store only the first K of each half
    // (and the scale in its slot)
    IMQ_CUDA(cudaMemsetAsync(Mpk.ptr, 0, sizeof(float) * (size_t)P.nbox * d.KP, s));
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
int m2l_umma_min_stages() { return kMinStages; }

void m2l_umma_launch(const Plan &P, const float *M, float *L, const TypedOps &O, int Kout, cudaStream_t s,
                     bool packed) {
    if (P.n_m2l_tiles == 0) return;
    const int K = P.layout.K;
    UmmaDims d = umma_dims(K, Kout);
    // the plan's tile choice: fewer pipeline stages than fit (never more, never fewer than kMinStages)
    if (P.m2l_stages >= kMinStages && P.m2l_stages < d.stages) d.stages = P.m2l_stages;
    float *Mpk = O.Mpk.as<float>();
    if (!packed) {
        k_pack_m<<<(unsigned)((P.nbox + 7) / 8), 256, 0, s>>>(M, P.nbox, K, d.KP, Mpk);
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
    const unsigned char *img = O.m2l_img.as<unsigned char>();
    const int nblk = O.m2l_nblk;
    const float *t_inv =
        reinterpret_cast<const float *>(img + (size_t)nblk * kOffsetClasses * d.NKC * 2 * (size_t)d.Kn * 64);
    const uint64_t *tmask = O.m2l_tmask.as<uint64_t>();
    const int32_t *order = O.m2l_order.as<int32_t>();
    const __half *mp = reinterpret_cast<const __half *>(Mpk);
#define IMQ_UMMA_CASE(NCC)                                                                                        \
    if (d.tcols == NCC) {                                                                                        \
        IMQ_CUDA(cudaFuncSetAttribute(k_m2l_umma<NCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));  \
        k_m2l_umma<NCC><<<grid, kThreadsWS, smem, s>>>(P.m2l_tiles.as<int4>(), tmask, order,                      \
                                                       P.m2l_tbox.as<int32_t>(), P.vtab.as<int32_t>(), mp, L, img, \
                                                       t_inv, K, Kout, d.Kn, d.NKC, d.stages, n_items, nsplit,     \
                                                       counter, err);                                              \
        launched = true;                                                                                          \
    }
    bool launched = false;
    IMQ_UMMA_CASE(1)
    IMQ_UMMA_CASE(2)
    IMQ_UMMA_CASE(3)
    IMQ_UMMA_CASE(4)
    IMQ_UMMA_CASE(5)
    IMQ_UMMA_CASE(6)
#undef IMQ_UMMA_CASE
    if (!launched) fail(IMQ_UNSUPPORTED, "M2L: no tensor-core kernel for this expansion size");
    IMQ_LAUNCH_CHECK();
}

}  // namespace imq
