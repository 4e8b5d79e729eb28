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
#include "imq_internal.h"
#include "ptx.cuh"
#include "umma.cuh"
#include "util.cuh"

namespace imq {
namespace {

constexpr int kTB = 128;         // target boxes per tile = MMA M
constexpr int kThreads = 128;    // thread b gathers and stores target row b
constexpr int kAStage = 16384;   // 128 rows x 128 bytes, one of hi / lo

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
    d.stages = 3;
    while (d.stages > 2 && d.smem() + sizeof(int) * kOffsetClasses * (kTB + 1) + 256 > 227 * 1024) --d.stages;
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

// S: shared-memory stages; NC: 32-column groups of the accumulator (Kn <= 32 NC)
template <int S, int NC>
__global__ void __launch_bounds__(kThreads, 1)
    k_m2l_umma(const int4 *__restrict__ tiles, const int32_t *__restrict__ tbox, const int32_t *__restrict__ vtab,
               const float *__restrict__ Mpk, float *__restrict__ L, const float *__restrict__ img, int Kout, int Kn,
               int NKC, int *err) {
    constexpr uint32_t kAccCols = NC <= 2 ? 64 : NC <= 4 ? 128 : 256;   // column offset of accumulator 1
    constexpr uint32_t kTCols = 2 * kAccCols;
    extern __shared__ unsigned char smraw[];
    __shared__ int s_src[kOffsetClasses][kTB];
    __shared__ int s_cls[kOffsetClasses];
    __shared__ int s_present[kOffsetClasses];
    __shared__ int s_ncls, s_abort;
    __shared__ __align__(8) uint64_t s_bar[S];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, w = tid >> 5;
    const uint32_t raw0 = smem_u32(smraw);
    const uint32_t sbase = (raw0 + 1023u) & ~1023u;
    const uint32_t stage_bytes = 2u * kAStage + 2u * (uint32_t)Kn * 128u;
    const int KP = 32 * NKC;
    const int4 tile = tiles[blockIdx.x];
    const int blk = tile.x, b0 = tile.y, nbt = tile.z;

    if (w == 0) tmem_alloc(&s_tmem, kTCols);
    if (tid < kOffsetClasses) s_present[tid] = 0;
    if (tid == 0) {
        s_abort = 0;
        for (int i = 0; i < S; ++i) mbar_init(&s_bar[i], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int t = tid < nbt ? tbox[b0 + tid] : -1;
    for (int o = 0; o < kOffsetClasses; ++o) {
        const int sb = t >= 0 ? vtab[(int64_t)kOffsetClasses * t + o] : -1;
        s_src[o][tid] = sb;
        if (sb >= 0) s_present[o] = 1;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
        int n = 0;
        for (int o = 0; o < kOffsetClasses; ++o)
            if (s_present[o]) s_cls[n++] = o;
        s_ncls = n;
    }
    __syncthreads();
    const uint32_t tmem = s_tmem;
    const uint32_t tlane = (uint32_t)(w * 32) << 16;
    const int nitems = s_ncls * NKC;
    const unsigned char *imgb = reinterpret_cast<const unsigned char *>(img);

    auto load = [&](int it) {
        const int o = s_cls[it / NKC], kc = it - (it / NKC) * NKC;
        const uint32_t st = sbase + (uint32_t)(it % S) * stage_bytes;
        const int sb = s_src[o][tid];
        const float *mh = Mpk + (int64_t)sb * 2 * KP + kc * 32;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const uint32_t off = sw128_offset((uint32_t)tid, (uint32_t)j);
            if (sb >= 0) {
                cp_async16(st + off, mh + 4 * j);
                cp_async16(st + kAStage + off, mh + KP + 4 * j);
            } else {
                st_shared_zero16(st + off);
                st_shared_zero16(st + kAStage + off);
            }
        }
        const unsigned char *src = imgb + (((size_t)blk * kOffsetClasses + o) * NKC + kc) * (2 * (size_t)Kn * 128);
        const int n16 = Kn * 16;   // 2 parts x Kn rows x 8 chunks
        for (int e = tid; e < n16; e += kThreads) cp_async16(st + 2 * kAStage + 16u * e, src + 16 * (size_t)e);
    };

    // Each chunk accumulates into a fresh TMEM accumulator (the two alternate)
    // and is added to FP32 registers once its MMAs complete: long accumulation
    // chains inside the tensor core lose precision, one chunk of 12 MMAs does not.
    float acc[NC * 32];
#pragma unroll
    for (int i = 0; i < NC * 32; ++i) acc[i] = 0.f;
    bool ok = true;
    auto drain = [&](int it) {   // every thread: wait for item it, add its accumulator
        const bool got = mbar_wait(&s_bar[it % S], (uint32_t)(it / S) & 1u);
        if (!__all_sync(0xFFFFFFFFu, got)) {   // the TMEM loads below need the whole warp
            ok = false;
            s_abort = 1;
            return;
        }
        tc_fence_after();
        const uint32_t a = tmem + tlane + (uint32_t)(it & 1) * kAccCols;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float v[32];
            tmem_ld32(a + (uint32_t)(c * 32), v);
#pragma unroll
            for (int i = 0; i < 32; ++i) acc[c * 32 + i] += v[i];
        }
        tc_fence_before();
    };

    const uint32_t idesc = umma_idesc_tf32(kTB, (uint32_t)Kn);
#pragma unroll
    for (int it = 0; it < S - 1; ++it) {
        if (it < nitems) load(it);
        cp_async_commit();
    }
    for (int it = 0; it < nitems; ++it) {
        cp_async_wait<S - 2>();
        fence_proxy_async_smem();
        __syncthreads();   // stage it landed; accumulator (it & 1) drained (item it - 2)
        if (s_abort) break;
        if (tid == 0) {
            tc_fence_after();
            const uint32_t st = sbase + (uint32_t)(it % S) * stage_bytes;
            const uint32_t bh = st + 2 * kAStage, bl = bh + (uint32_t)Kn * 128u;
            const uint32_t d = tmem + (uint32_t)(it & 1) * kAccCols;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t dah = umma_desc_sw128(st + 32 * ks), dal = umma_desc_sw128(st + kAStage + 32 * ks);
                const uint64_t dbh = umma_desc_sw128(bh + 32 * ks), dbl = umma_desc_sw128(bl + 32 * ks);
                umma_tf32(d, dah, dbh, idesc, ks > 0 ? 1u : 0u);
                umma_tf32(d, dah, dbl, idesc, 1u);
                umma_tf32(d, dal, dbh, idesc, 1u);
            }
            umma_commit(&s_bar[it % S]);
        }
        __syncwarp();
        // item it - 1 done: its accumulator is added and its stage is free for item it + S - 1
        if (it >= 1) drain(it - 1);
        const int nx = it + S - 1;
        if (nx < nitems && ok) load(nx);
        cp_async_commit();
    }
    cp_async_wait<0>();
    __syncthreads();
    if (nitems > 0 && !s_abort) drain(nitems - 1);
    if (!ok) set_error(err, kErrWaitTimeout);
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    if (nitems > 0 && all_ok && tid < nbt) {
        float *Lb = L + (int64_t)tbox[b0 + tid] * Kout;
#pragma unroll
        for (int i = 0; i < NC * 32; ++i)
            if (i < Kout) Lb[i] = acc[i];
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (w == 0) tmem_dealloc(tmem, kTCols);
}

}  // namespace

bool m2l_umma_supported(int K, int Kout) {
    if (K < 1 || Kout < 1 || K > 256 || Kout > 256) return false;
    const UmmaDims d = umma_dims(K, Kout);
    return d.smem() + sizeof(int) * kOffsetClasses * (kTB + 2) + 256 <= 227 * 1024;
}

void m2l_umma_prepare(const Plan &P, const float *ops, int nblk, int Kout, DevMem &img, DevMem &Mpk, cudaStream_t s) {
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
}

void m2l_umma_launch(const Plan &P, const float *M, float *L, const float *img, float *Mpk, int Kout, cudaStream_t s) {
    if (P.n_m2l_tiles == 0) return;
    const int K = P.layout.K;
    const UmmaDims d = umma_dims(K, Kout);
    k_pack_m<<<blocks_for((int64_t)P.nbox * d.KP, 256), 256, 0, s>>>(M, P.nbox, K, d.KP, Mpk);
    IMQ_LAUNCH_CHECK();
    const size_t smem = d.smem();
    int *err = device_error_word();
#define IMQ_UMMA_CASE(SS, NCC)                                                                                    \
    if (d.stages == SS && d.tcols == NCC) {                                                                      \
        IMQ_CUDA(cudaFuncSetAttribute(k_m2l_umma<SS, NCC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
        k_m2l_umma<SS, NCC><<<P.n_m2l_tiles, kThreads, smem, s>>>(P.m2l_tiles.as<int4>(), P.m2l_tbox.as<int32_t>(), \
                                                                 P.vtab.as<int32_t>(), Mpk, L, img, Kout, d.Kn,    \
                                                                 d.NKC, err);                                      \
        launched = true;                                                                                          \
    }
    bool launched = false;
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
