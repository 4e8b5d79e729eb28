// Inline-PTX helpers for the 5th-generation tensor cores of sm_103a:
// tcgen05.mma (kind::f16) with operands in shared memory and the accumulator in
// tensor memory (TMEM), tcgen05.ld for the drain, the 16-byte cp.async that
// gathers operand rows, and the power-of-two scaled fp16 hi / lo split of the
// M2L operands.  Operand layout: K-major, 64-byte swizzle (sw64_offset,
// umma_desc_sw64).
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include "ptx.cuh"

namespace imq {

__device__ __forceinline__ void cp_async16(uint32_t dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst_smem), "l"(src) : "memory");
}
// 16 bytes of zeros (no bytes read from src, which must still be a valid address)
__device__ __forceinline__ void cp_async16_zero(uint32_t dst_smem, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 0;" ::"r"(dst_smem), "l"(src) : "memory");
}
// arrive on an mbarrier once every cp.async issued so far by this thread has
// landed; the arrival is counted in the barrier's expected count (noinc)
__device__ __forceinline__ void cp_async_arrive_noinc(uint64_t *bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
// generic-proxy writes to shared memory -> visible to tcgen05.mma (async proxy)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// TMEM allocation: one full warp executes these.  ncols: power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem_word, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem_word)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 64-byte swizzle (the fp16 M2L): a row of 32 fp16 values is 64 bytes, an atom
// is 8 rows (512 bytes), and the 16-byte chunk j (values 8j .. 8j+7) of row r
// sits at chunk position j ^ ((r >> 1) & 3): the XOR of address bits 4-5 with
// bits 7-8.
__host__ __device__ __forceinline__ uint32_t sw64_offset(uint32_t r, uint32_t j) {
    return r * 64u + ((j ^ ((r >> 1) & 3u)) << 4);
}
// Shared-memory matrix descriptor of a K-major, 64-byte-swizzled operand.
// Fields: start address >> 4 (bits 0-13), leading byte offset >> 4 (16-29,
// unused by swizzled K-major layouts: 1), stride byte offset >> 4 (32-45: the
// 8-row atoms 512 bytes apart), descriptor version 1 (46-47), base offset 0
// (49-51), swizzle mode 4 = 64B (61-63).  A K-step of 16 fp16 values advances
// the start address by 32 bytes inside the atom.
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(512u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)4u << 61;
    return d;
}

// Instruction descriptor, kind::f16 with fp16 A and B (formats 0 at bits 7-9 and
// 10-12), D f32 (bits 4-5 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_f16(uint32_t M, uint32_t N) {
    return (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

// D[tmem] (+)= A * B^T for one K-step of 16 fp16 values; issued by a single thread.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Power-of-two scaling into the fp16 range: e with m 2^e in [2^13, 2^14) for the
// largest magnitude m of a row (0 for a zero or non-finite m), clamped so that
// 2^e and 2^-e are normal floats.
__device__ __forceinline__ int m2l_pow2_exp(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    return max(-120, min(120, 13 - ilogbf(m)));
}
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }
// Half index (even) inside the hi part of a packed fp16 multipole row where the row's
// inverse scale is kept as a float: past the K coefficients, inside the padding (for
// every K = (p+1)(p+2)/2 with p <= 18 the padding to a multiple of 32 leaves room).
__host__ __device__ constexpr int m2l_scale_slot(int K) { return (K + 1) & ~1; }

// fp16 split x = hi + lo (each rounded to nearest), for values already scaled into
// the fp16 range
__device__ __forceinline__ void f16_split(float x, __half &hi, __half &lo) {
    hi = __float2half_rn(x);
    lo = __float2half_rn(x - __half2float(hi));
}

// arrive on an mbarrier once every tcgen05.mma issued so far by this thread completes
__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// Issue (without waiting) a load of 32 lanes x 16 consecutive 32-bit columns:
// thread t of the warp gets lane (warp's lane quarter + t), columns
// [col, col + 16).  The registers are valid only after tmem_ld_wait_regs.
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
// Wait for every tcgen05.ld this thread issued; the N destination registers are
// tied to the wait (in groups of 16) so that no use of them is scheduled before it.
template <int N>
__device__ __forceinline__ void tmem_ld_wait_regs(uint32_t *r) {
    static_assert(N % 16 == 0, "groups of 16 registers");
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
#pragma unroll
    for (int g = 16; g < N; g += 16)
        asm volatile(""
                     : "+r"(r[g + 0]), "+r"(r[g + 1]), "+r"(r[g + 2]), "+r"(r[g + 3]), "+r"(r[g + 4]),
                       "+r"(r[g + 5]), "+r"(r[g + 6]), "+r"(r[g + 7]), "+r"(r[g + 8]), "+r"(r[g + 9]),
                       "+r"(r[g + 10]), "+r"(r[g + 11]), "+r"(r[g + 12]), "+r"(r[g + 13]), "+r"(r[g + 14]),
                       "+r"(r[g + 15])
                     :
                     : "memory");
}

}  // namespace imq
