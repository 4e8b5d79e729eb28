// Inline-PTX helpers for sm_103a: mbarrier, 1-D TMA bulk copies, error flags.
// Every wait is bounded: after kSpinLimit polls or 0.5 s it reports failure
// instead of spinning forever, and the caller records an error word the host
// reads back.
#pragma once

#include <stdint.h>

namespace imq {

constexpr uint32_t kSpinLimit = 1u << 24;   // polls of try_wait before giving up
enum DeviceError : int {
    kErrWaitTimeout = 1,     // an mbarrier wait ran out
    kErrListOverflow = 2,    // a per-box list exceeded its fixed capacity
    kErrNonFinite = 4,       // NaN/Inf coordinate
    kErrDuplicate = 8,       // two points exactly equal
    kErrStackOverflow = 16,  // tree traversal stack exhausted
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Returns true when the phase with the given parity has completed.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait; returns false on timeout: after kSpinLimit polls, or once
// kWaitLimitNs of wall time have passed (each try_wait may suspend the thread
// for a while, so the poll count alone does not bound the time).
constexpr uint64_t kWaitLimitNs = 500000000ull;   // 0.5 s
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer_ns();
    for (uint32_t i = 1; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255u) == 0 && globaltimer_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

// 1-D bulk copy global -> shared, completing on an mbarrier (TMA, non-tensor form).
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void set_error(int *flag, int code) {
    if (flag) atomicOr(flag, code);
}

}  // namespace imq
