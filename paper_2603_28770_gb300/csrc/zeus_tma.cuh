// zeus_tma.cuh -- inline PTX for one-dimensional bulk copies from global to
// shared memory (the TMA unit's cp.async.bulk) completed on an mbarrier, as
// the streamed-H pass uses them: one thread issues the copy of a chunk, the
// block waits on the chunk's mbarrier phase.  sm_90 and later; every wait
// here is bounded by the caller.
#pragma once

#include <stdint.h>

namespace zeus {

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// an mbarrier with `count` expected arrivals per phase
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

// make barrier initialisation and earlier shared-memory writes visible to
// the async proxy (the bulk-copy unit)
__device__ __forceinline__ void fence_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// order this thread's earlier global-memory writes before later reads of
// the same memory by the async proxy
__device__ __forceinline__ void fence_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// one arrival that also announces `bytes` of transfer for this phase
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// bulk copy of `bytes` (multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, counted on `bar`
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// true once the phase of parity `parity` has completed (non-blocking)
__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// waits for the phase of parity `parity`, at most `limit` polls (the first
// few back to back, then about 64 ns apart); false if it gave up
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, unsigned limit) {
    for (unsigned spin = 0;; ++spin) {
        if (mbar_test(bar, parity)) return true;
        if (spin >= limit) return false;
        if (spin >= 16) __nanosleep(64);
    }
}

}  // namespace zeus
