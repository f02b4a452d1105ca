// Bulk asynchronous copies (global -> shared) completing on an mbarrier.
//
// One thread arms the barrier with the number of bytes it expects
// (mbarrier.arrive.expect_tx) and issues cp.async.bulk copies that signal
// completion on it; every thread then waits for the barrier phase.  Each copy
// must start and end on 16-byte boundaries in both spaces.  Waits are
// bounded: after kMbarTimeoutCycles of polling a wait gives up and returns
// false, so a kernel can record an error and return instead of hanging.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fdas {

constexpr long long kMbarTimeoutCycles = 2000000000LL;   // about one second

__device__ __forceinline__ unsigned smem_u32(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// make the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

// order earlier shared-memory accesses of this thread before later
// asynchronous-proxy accesses (bulk copies into a reused buffer)
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// raise the barrier's expected transaction bytes without arriving (several
// threads can each announce their own copies before one of them arrives)
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// plain arrival on an mbarrier
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes,
                                              uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// non-blocking probe of the given phase (cheaper than try_wait when the
// phase is usually complete already)
__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned phase) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// wait for the given phase of the barrier; false once `limit` clock cycles
// have passed without it
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned phase,
                                          long long limit = kMbarTimeoutCycles) {
    if (mbar_try_wait(bar, phase)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, phase))
        if (clock64() - t0 > limit) return false;
    return true;
}

}  // namespace fdas
