// Shared-memory mbarriers and bulk global->shared copies (cp.async.bulk, the
// TMA's untiled form) for the kernels that stream the plan tensor through a
// ring of shared-memory stages.
//
// Every wait is bounded: after kWaitLimitCycles (about one second at the
// GB300's clock) the waiting thread counts a timeout in the caller's device
// counter and returns false, so a copy that never lands cannot hang the GPU.
// The host reads and clears the counter through demag_wait_timeouts().
#pragma once
#include <cstdint>

namespace demag {

constexpr long long kWaitLimitCycles = 1LL << 31;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialisations visible to the other threads and to the async proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// One arrival that also announces `bytes` of transaction (the copies that follow).
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Tests the phase; a thread whose phase is not complete is suspended (it does
// not spin on issue slots) until the phase completes or about 10 us pass.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(10000u)
        : "memory");
    return done != 0;
}

// Waits for the phase of the given parity to complete; false (and one count
// in *timeouts) if it has not after `limit` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned *timeouts,
                                          long long limit = kWaitLimitCycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) {
            atomicAdd(timeouts, 1u);
            return false;
        }
    }
    return true;
}

// Bulk copy of `bytes` (a multiple of 16; both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace demag
