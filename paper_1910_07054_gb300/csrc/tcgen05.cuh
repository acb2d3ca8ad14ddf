// Fifth-generation tensor core (tcgen05) wrappers: tensor-memory allocation,
// shared-memory operand descriptors, the kind::tf32 MMA (A from shared or from
// tensor memory), completion through an mbarrier, tensor-memory stores and
// accumulator reads.
//
// Operands sit in shared memory in the K-major, unswizzled canonical layout:
// core matrices of 8 rows x 16 bytes (8 x 4 tf32), each 128 contiguous bytes;
// the descriptor's leading byte offset is the distance between core matrices
// adjacent along K, its stride byte offset the distance between 8-row groups.
// The accumulator D (M = 128) occupies TMEM lanes 0..127 (row r in lane r),
// one 32-bit column per output column.
#pragma once
#include <cstdint>

#include "mbar.cuh"

namespace demag {

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets, descriptor version 1, no base offset, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(unsigned saddr, unsigned lbo, unsigned sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32 with FP32 accumulation, both operands
// K-major: D format F32 (bits 4-5), A and B format TF32 (bits 7-9, 10-12),
// N / 8 (bits 17-22), M / 16 (bits 24-28).
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with BF16 operands and FP32
// accumulation, both operands K-major: D format F32 (bits 4-5), A and B format
// BF16 (bits 7-9, 10-12), N / 8 (bits 17-22), M / 16 (bits 24-28).  In tensor
// memory and in a 16-byte core-matrix row an operand word holds two BF16
// values, the lower K index in the low half.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Whole warp: allocate `ncols` TMEM columns (power of two, 32..512); the base
// address is written to *slot (shared memory).
__device__ __forceinline__ void tc_alloc(unsigned *slot, unsigned ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Whole warp (the allocating one): free the columns.
__device__ __forceinline__ void tc_dealloc(unsigned taddr, unsigned ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Makes this thread's generic-proxy shared-memory writes visible to the
// tensor core (which reads operands through the async proxy).
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One thread: D[tmem] (+)= A[adesc] * B[bdesc].
__device__ __forceinline__ void tc_mma_tf32(unsigned dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
        : "memory");
}

// One thread: D[tmem] (+)= A[a_tmem] * B[bdesc], A read from tensor memory (row r
// of an M = 128 operand in lane r, K element k of the instruction in column
// a_tmem + k, one 32-bit tf32 value per column).
__device__ __forceinline__ void tc_mma_tf32_ta(unsigned dtmem, unsigned atmem, uint64_t bdesc, uint32_t idesc,
                                               bool accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(dtmem),
        "r"(atmem), "l"(bdesc), "r"(idesc), "r"((unsigned)accumulate)
        : "memory");
}

// Whole warp: lane t writes 8 consecutive 32-bit columns of TMEM lane
// (lane base of taddr + t); the lane base is the warp's own quarter.
__device__ __forceinline__ void tc_st8(unsigned taddr, const uint32_t (&r)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
                 "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                 : "memory");
}

// Whole warp: this thread's tcgen05.st writes have completed.
__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// One thread: arrive once on `bar` when all tcgen05 operations it issued so far
// have completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Whole warp: 32 lanes (this warp's quarter of TMEM) x 32 consecutive columns,
// lane t receives row (lane base + t).
__device__ __forceinline__ void tc_ld32(unsigned taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tc_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

}  // namespace demag
