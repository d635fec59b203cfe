// Inline-PTX wrappers for the Blackwell (sm_100 family) features the split
// history kernel uses: mbarriers with bounded waits, 1-D bulk async copies,
// and the tcgen05 tensor-memory / MMA instructions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fabm {
namespace ptx {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity to complete, for at most
// `budget` clock cycles.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > budget) return false;
    return true;
}

// 1-D bulk copy global -> shared, completing `bytes` of transaction count on bar.
// dst/src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ------------------------------------------------------------- tcgen05 ---

__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Instruction descriptor for kind::f16 with bf16 A and B (both K-major) and an
// fp32 accumulator, shape M x N.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// The six products of order <= 2 of three-term splits a = a0+a1+a2 and
// b = b0+b1+b2 for one K step: a0*b0 into d0 (accumulating unless `first`),
// a0*b1 (idem), a1*b0, a0*b2, a1*b1, a2*b0 into d12; for two weight operands
// (b*, c*) that share the f operand a, into two accumulator pairs (d0, d12)
// and (e0, e12), issued alternately in one statement (one predicate setup for
// twelve MMAs; the alternation measured ~5% faster than one kind after the
// other inside the solve).
__device__ __forceinline__ void mma_bf16_split6x2(uint32_t d0, uint32_t d12, uint32_t e0,
                                                  uint32_t e12, uint64_t a0, uint64_t a1,
                                                  uint64_t a2, uint64_t b0, uint64_t b1,
                                                  uint64_t b2, uint64_t c0, uint64_t c1,
                                                  uint64_t c2, uint32_t idesc, uint32_t first)
{
    asm volatile(
        "{\n .reg .pred pa, pt;\n"
        " setp.eq.b32 pa, %14, 0;\n"
        " setp.eq.b32 pt, %14, %14;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %4, %7, %13, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %8, %13, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%2], %4, %10, %13, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%3], %4, %11, %13, pa;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %5, %7, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%3], %5, %10, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %4, %9, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%3], %4, %12, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %5, %8, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%3], %5, %11, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%1], %6, %7, %13, pt;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%3], %6, %10, %13, pt;\n}\n" ::"r"(d0),
        "r"(d12), "r"(e0), "r"(e12), "l"(a0), "l"(a1), "l"(a2), "l"(b0), "l"(b1), "l"(b2),
        "l"(c0), "l"(c1), "l"(c2), "r"(idesc), "r"(first)
        : "memory");
}

// Shared-memory matrix descriptor of a no-swizzle K-major operand, as two
// 32-bit words: bits 0-13 start address / 16, bits 16-29 leading-dimension
// byte offset / 16, bits 32-45 stride-dimension byte offset / 16, bit 46 the
// descriptor version, swizzle bits 0.  The address field is the low 14 bits
// of `lo`, so adding o/16 to lo moves the operand by o bytes as long as the
// address stays below 256 KB.
__device__ __forceinline__ uint32_t smem_desc_lo(uint32_t addr, uint32_t lbo)
{
    return ((addr >> 4) & 0x3FFF) | (((lbo >> 4) & 0x3FFF) << 16);
}
__host__ __device__ constexpr uint32_t smem_desc_hi(uint32_t sbo)
{
    return ((sbo >> 4) & 0x3FFF) | (1u << 14);
}
__device__ __forceinline__ uint64_t desc_join(uint32_t lo, uint32_t hi)
{
    return ((uint64_t)hi << 32) | lo;
}

// Arrive on bar once every tcgen05 operation issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Issue two loads of 32 lanes x 8 consecutive 32-bit columns into r[0..7] and
// r[8..15].  The registers are written asynchronously: they must not be read
// (or copied) before tmem_wait16(r).
__device__ __forceinline__ void tmem_ld8x2_issue(uint32_t ta0, uint32_t ta1, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta0), "r"(ta1)
        : "memory");
}

// Wait for every tcgen05.ld this thread issued; r is passed through so that
// its uses are ordered after the wait.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]) : : "memory");
}

}  // namespace ptx
}  // namespace fabm
