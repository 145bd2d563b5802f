// qw_tc.cuh -- fifth-generation tensor-core (tcgen05) helpers shared by the
// kernels that issue tcgen05.mma: shared-memory matrix descriptors for the
// no-swizzle K-major layout, instruction descriptors, the MMA, commit, fences,
// TMEM loads, and a bounded mbarrier wait.  All inline PTX.
//
// Layout of an operand tile in shared memory: 8-row x 16-byte core matrices,
// core matrix (i, j) (rows 8i..8i+7, 16-bit elements k 8j..8j+7) at byte
// (i * K / 8 + j) * 128 of the tile: core matrices adjacent in k are 128 bytes
// apart (the descriptor's leading-dimension offset) and adjacent in rows
// K * 16 bytes apart (its stride offset).
#pragma once

#include <cstdint>

namespace qw {

__device__ __forceinline__ uint32_t tc_smem(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: no swizzle, K-major; start, leading
// (k-direction) and stride (row-direction) byte offsets in 16-byte units;
// bits 46-47 hold the descriptor version of this architecture (1).
__device__ __forceinline__ uint64_t tc_desc(const void *start, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((tc_smem(start) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP16 A and B (K-major), FP32 D, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// The same with BF16 A and B (A and B formats, bits 7-9 and 10-12, = 1).
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N)
{
    return tc_idesc(M, N) | (1u << 7) | (1u << 10);
}

__device__ __forceinline__ void tc_mma(uint32_t dcol, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Bounded wait on an mbarrier phase (about 2 s); false when it gave up.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(tc_smem(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > 4000000000LL) return false;
    }
}

// Byte offset of element (r, k) in a no-swizzle K-major tile with K columns.
__device__ __forceinline__ uint32_t tc_off(int r, int k, int K)
{
    return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}


}  // namespace qw
