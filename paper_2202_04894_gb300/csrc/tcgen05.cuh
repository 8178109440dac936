// Thin inline-PTX wrappers for the 5th-generation tensor cores (tcgen05, sm_100
// family): tensor-memory (TMEM) allocation, single-thread MMA issue with
// shared-memory operand descriptors, completion on an mbarrier, and TMEM loads.
// Only what the near-field kernel uses: kind::tf32, one CTA (cta_group::1),
// operands K-major without swizzle.
#pragma once

#include <cstdint>

namespace defmm {
namespace tc {

// Shared-memory matrix descriptor, no swizzle, K-major.  The matrix is stored
// as 8-row x 16-byte core matrices of 128 contiguous bytes (row i of a core
// matrix at +16 i); `lbo` is the byte distance between core matrices adjacent
// along K, `sbo` between core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // bits  0-13: start address >> 4
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;      // bits 16-29: leading byte offset >> 4
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;      // bits 32-45: stride byte offset >> 4
    d |= (uint64_t)1 << 46;                           // bits 46-47: descriptor version 1
    // bits 49-51 base offset 0, bit 52 absolute LBO mode off, bits 61-63 layout 0 (no swizzle)
    return d;
}

// Instruction descriptor of kind::tf32 with an f32 accumulator, A and B
// K-major, no negation or sparsity, shape M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4)                         // bits 4-5:   D format f32
         | (2u << 7)                         // bits 7-9:   A format tf32
         | (2u << 10)                        // bits 10-12: B format tf32
         | ((uint32_t)(N >> 3) << 17)        // bits 17-22: N / 8
         | ((uint32_t)(M >> 4) << 24);       // bits 24-28: M / 16
}

// Allocates ncols TMEM columns (a power of two >= 32); one full warp calls it.
// The TMEM address is written to *dst (shared memory).
__device__ __forceinline__ void alloc(uint32_t* dst, uint32_t ncols) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(a), "r"(ncols) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]; issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         bool accumulate) {
    const uint32_t acc = accumulate ? 1u : 0u;
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
        ::"r"(d_tmem), "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(acc) : "memory");
}

// The mbarrier at `bar` (shared) receives one arrival when every tcgen05
// operation issued so far by this thread has completed.
__device__ __forceinline__ void commit(uint64_t* bar) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(bar);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(a) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Generic-proxy shared-memory writes made visible to the tensor cores.
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive 32-bit columns of this warp's 32 TMEM lanes (lane = thread):
// taddr = (lane_base << 16) | column.  Waits for the load.
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Round to the nearest tf32 (10-bit mantissa), ties away from zero; the result
// is exactly representable, so x - to_tf32(x) is exact in float.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

}  // namespace tc
}  // namespace defmm
