// tcgen05 helpers shared by the tensor-core kernels (sm_103a): shared-memory
// matrix and instruction descriptors of the PTX ISA's documented bit
// layout, the K-major no-swizzle canonical operand layout (8-row x 16-byte
// core matrices) and the K-major 128-byte-swizzled one, TF32 rounding for
// the hi + lo operand split, and a bounded mbarrier wait.
#pragma once
#include <stdint.h>

namespace pn {

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// tcgen05 shared-memory matrix descriptor: start, leading (K-direction) and
// stride (M/N-direction) byte offsets of the core matrices, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: D F32, A and B TF32, both K-major, M x N.
__device__ __forceinline__ uint32_t umma_idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Element (row, k) of a K-major canonical layout with kg = KS/4 core matrices along K.
__device__ __forceinline__ int kmaj(int row, int k, int kg) {
    return ((row >> 3) * kg + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

__device__ __forceinline__ float tf32_hi(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Byte offset of element (row, k) in a K-major 128-byte-swizzled tile of
// `rows` rows (atoms of 64 16-bit values along K, rows x 128 bytes each).
__device__ __forceinline__ uint32_t sw128_off(int row, int k, int rows) {
    const int kk = k & 63;
    return (uint32_t)((k >> 6) * rows * 128 + row * 128 + ((((kk >> 3) ^ (row & 7))) << 4) + (kk & 7) * 2);
}

// tcgen05 shared-memory descriptor of a K-major 128-byte-swizzled operand:
// stride 1024 bytes between eight-row groups, layout type 2 (128B swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                          // leading offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;                // stride offset
    d |= (uint64_t)1 << 46;                          // descriptor version
    d |= (uint64_t)2 << 61;                          // 128-byte swizzle
    return d;
}

// Instruction descriptor: D F32, A and B f16, both K-major, M x N.
__device__ __forceinline__ uint32_t umma_idesc_f16(int M, int N) {
    return (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, int spin) {
    uint32_t done = 0;
    for (int it = 0; it < spin && !done; ++it) {
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
                     : "=r"(done)
                     : "r"(mbar), "r"(phase)
                     : "memory");
    }
    return done != 0;
}


}  // namespace pn
