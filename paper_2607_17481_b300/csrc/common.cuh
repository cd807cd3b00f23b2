// Shared device helpers of the Panache CUDA path (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Opts a kernel in to dynamic shared memory up to the device's per-block
// limit (less the kernel's static shared memory), and checks that `need`
// fits.  The value set is the same for every call, so host threads that
// launch the same kernel concurrently with different sizes never see
// another thread's smaller setting.
template <class K>
inline cudaError_t pn_allow_smem(K kernel, size_t need) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(kernel));
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((long long)need > (long long)lim) return cudaErrorInvalidValue;
    if (fa.maxDynamicSharedSizeBytes == lim) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
}

#define PN_WARP 32
#define PN_FEAT 32            // floats per feature row: 2(K-1) <= 30 used, padded to 32 (128 B)
#define PN_MAXB 24            // signature bits
#define PN_MAXK 16            // spectral width K (bins 1..K-1 kept)

// ---------------------------------------------------------------------------
// Profile cells.  A cell (m, i) holds one 64-bit key: the non-negative
// distance's IEEE-754 double bit pattern with its low PN_IDX_BITS bits
// replaced by the partner's start index.  For non-negative doubles the bit
// pattern is monotone in the value, so an unsigned atomicMin keeps the
// smallest distance and, among equal (truncated) distances, the lowest
// partner index -- the tie rule of the exact profile (Sec. 2).  The stored
// distance is the true one truncated to 64 - PN_IDX_BITS bits (relative
// resolution 2^-26); reported distances are recomputed in FP64.
// ---------------------------------------------------------------------------
#define PN_IDX_BITS 26
#define PN_IDX_MASK ((1ull << PN_IDX_BITS) - 1ull)
#define PN_EMPTY_KEY 0xFFFFFFFFFFFFFFFFull
#define PN_MAX_SERIES_LEN ((int64_t)PN_IDX_MASK)   // partner index 2^26-1 is reserved

__host__ __device__ __forceinline__ uint64_t pn_pack(double d, uint32_t idx) {
#ifdef __CUDA_ARCH__
    uint64_t b = (uint64_t)__double_as_longlong(d);
#else
    uint64_t b;
    __builtin_memcpy(&b, &d, 8);
#endif
    return (b & ~PN_IDX_MASK) | (uint64_t)idx;
}

__host__ __device__ __forceinline__ double pn_key_dist(uint64_t key) {
    uint64_t b = key & ~PN_IDX_MASK;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    __builtin_memcpy(&d, &b, 8);
    return d;
#endif
}

__host__ __device__ __forceinline__ uint32_t pn_key_idx(uint64_t key) { return (uint32_t)(key & PN_IDX_MASK); }

// Key of a non-negative float distance, built with integer operations only:
// the float's 23 mantissa bits land above the 26-bit index field, so the
// result equals pn_pack((double)d, idx) exactly.
__device__ __forceinline__ uint64_t pn_pack_f(float d, uint32_t idx) {
    const uint32_t fb = __float_as_uint(d);
    const uint32_t e = fb >> 23;
    uint64_t db;
    if (e == 0) db = 0ull;                                  // zero (subnormals flush to zero)
    else if (e >= 0xFF) db = 0x7FF0000000000000ull;         // +inf
    else db = ((uint64_t)(e - 127 + 1023) << 52) | ((uint64_t)(fb & 0x7FFFFFu) << 29);
    return (db & ~PN_IDX_MASK) | (uint64_t)idx;
}

// Distance of a key as a float, truncated toward zero (integer operations
// only); an empty cell reads as +inf.
__device__ __forceinline__ float pn_key_distf(uint64_t key) {
    if (key == PN_EMPTY_KEY) return __int_as_float(0x7f800000);
    const uint32_t e = (uint32_t)(key >> 52) & 0x7FFu;
    const int ef = (int)e - 1023 + 127;
    if (e == 0 || ef <= 0) return 0.0f;
    if (ef >= 0xFF) return __int_as_float(0x7f800000);
    return __uint_as_float(((uint32_t)ef << 23) | ((uint32_t)(key >> 29) & 0x7FFFFFu));
}

__device__ __forceinline__ float pn_warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double pn_warp_sumd(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Orderable unsigned image of a float (ascending float order -> ascending uint order).
__device__ __forceinline__ uint32_t pn_float_order(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Number of retained non-DC bins at length m: K' = min(K-1, ceil(m/2)-1) (Sec. 3.2).
__host__ __device__ __forceinline__ int pn_kprime(int m, int K) {
    int c = (m + 1) / 2 - 1;
    int k = K - 1 < c ? K - 1 : c;
    return k < 0 ? 0 : k;
}

// Global depth after P insertions: smallest d >= 0 with P <= alpha 2^d, capped at B (Sec. 3.4).
// Device form: d = ceil(log2(ceil(P / alpha))) by a leading-zero count.
__device__ __forceinline__ int pn_depth_dev(uint32_t P, uint32_t alpha, int B) {
    if (P <= alpha) return 0;
    const uint32_t u = (P + alpha - 1u) / alpha;
    const int d = 32 - __clz(u - 1u);
    return d < B ? d : B;
}

__host__ __device__ __forceinline__ int pn_depth(int64_t P, int alpha, int B) {
    int d = 0;
    while (d < B && P > ((int64_t)alpha << d)) ++d;
    return d;
}
