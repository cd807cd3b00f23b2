// Throughput probes of the arithmetic pipes the path's kernels run on: FP32
// fused multiply-add (scalar and packed two-wide) and FP64 fused
// multiply-add.  They give the measured denominators of the per-kernel
// roofline fractions; the method does not use them.
//
// Every thread carries 8 independent FMA chains (enough to cover the FMA
// latency at the occupancy used), the grid fills every SM 8 blocks deep, and
// the result of every chain is stored so that no chain can be removed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "panache.h"

namespace {

constexpr int PK_THREADS = 256;
constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(PK_THREADS) k_fma32(int iters, float b, float c, float *out) {
    float a[PK_CHAINS];
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = (float)(threadIdx.x + u) * 1e-3f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int u = 0; u < PK_CHAINS; ++u) a[u] = fmaf(a[u], b, c);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) acc += a[u];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(PK_THREADS) k_fma32x2(int iters, float b, float c, float *out) {
    float2 a[PK_CHAINS];
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = make_float2((float)(threadIdx.x + u) * 1e-3f, (float)u * 1e-3f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int u = 0; u < PK_CHAINS; ++u) a[u] = __ffma2_rn(a[u], b2, c2);
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) acc += a[u].x + a[u].y;
    out[blockIdx.x * PK_THREADS + threadIdx.x] = acc;
}

__global__ void __launch_bounds__(PK_THREADS) k_fma64(int iters, double b, double c, float *out) {
    double a[PK_CHAINS];
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) a[u] = (double)(threadIdx.x + u) * 1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int u = 0; u < PK_CHAINS; ++u) a[u] = fma(a[u], b, c);
        }
    }
    double acc = 0.0;
#pragma unroll
    for (int u = 0; u < PK_CHAINS; ++u) acc += a[u];
    out[blockIdx.x * PK_THREADS + threadIdx.x] = (float)acc;
}

cudaError_t launch(int kind, int blocks, int iters, float *out, cudaStream_t st) {
    if (kind == 0) k_fma32<<<blocks, PK_THREADS, 0, st>>>(iters, 0.999999f, 1e-6f, out);
    else if (kind == 1) k_fma32x2<<<blocks, PK_THREADS, 0, st>>>(iters, 0.999999f, 1e-6f, out);
    else k_fma64<<<blocks, PK_THREADS, 0, st>>>(iters, 0.999999, 1e-6, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" int panache_alu_peak(int32_t kind, double *tflops) {
    if (!tflops || kind < 0 || kind > 2) return PANACHE_EINVAL;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PANACHE_ENODEV;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PANACHE_ENODEV;
    const int blocks = sms * 8;
    cudaStream_t st = nullptr;
    float *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PANACHE_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PANACHE_ECUDA;
    if (cudaMallocAsync((void **)&out, sizeof(float) * (size_t)blocks * PK_THREADS, st) != cudaSuccess) {
        cudaStreamDestroy(st);
        return PANACHE_ENOMEM;
    }
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = PANACHE_ECUDA;
    // a short run sizes the timed one to about 50 ms
    int iters = kind == 2 ? 8 : 256;
    float ms = 0.0f;
    for (int pass = 0; pass < 3 && rc == PANACHE_OK; ++pass) {
        if (launch(kind, blocks, iters, out, st) != cudaSuccess) rc = PANACHE_ECUDA;      // warm
        if (rc == PANACHE_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = PANACHE_ECUDA;
        if (rc == PANACHE_OK && launch(kind, blocks, iters, out, st) != cudaSuccess) rc = PANACHE_ECUDA;
        if (rc == PANACHE_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = PANACHE_ECUDA;
        if (rc == PANACHE_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = PANACHE_ECUDA;
        if (rc == PANACHE_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PANACHE_ECUDA;
        if (rc != PANACHE_OK || ms >= 40.0f || iters >= (1 << 24)) break;
        const double scale = 50.0 / (ms > 0.01f ? ms : 0.01f);
        iters = (int)(iters * (scale < 64.0 ? scale : 64.0)) + 1;
    }
    if (rc == PANACHE_OK) {
        const double fma_per_thread = (double)iters * 16 * PK_CHAINS * (kind == 1 ? 2 : 1);
        const double flop = 2.0 * fma_per_thread * (double)blocks * PK_THREADS;
        *tflops = flop / (ms * 1e-3) / 1e12;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return rc;
}
