// z-normalised samples of anchor windows from the per-window moments table.
#pragma once
#include "kernels.cuh"

template <typename ZT>
struct ZOps;

// Mixed form: samples as (hi, lo) floats, centred in float-float, FP32 sums.
template <>
struct ZOps<float> {
    using M = float4;   // (mu_hi, mu_lo, 1/sigma, 0)
    using X = float2;
    __device__ static M load(const PnView &v, int64_t w) { return v.wmf[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.xs + t; }
    __device__ static float z(const M &m, const X &x) { return ((x.x - m.x) + (x.y - m.y)) * m.z; }
    __device__ static bool degenerate(const M &m) { return m.z == 0.0f; }
    __device__ static double finish(float acc) { return sqrt((double)pn_warp_sum(acc)); }
};

// Plain form: FP64 throughout.
template <>
struct ZOps<double> {
    using M = double2;  // (mu, 1/sigma)
    using X = double;
    __device__ static M load(const PnView &v, int64_t w) { return v.wmd[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.x + t; }
    __device__ static double z(const M &m, const X &x) { return (x - m.x) * m.y; }
    __device__ static bool degenerate(const M &m) { return m.y == 0.0; }
    __device__ static double finish(double acc) { return sqrt(pn_warp_sumd(acc)); }
};
