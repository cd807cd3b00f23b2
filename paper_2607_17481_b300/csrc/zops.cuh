// Arithmetic policies of the exact-distance and bound tests on anchor windows.
//
// Mixed form (ZMix2 / ZMix1): z = ((x_hi - mu_hi) + (x_lo - mu_lo)) / sigma in
// FP32 with FP32 sums, thresholds compared as floats.  ZMix1 reads one float
// per sample (series given as float32, whose low part is exactly zero);
// ZMix2 reads (hi, lo) pairs (float64 series).
// Plain form (ZPlain): FP64 throughout.
#pragma once
#include "distance.cuh"

struct ZMix2 {
    using T = float;
    using M = float4;   // (mu_hi, mu_lo, 1/sigma, 0)
    using X = float2;
    __device__ static M load(const PnView &v, int64_t w) { return v.wmf[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.xs + t; }
    __device__ static float z(const M &m, const X &x) { return ((x.x - m.x) + (x.y - m.y)) * m.z; }
    __device__ static bool degenerate(const M &m) { return m.z == 0.0f; }
    __device__ static float finish(float acc) { return sqrtf(pn_warp_sum(acc)); }
    __device__ static float root(float s) { return sqrtf(s); }
    __device__ static float cell(unsigned long long key) { return pn_key_distf(key); }
    __device__ static unsigned long long pack(float d, uint32_t idx) { return pn_pack_f(d, idx); }
    __device__ static float fmn(float a, float b) { return fminf(a, b); }
    __device__ static float fmx(float a, float b) { return fmaxf(a, b); }
};

struct ZMix1 : ZMix2 {
    using X = float;
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.x1 + t; }
    __device__ static float z(const M &m, const X &x) { return ((x - m.x) - m.y) * m.z; }
};

struct ZPlain {
    using T = double;
    using M = double2;  // (mu, 1/sigma)
    using X = double;
    __device__ static M load(const PnView &v, int64_t w) { return v.wmd[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.x + t; }
    __device__ static double z(const M &m, const X &x) { return (x - m.x) * m.y; }
    __device__ static bool degenerate(const M &m) { return m.y == 0.0; }
    __device__ static double finish(double acc) { return sqrt(pn_warp_sumd(acc)); }
    __device__ static double root(double s) { return sqrt(s); }
    __device__ static double cell(unsigned long long key) { return pn_cell_dist(key); }
    __device__ static unsigned long long pack(double d, uint32_t idx) { return pn_pack(d, idx); }
    __device__ static double fmn(double a, double b) { return fmin(a, b); }
    __device__ static double fmx(double a, double b) { return fmax(a, b); }
};
