// Arithmetic policies of the exact-distance and bound tests on anchor windows.
//
// Mixed form (ZMix2 / ZMix1): z = fma(x, 1/sigma, -mu/sigma) in FP32 (one
// rounding: no cancellation when |mu| >> sigma; the rounding of -mu/sigma is a
// per-window constant whose effect on the distance cancels to first order),
// FP32 sums, thresholds compared as floats.  ZMix1 reads one float per sample
// (series given as float32); ZMix2 reads (hi, lo) pairs (float64 series).
// Plain form (ZPlain): the same in FP64.
//
// Q is the type of one staged query sample: the mixed forms stage (z, z) so
// that one shared-memory load feeds both halves of a packed two-wide FP32
// operation (eval_batch); the plain form stages z.
#pragma once
#include "distance.cuh"

struct ZMix2 {
    using T = float;
    using M = float2;   // (1/sigma, -mu/sigma)
    using X = float2;
    using Q = float2;   // staged query sample (z, z)
    __device__ static Q stage(float z) { return make_float2(z, z); }
    __device__ static float qval(const Q &s) { return s.x; }
    __device__ static M load(const PnView &v, int64_t w) { return v.wmf[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.xs + t; }
    __device__ static float z(const M &m, const X &x) { return fmaf(x.x, m.x, fmaf(x.y, m.x, m.y)); }
    __device__ static bool degenerate(const M &m) { return m.x == 0.0f; }
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
    __device__ static float z(const M &m, const X &x) { return fmaf(x, m.x, m.y); }
    // -z of two windows at once from (-1/sigma, mu/sigma) pairs ns, no: the
    // rounding of z, negated exactly
    __device__ static float2 nz2(X xa, X xb, float2 ns, float2 no) {
        return __ffma2_rn(make_float2(xa, xb), ns, no);
    }
};

struct ZPlain {
    using T = double;
    using M = double2;  // (1/sigma, -mu/sigma)
    using X = double;
    using Q = double;
    __device__ static Q stage(double z) { return z; }
    __device__ static double qval(const Q &s) { return s; }
    __device__ static M load(const PnView &v, int64_t w) { return v.wmd[w]; }
    __device__ static const X *samples(const PnView &v, int64_t t) { return v.x + t; }
    __device__ static double z(const M &m, const X &x) { return fma(x, m.x, m.y); }
    __device__ static bool degenerate(const M &m) { return m.x == 0.0; }
    __device__ static double finish(double acc) { return sqrt(pn_warp_sumd(acc)); }
    __device__ static double root(double s) { return sqrt(s); }
    __device__ static double cell(unsigned long long key) { return pn_cell_dist(key); }
    __device__ static unsigned long long pack(double d, uint32_t idx) { return pn_pack(d, idx); }
    __device__ static double fmn(double a, double b) { return fmin(a, b); }
    __device__ static double fmx(double a, double b) { return fmax(a, b); }
};
