// Exact z-normalised distance of one pair, computed by a whole warp
// (Sec. 2: d_m(i,j) = || Z_i - Z_j ||, Z = (T - mu) / sigma).
#pragma once
#include "kernels.cuh"

struct PnWin {
    double mu;     // window mean
    double inv;    // 1 / sigma (0 for a degenerate window)
    float mu_hi, mu_lo;
    float invf;
};

__device__ __forceinline__ PnWin pn_window(const PnView &v, int s, int64_t i, int m) {
    PnWin w;
    double var;
    pn_moments(v, s, i, m, w.mu, var);
    w.inv = var > 0.0 ? 1.0 / sqrt(var) : 0.0;
    w.mu_hi = (float)w.mu;
    w.mu_lo = (float)(w.mu - (double)w.mu_hi);
    w.invf = (float)w.inv;
    return w;
}

// Warp-cooperative distance.  Plain form: FP64 throughout.  Mixed form: the
// samples are (hi, lo) float pairs and the centring is done in float-float,
// (x_hi - mu_hi) + (x_lo - mu_lo), before the FP32 scaling and sum; the root
// of the FP32 sum is taken in FP32 too (a float distance, as the streaming
// search packs it), since a warp-wide FP64 root costs the FP64 pipe far more.
// Returns +inf when either window is degenerate (sigma = 0).
__device__ __forceinline__ double pn_dist_warp(const PnView &v, int64_t x_off, int m, int64_t i, const PnWin &wi,
                                               int64_t j, const PnWin &wj, int lane) {
    if (wi.inv == 0.0 || wj.inv == 0.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (v.precision == 0) {
        const double *xi = v.x + x_off + i;
        const double *xj = v.x + x_off + j;
        double acc = 0.0;
        for (int r = lane; r < m; r += 32) {
            double dz = (xi[r] - wi.mu) * wi.inv - (xj[r] - wj.mu) * wj.inv;
            acc = fma(dz, dz, acc);
        }
        return sqrt(pn_warp_sumd(acc));
    } else {
        const float2 *xi = v.xs + x_off + i;
        const float2 *xj = v.xs + x_off + j;
        float acc = 0.0f;
        for (int r = lane; r < m; r += 32) {
            float2 a = xi[r], b = xj[r];
            float za = ((a.x - wi.mu_hi) + (a.y - wi.mu_lo)) * wi.invf;
            float zb = ((b.x - wj.mu_hi) + (b.y - wj.mu_lo)) * wj.invf;
            float dz = za - zb;
            acc = fmaf(dz, dz, acc);
        }
        return (double)sqrtf(pn_warp_sum(acc));
    }
}

__device__ __forceinline__ double pn_cell_dist(unsigned long long key) {
    return key == PN_EMPTY_KEY ? __longlong_as_double(0x7ff0000000000000ll) : pn_key_dist(key);
}
