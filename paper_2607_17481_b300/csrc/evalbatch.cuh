// Exact-distance evaluation of bound survivors against one staged window,
// shared by the streaming search and the hot-class sieve.
#pragma once
#include <type_traits>

#include "zops.cuh"

namespace pn {

// Exact distances of up to four queued survivors at once (warp-cooperative
// over samples, four independent accumulators), then the packed-key updates:
// the query's running best in registers, the candidate's cell by atomicMin
// only when the new key is below the snapshot read for the bound test (cells
// only decrease, so a key at or above the snapshot cannot change the cell).
template <class Z>
__device__ __forceinline__ void eval_batch(const PnView &v, const typename Z::Q *zq, const uint32_t *sc,
                                           const unsigned long long *sk, int nb, int64_t x_off, int64_t win_off,
                                           int a, uint32_t q, unsigned long long *prow,
                                           unsigned long long &bestkey, int lane) {
    using ZT = typename Z::T;
    const uint32_t c0 = sc[0], c1 = sc[nb > 1 ? 1 : 0], c2 = sc[nb > 2 ? 2 : 0], c3 = sc[nb > 3 ? 3 : 0];
    const auto m0 = Z::load(v, win_off + c0), m1 = Z::load(v, win_off + c1);
    const auto m2 = Z::load(v, win_off + c2), m3 = Z::load(v, win_off + c3);
    const auto *x0 = Z::samples(v, x_off + c0), *x1 = Z::samples(v, x_off + c1);
    const auto *x2 = Z::samples(v, x_off + c2), *x3 = Z::samples(v, x_off + c3);
    ZT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if constexpr (std::is_same<typename Z::X, float>::value) {
        // Float32 series: packed two-wide FP32, survivors (0, 1) and (2, 3)
        // side by side, the staged sample (z, z) one 8-byte load.
        // fma(x, -1/sigma, mu/sigma) is exactly -z, so zr + (-z) is exactly
        // zr - z: the sums are the scalar loop's bit for bit, at half the FP32
        // instructions.  (Float64 series keep the scalar loop: their (hi, lo)
        // samples need more registers than the packed form leaves.)
        const float2 ns01 = make_float2(-m0.x, -m1.x), no01 = make_float2(-m0.y, -m1.y);
        const float2 ns23 = make_float2(-m2.x, -m3.x), no23 = make_float2(-m2.y, -m3.y);
        float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
        if (nb > 2) {
#pragma unroll 2
            for (int r = lane; r < a; r += 32) {
                const float2 zz = zq[r];
                const float2 d01 = __fadd2_rn(zz, Z::nz2(x0[r], x1[r], ns01, no01));
                const float2 d23 = __fadd2_rn(zz, Z::nz2(x2[r], x3[r], ns23, no23));
                s01 = __ffma2_rn(d01, d01, s01);
                s23 = __ffma2_rn(d23, d23, s23);
            }
        } else {   // a trailing batch of one or two: the second pair is not evaluated
#pragma unroll 2
            for (int r = lane; r < a; r += 32) {
                const float2 d01 = __fadd2_rn(zq[r], Z::nz2(x0[r], x1[r], ns01, no01));
                s01 = __ffma2_rn(d01, d01, s01);
            }
        }
        a0 = s01.x;
        a1 = s01.y;
        a2 = s23.x;
        a3 = s23.y;
    } else {
        // two iterations in flight: eight independent sample loads per lane
#pragma unroll 2
        for (int r = lane; r < a; r += 32) {
            const ZT zr = Z::qval(zq[r]);
            const ZT d0 = zr - Z::z(m0, x0[r]);
            const ZT d1 = zr - Z::z(m1, x1[r]);
            const ZT d2 = zr - Z::z(m2, x2[r]);
            const ZT d3 = zr - Z::z(m3, x3[r]);
            a0 = fma(d0, d0, a0);
            a1 = fma(d1, d1, a1);
            a2 = fma(d2, d2, a2);
            a3 = fma(d3, d3, a3);
        }
    }
    // transposed reduction of the four sums (6 shuffles): afterwards lanes
    // 8v..8v+7 hold the total of survivor v
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    ZT k0 = hi16 ? a2 : a0, k1 = hi16 ? a3 : a1;
    const ZT s0 = hi16 ? a0 : a2, s1 = hi16 ? a1 : a3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    ZT t = hi8 ? k1 : k0;
    const ZT u = hi8 ? k0 : k1;
    t += __shfl_xor_sync(0xffffffffu, u, 8);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    const int vi = lane >> 3;
    const uint32_t cv = vi == 0 ? c0 : (vi == 1 ? c1 : (vi == 2 ? c2 : c3));
    const bool dg = Z::degenerate(vi == 0 ? m0 : (vi == 1 ? m1 : (vi == 2 ? m2 : m3)));
    const bool ok = vi < nb && !dg;
    const ZT dd = Z::root(t);
    unsigned long long kq = ok ? Z::pack(dd, cv) : PN_EMPTY_KEY;
    if (ok && (lane & 7) == 0) {
        const unsigned long long kc = Z::pack(dd, q);
        if (kc < sk[vi]) atomicMin(&prow[cv], kc);
    }
    unsigned long long o = __shfl_xor_sync(0xffffffffu, kq, 8);
    kq = o < kq ? o : kq;
    o = __shfl_xor_sync(0xffffffffu, kq, 16);
    kq = o < kq ? o : kq;
    if (kq < bestkey) bestkey = kq;
}

// The same evaluation split in two, for callers that queue many survivors:
// eval_sums leaves the sums of squared differences of up to four survivors
// (moments read from the caller's queue instead of global memory), and
// eval_finish roots, packs and applies them for a run of survivors at once,
// one survivor per lane.  Per-lane order and reduction tree are eval_batch's,
// so the distances are the same bit for bit; only the per-batch epilogue
// (root, two packs, compare, atomic, two 64-bit shuffles) is paid once per
// 32 survivors instead of once per four.
template <class Z>
__device__ __forceinline__ void eval_sums(const typename Z::Q *zq, const typename Z::X *xb, const uint32_t *sc,
                                          const typename Z::M *sm, int nb, int a, typename Z::T *ssum, int lane) {
    using ZT = typename Z::T;
    const uint32_t c0 = sc[0], c1 = sc[nb > 1 ? 1 : 0], c2 = sc[nb > 2 ? 2 : 0], c3 = sc[nb > 3 ? 3 : 0];
    const auto m0 = sm[0], m1 = sm[nb > 1 ? 1 : 0], m2 = sm[nb > 2 ? 2 : 0], m3 = sm[nb > 3 ? 3 : 0];
    const auto *x0 = xb + c0, *x1 = xb + c1, *x2 = xb + c2, *x3 = xb + c3;
    ZT a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if constexpr (std::is_same<typename Z::X, float>::value) {
        const float2 ns01 = make_float2(-m0.x, -m1.x), no01 = make_float2(-m0.y, -m1.y);
        const float2 ns23 = make_float2(-m2.x, -m3.x), no23 = make_float2(-m2.y, -m3.y);
        float2 s01 = make_float2(0.0f, 0.0f), s23 = make_float2(0.0f, 0.0f);
        if (nb > 2) {
#pragma unroll 2
            for (int r = lane; r < a; r += 32) {
                const float2 zz = zq[r];
                const float2 d01 = __fadd2_rn(zz, Z::nz2(x0[r], x1[r], ns01, no01));
                const float2 d23 = __fadd2_rn(zz, Z::nz2(x2[r], x3[r], ns23, no23));
                s01 = __ffma2_rn(d01, d01, s01);
                s23 = __ffma2_rn(d23, d23, s23);
            }
        } else {
#pragma unroll 2
            for (int r = lane; r < a; r += 32) {
                const float2 d01 = __fadd2_rn(zq[r], Z::nz2(x0[r], x1[r], ns01, no01));
                s01 = __ffma2_rn(d01, d01, s01);
            }
        }
        a0 = s01.x;
        a1 = s01.y;
        a2 = s23.x;
        a3 = s23.y;
    } else {
#pragma unroll 2
        for (int r = lane; r < a; r += 32) {
            const ZT zr = Z::qval(zq[r]);
            const ZT d0 = zr - Z::z(m0, x0[r]);
            const ZT d1 = zr - Z::z(m1, x1[r]);
            const ZT d2 = zr - Z::z(m2, x2[r]);
            const ZT d3 = zr - Z::z(m3, x3[r]);
            a0 = fma(d0, d0, a0);
            a1 = fma(d1, d1, a1);
            a2 = fma(d2, d2, a2);
            a3 = fma(d3, d3, a3);
        }
    }
    const bool hi16 = (lane & 16) != 0, hi8 = (lane & 8) != 0;
    ZT k0 = hi16 ? a2 : a0, k1 = hi16 ? a3 : a1;
    const ZT s0 = hi16 ? a0 : a2, s1 = hi16 ? a1 : a3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    ZT t = hi8 ? k1 : k0;
    const ZT u = hi8 ? k0 : k1;
    t += __shfl_xor_sync(0xffffffffu, u, 8);
    t += __shfl_xor_sync(0xffffffffu, t, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    const int vi = lane >> 3;
    if ((lane & 7) == 0 && vi < nb) ssum[vi] = t;
}

// Roots, packs and applies queued sums [f0, f1): the candidate's cell by
// atomicMin below its snapshot, the query's running best in registers.
template <class Z>
__device__ __forceinline__ void eval_finish(const typename Z::T *ssum, const uint32_t *sc,
                                            const unsigned long long *sk, const typename Z::M *sm, int f0, int f1,
                                            uint32_t q, unsigned long long *prow, unsigned long long &bestkey,
                                            int lane) {
    for (int t0 = f0; t0 < f1; t0 += 32) {
        const int t = t0 + lane;
        unsigned long long kq = PN_EMPTY_KEY;
        if (t < f1 && !Z::degenerate(sm[t])) {
            const auto dd = Z::root(ssum[t]);
            const uint32_t c = sc[t];
            kq = Z::pack(dd, c);
            const unsigned long long kc = Z::pack(dd, q);
            if (kc < sk[t]) atomicMin(&prow[c], kc);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ok = __shfl_xor_sync(0xffffffffu, kq, o);
            kq = ok < kq ? ok : kq;
        }
        if (kq < bestkey) bestkey = kq;
    }
}

// Exact distance of one candidate (warp-cooperative), same updates as eval_batch.
template <class Z>
__device__ __forceinline__ void eval_one(const PnView &v, const typename Z::Q *zq, uint32_t c,
                                         unsigned long long snapkey, int64_t x_off, int64_t win_off, int a,
                                         uint32_t q, unsigned long long *prow, unsigned long long &bestkey,
                                         int lane) {
    using ZT = typename Z::T;
    const auto m = Z::load(v, win_off + c);
    if (Z::degenerate(m)) return;
    const auto *x = Z::samples(v, x_off + c);
    ZT acc = 0;
    for (int r = lane; r < a; r += 32) {
        const ZT dz = Z::qval(zq[r]) - Z::z(m, x[r]);
        acc = fma(dz, dz, acc);
    }
    const ZT dd = Z::finish(acc);
    const unsigned long long kq = Z::pack(dd, c);
    if (kq < bestkey) bestkey = kq;
    if (lane == 0) {
        const unsigned long long kc = Z::pack(dd, q);
        if (kc < snapkey) atomicMin(&prow[c], kc);
    }
}

}  // namespace pn
