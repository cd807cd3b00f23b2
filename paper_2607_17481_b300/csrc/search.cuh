// Budgeted candidate lists of the streaming search (Sec. 3.4): the device
// function both search kernels build each query's list with.
#pragma once
#include "kernels.cuh"

namespace pn {

constexpr int SR_WARM = 32;    // candidates a query's warm start inspects

// The budgeted candidate list of query window q (key index w) of anchor
// ai at global depth d (Sec. 3.4): the exact d-bit prefix bucket, then
// 1 + max(0, d - d0) Hamming-1 buckets (capped by d and the probe cap) in
// increasing |<g_{a,l}, F_q>| (ties to the lower bit), each bucket's valid
// entries (start <= q - excl) taken in full while the budget allows, else
// ceil(r/2) most recent and floor(r/2) evenly spaced.  The whole warp runs
// it; the query's row is left in frow, the list in cand, and its length is
// returned.  WARM: the warm start's list (the exact bucket's most recent
// entries only).
template <bool HALF, bool WARM>
__device__ __forceinline__ int sr_candidates(const PnView &v, int ai, const PnAnchor &A, const PnSeries &S, int64_t w,
                                             int64_t q, int d, int lane, float *frow, uint32_t *probe, uint32_t *cand,
                                             const void *Fa, uint32_t nch, int dims, int R) {
    const PnLevel &L = v.levels[A.level_begin + d];
    frow[lane] = pn_row_elem<HALF>(Fa, pn_row32((uint32_t)q, v.cshift, nch), lane);
    __syncwarp();
    float mg = __int_as_float(0x7f800000);
    if (!WARM && lane < d) {
        // <g_lane, F> in the FMA order of pn_margin, the projection read from
        // the transposed copy (one coalesced 128-byte row per dimension)
        const float *gt = v.gT + (int64_t)ai * PN_FEAT * 32 + lane;
        float acc = 0.0f;
#pragma unroll
        for (int t = 0; t < PN_FEAT - 2; ++t)
            if (t < dims) acc = fmaf(gt[t * 32], frow[t], acc);
        mg = fabsf(acc);
        if (!(mg <= 3.0e38f)) mg = 3.0e38f;            // non-finite input: still a bit below d
    }
    const uint32_t sgq = v.sig[w];
    const uint32_t pre = d > 0 ? (sgq >> (v.B - d)) : 0u;
    const int h = (WARM || d <= 0) ? 0 : min(d, min(v.probe_cap, 1 + max(0, d - v.d0)));
    // lane j (0 <= j <= h) owns probe j: the exact prefix, then Hamming-1
    // buckets in increasing margin (ties to the lower bit).  Each bit lane
    // ranks its margin among the d bits; the lane of rank r flips its bit
    // for probe r + 1, handed to lane r + 1 through shared memory.
    if (h > 0) {
        int rank = 0;
        for (int k = 0; k < d; ++k) {
            const float o = __shfl_sync(0xffffffffu, mg, k);
            rank += (o < mg || (o == mg && k < lane)) ? 1 : 0;
        }
        if (lane < d && rank < h) probe[rank + 1] = pre ^ (1u << (d - 1 - lane));
    }
    __syncwarp();
    const uint32_t my_probe = (lane >= 1 && lane <= h) ? probe[lane] : pre;
    // every probe's bucket range and valid prefix (start <= q - excl), in parallel
    const int64_t qmax = q - S.excl;
    uint32_t my_lo = 0, my_sz = 0;
    if (lane <= h) {
        const uint32_t gb = (uint32_t)(L.bucket_base + my_probe);
        const uint32_t lo = v.bstart[gb], hi = v.bstart[gb + 1];
        uint32_t l = lo, r = hi;                       // first entry with start > qmax
        while (l < r) {
            const uint32_t mid = (l + r) >> 1;
            if ((int64_t)v.dir_vals[mid] <= qmax) l = mid + 1; else r = mid;
        }
        my_lo = lo;
        my_sz = l - lo;
    }
    // budgeted candidate list, in probe order
    int taken = 0;
    if constexpr (WARM) {
        // the most recent valid entries of the exact bucket
        const uint32_t lo = __shfl_sync(0xffffffffu, my_lo, 0);
        const int sz = (int)__shfl_sync(0xffffffffu, my_sz, 0);
        taken = min(sz, SR_WARM);
        if (lane < taken) cand[lane] = v.dir_vals[lo + sz - taken + lane];
    }
    for (int j = 0; !WARM && j <= h && taken < R; ++j) {
        const uint32_t lo = __shfl_sync(0xffffffffu, my_lo, j);
        const int sz = (int)__shfl_sync(0xffffffffu, my_sz, j);
        const int rem = R - taken;
        const int cnt = min(sz, rem);
        // even-interval positions floor(t (sz - h1) / h2), with rest = sz - h1
        // split as rest = qh h2 + rh so only t rh (< 2^18) is divided
        const int h1 = (rem + 1) / 2, h2 = rem / 2, h2d = max(1, h2);
        const int rest = sz - h1;
        int qh = 0, rh = 0;
        if (sz > rem) {                                // warp-uniform: only an overflowing bucket divides
            qh = rest / h2d;
            rh = rest - qh * h2d;
        }
        for (int t = lane; t < cnt; t += 32) {
            int pos;
            if (sz <= rem) pos = t;
            else pos = t < h2 ? t * qh + (t * rh) / h2d : (rest + (t - h2));
            cand[taken + t] = v.dir_vals[lo + pos];
        }
        taken += cnt;
    }
    __syncwarp();
    return taken;
}

}  // namespace pn
