// Kernel-side view of one request and the launch wrappers of every step.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "ktimer.h"
#include "plan.h"

// Everything a kernel needs to know about a request, passed by value.
struct PnView {
    // tables
    const PnSeries *series;
    const PnAnchor *anchors;
    const PnLevel *levels;
    int32_t nseries, nanchors, nlevels;
    int32_t B;            // signature bits
    int32_t K;            // spectral width
    int32_t C;            // chunk length of the feature kernel (slides per direct-DFT anchor), a power of two
    int32_t cshift;       // log2(C)
    int32_t alpha;        // occupancy target
    int32_t R;            // verification budget gamma * alpha
    int32_t d0;           // probe reference depth
    int32_t probe_cap;    // implementation cap on Hamming-1 probes
    int32_t beta;         // batch length (samples) of the streaming schedule
    float lam;            // bound shrink lambda
    int32_t precision;    // 0 plain FP64, 1 mixed
    // samples
    const double *x;      // samples widened to FP64, concatenated over series
    const float2 *xs;     // samples as (hi, lo) float pairs: hi + lo == x to ~2^-48
    const float *x1;      // samples as floats (null unless every series was given as float32)
    const double2 *sq;    // per series n+1 prefix sums (sum, sum of squares) of x - shift
    const double *shift;  // per series shift subtracted before the prefix sums
    const int32_t *runlen;// equal-value run length from each sample, capped at the series' m_max
    // per-window arrays (indexed by anchor.win_off + q)
    float *F;             // feature rows, anchor.row_off + row(q), PN_FEAT floats each (null with Fh)
    __half *Fh;           // the same rows rounded to half precision (PANACHE_FLAG_HALF_FEATURES), else null
    float *sproj;         // per window, its projection on the sieve direction g_{a,B+1}, from the
                          // FP32 row (before rounding, with Fh): the sieve's sort key
    float lb_eps;         // relative precision of Fh against the FP32 rows (2^-11), 0 without Fh
    uint32_t *sig;        // B-bit SimHash keys
    uint32_t *cnt;        // inclusive count of non-constant windows with start <= q
    uint32_t *nclist;     // start of the r-th non-constant window
    float2 *wmf;          // mixed form: per-window (1/sigma, -mu/sigma) as floats; 1/sigma = 0 if degenerate
    double2 *wmd;         // plain form: per-window (1/sigma, -mu/sigma)
    uint32_t *qorder;     // search order of the flat query space (grouped by probe bucket)
    const float *g;       // projections [nanchors][B+1][PN_FEAT]
    const float *gT;      // the same, transposed per anchor: [nanchors][PN_FEAT][32] (projection l in lane l)
    float *anc;           // mixed form: tensor-core chunk anchors, [flat chunk][PN_FEAT] (null: FP64 direct DFT)
    const float *twb;     // with anc: the contraction's twiddle operand per anchor, [anchor][32][twb_ld]
    int32_t twb_ld;       // row length of twb (>= every anchor length)
    int32_t tc_fault;     // test hook: the anchor kernel issues no MMA and its waits give up quickly
    int *err;             // device error word (PN_ERR_*), 0 when every bounded wait succeeded
    // directory
    uint32_t *dir_keys;   // global bucket id of every item (sorted)
    uint32_t *dir_vals;   // window start of every item (sorted by (bucket, start))
    uint32_t *bstart;     // first sorted item of every global bucket (+1 sentinel)
    // profile rows, PN_EMPTY_KEY when unset
    unsigned long long *prof;
    // counters (device)
    unsigned long long *stats;
    // per-kernel event timer of the request (host object; null unless timing)
    PnKTimer *kt;
    // device-driven rounds of the emit stage: the kernels of a completion
    // round or refinement pass return at once when *gate is 0 (null: run)
    const int *gate;
};

// True when the current device-driven round has been closed.
__device__ __forceinline__ bool pn_gated(const PnView &v) { return v.gate && *(volatile const int *)v.gate == 0; }

#define PN_FT_CHUNKS 4         // chunks (one warp each) per block of the feature kernel
#define PN_ERR_TC_TIMEOUT 1   // a tensor-core anchor tile's bounded wait ran out
// Samples allocated (zero) past the last series in the FP32 sample buffers:
// the top-k sieve's staging reads whole 64-sample steps of a window without
// per-sample bounds and masks the samples past the window's end.
#define PN_SAMPLE_PAD 256

enum PnStat {
    PN_ST_QUERIES = 0,
    PN_ST_CANDIDATES,
    PN_ST_LB_PASSED,
    PN_ST_EXACT_SIEVE,
    PN_ST_EXACT_COMPLETION,
    PN_ST_HOT_CLASSES,
    PN_ST_IMPROVED,
    PN_ST_EXACT_REFINE,
    PN_ST_COUNT
};

// Window row inside an anchor's feature block: windows are interleaved by
// chunk, row(q) = (q mod C) * nchunk + q / C, so that the chunks advanced in
// lock-step by one warp write one contiguous run of rows.
__host__ __device__ __forceinline__ int64_t pn_row(int64_t q, int32_t C, int64_t nchunk) {
    return (q % C) * nchunk + q / C;
}

// The same row with C = 2^cshift and 32-bit window indices (kernels' hot loops).
__device__ __forceinline__ uint32_t pn_row32(uint32_t q, int cshift, uint32_t nchunk) {
    return (q & ((1u << cshift) - 1u)) * nchunk + (q >> cshift);
}

// Feature rows in either storage precision: the row block of an anchor
// (anchor.row_off), then row r of it widened to float, as components
// 4j..4j+3 (16 B of FP32 row or 8 B of half row) or as component t alone.
template <bool HALF>
__device__ __forceinline__ const void *pn_rows(const PnView &v, int64_t row_off) {
    if constexpr (HALF) return v.Fh + row_off * PN_FEAT;
    else return v.F + row_off * PN_FEAT;
}

template <bool HALF>
__device__ __forceinline__ float4 pn_row_quad(const void *rows, uint32_t r, int j) {
    if constexpr (HALF) {
        const uint2 u = reinterpret_cast<const uint2 *>(static_cast<const __half *>(rows) + (size_t)r * PN_FEAT)[j];
        const float2 lo = __half22float2(*reinterpret_cast<const __half2 *>(&u.x));
        const float2 hi = __half22float2(*reinterpret_cast<const __half2 *>(&u.y));
        return make_float4(lo.x, lo.y, hi.x, hi.y);
    } else {
        return reinterpret_cast<const float4 *>(static_cast<const float *>(rows) + (size_t)r * PN_FEAT)[j];
    }
}

template <bool HALF>
__device__ __forceinline__ float pn_row_elem(const void *rows, uint32_t r, int t) {
    if constexpr (HALF) return __half2float(static_cast<const __half *>(rows)[(size_t)r * PN_FEAT + t]);
    else return static_cast<const float *>(rows)[(size_t)r * PN_FEAT + t];
}

// Additive margin on a bound read from rows rounded, at relative precision
// eps, from the FP32 rows.  The proof of Lemma 5 bounds the absolute inflation
// of the computed bound by 4 sqrt(m) eps, using S = || |a| + |b| || <= sqrt(2) m
// (the stored bins of a z-normalised window hold at most m^2 / 2 of energy,
// Parseval).  The feature gap itself moves by at most eps S (each rounded
// difference is off by at most eps (|a_k| + |b_k|); triangle inequality), so
// the constant holds with a factor 2 to spare, which also covers the FP32
// rows' own rounding of that energy.  Subnormal halves add at most 2^-24 per
// component difference: sqrt(2n/m) 2^-24 in bound units.  A bound that minus
// this margin still clears a threshold is one the FP32 rows' bound clears.
__device__ __forceinline__ float pn_row_margin(float eps, int m) {
    if (eps <= 0.0f) return 0.0f;
    return 4.0f * sqrtf((float)m) * eps + sqrtf(2.0f * (float)PN_FEAT / (float)m) * 5.9604645e-8f;
}

// <g_l, F> in a fixed order of fused multiply-adds; the feature kernel and
// the query kernel both call this, so their margins agree bit for bit.
__device__ __forceinline__ float pn_margin(const float *g, const float *f, int dims) {
    float acc = 0.0f;
    for (int t = 0; t < dims; ++t) acc = fmaf(g[t], f[t], acc);
    return acc;
}

// Directory population seen by query window q of anchor A (Sec. 3.5,
// Algorithm 1): samples arrive in batches of beta (beta = excl unless a
// smaller batch is configured), every window a batch completes is inserted
// before that batch's searches, so q sees the non-constant windows whose last
// sample lies at or before the end of the batch holding its own last sample
// q + a - 1 (the last batch ends at the series' end).  cnt is inclusive.
__device__ __forceinline__ uint32_t pn_query_population(const PnView &v, const PnAnchor &A, const PnSeries &S,
                                                        int64_t q) {
    const int beta = (v.beta > 0 && v.beta < S.excl) ? v.beta : S.excl;
    const int64_t tau = q + A.a - 1;
    const int64_t tend = min(S.n - 1, (tau / beta + 1) * beta - 1);
    const int64_t last = tend - A.a + 1;
    return v.cnt[A.win_off + last];
}

// Binary search: index of the last table entry whose `off` is <= key.
template <class T, class F>
__device__ __forceinline__ int pn_find(const T *tab, int count, int64_t key, F off) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off(tab[mid]) <= key) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Window moments from the FP64 prefix sums (Sec. 3.2: mu = S/m, sigma^2 = Q/m - mu^2),
// of the shifted samples; returns mu of the unshifted window.
__device__ __forceinline__ void pn_moments(const PnView &v, int s, int64_t i, int m, double &mu, double &var) {
    const PnSeries &se = v.series[s];
    const double2 *p = v.sq + se.x_off + s;
    double2 a = p[i], b = p[i + m];
    double ms = (b.x - a.x) / m;
    var = (b.y - a.y) / m - ms * ms;
    mu = ms + v.shift[s];
}

namespace pn {
cudaError_t launch_runlen(const PnView &v, int64_t total, cudaStream_t st);
cudaError_t launch_moments(const PnView &v, int64_t total, double2 *sq_out, cudaStream_t st);
size_t features_smem(int a_max, int B);
cudaError_t launch_moment_table(const PnView &v, int64_t total_windows, cudaStream_t st);
cudaError_t launch_features(const PnView &v, const int32_t *blk_anchor, const int32_t *blk_chunk0,
                            int32_t nblocks, int a_max, cudaStream_t st);
cudaError_t launch_ranks(const PnView &v, int64_t total_windows, cudaStream_t st);
cudaError_t launch_directory(const PnView &v, int64_t total_items, int64_t total_buckets, cudaStream_t st);
size_t anchor_tc_smem();
cudaError_t launch_twiddles(const PnAnchor *anc_dev, int32_t nanc, int32_t ld, float *tw, cudaStream_t st);
cudaError_t launch_anchor_tc(const PnView &v, const int32_t *tile_anchor, const int32_t *tile_row0, int32_t ntiles,
                             cudaStream_t st);
// The search order (v.qorder) by first-probed bucket.  With keys_out, the
// sorted bucket keys are handed to the caller (a stream-ordered allocation
// it frees) instead of being freed: the Gram search groups queries by them.
cudaError_t launch_query_order(const PnView &v, int64_t total_queries, int64_t total_buckets, cudaStream_t st,
                               const PnQRange *rng = nullptr, int32_t nrng = 0, uint32_t **keys_out = nullptr);
int search_max_budget();
// Spectral-width calibration statistics: out[0..14] energy means and
// out[15..29] collision-probability means for K = 2..16, out[30] pairs.
cudaError_t launch_calibration(const double *x, const PnCalWin *win, int nwin, const int *g_off, const int *g_cnt,
                               const int *row_g, const int *row_a, int nrows, int B, double *out, cudaStream_t st);
// The streaming search of every query; with `warm`, the warm-start pass
// (one exact distance per query, within its admitted candidates) runs first.
cudaError_t launch_search(const PnView &v, int64_t total_queries, int grid_blocks, int a_max, cudaStream_t st,
                          bool warm);
// Whether the opt-in tensor-core Gram search can serve this request (mixed
// form, anchors of at most 192 samples, budget R <= 128).
bool search_gram_supported(const PnView &v, int a_max);
// The same search (same admitted pairs, same profile rows) with the
// tensor-core Gram filter in place of the per-query Parseval test; `keys`
// are the sorted bucket keys of the query order.
cudaError_t launch_search_gram(const PnView &v, const uint32_t *keys, int64_t total_queries, int sm_count,
                               int a_max, cudaStream_t st);
// Population and depth every window of anchor `anchor` would probe with, by
// the search's own rule; -1 for windows that are not searched (constant, or
// no valid earlier window).
cudaError_t launch_query_levels(const PnView &v, int32_t anchor, int64_t nw, int32_t *population, int32_t *depth,
                                cudaStream_t st);
// The candidate list each listed query of anchor `anchor` is searched with,
// by the search's own rule (counts[i] = -1 for windows the search skips).
cudaError_t launch_query_candidates(const PnView &v, int32_t anchor, const int64_t *qs, int32_t nq, uint32_t *cand,
                                    int32_t cap, int32_t *counts, cudaStream_t st);
}  // namespace pn
