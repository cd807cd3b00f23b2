// Work descriptors shared by the host runtime and the kernels.
//
// One request (a single series, or many series of a batch) is flattened into
// tables of series, anchors (one per (series, anchor length) pair) and
// directory levels.  Every kernel walks one of these flat index spaces, so a
// batch of thousands of series runs in the same launches as a single series.
#pragma once
#include <stdint.h>

struct PnSeries {
    int64_t x_off;        // first sample in the concatenated sample buffers
    int64_t n;            // samples
    int64_t row_off;      // first cell of this series' profile rows [L][ld]
    int64_t ld;           // profile row stride: n for a request, the resident capacity for a stream
    int32_t m_min, m_max; // length interval
    int32_t excl;         // exclusion zone: a pair is valid iff |i - j| >= excl
    int32_t k;            // motifs requested
    int32_t anchor_begin; // first anchor of the series in the anchor table
    int32_t anchor_count;
    int32_t mode;         // 0: global top-k, 1: top-k per length
    int32_t _pad;
};

struct PnAnchor {
    int32_t series;       // owning series
    int32_t a;            // anchor length
    int32_t kp;           // K' at this length
    int32_t dmax;         // deepest level allocated: depth(nw)
    int64_t nw;           // windows of length a: n - a + 1
    int64_t win_off;      // first window in the per-window arrays (keys, counts, lists)
    int64_t row_off;      // first feature row of this anchor (nchunk * C rows)
    int64_t nchunk;       // chunks of C windows: ceil(nw / C)
    int64_t chunk_off;    // first chunk of this anchor in the flat chunk space (tensor-core anchors)
    int64_t item_off;     // first directory item (all levels of this anchor)
    int64_t bucket_base;  // first global bucket id of level 0
    int32_t level_begin;  // first level in the level table
    int32_t nlevels;      // dmax + 1
};

// A run of queries [q_lo, q_lo + count) of one anchor, placed at `off` in a
// compact query space (the windows a stream append or snapshot searches).
struct PnQRange {
    int64_t off;
    int64_t q_lo;
    int32_t anchor;
    int32_t _pad;
};

// One sampled window of the spectral-width calibration.
struct PnCalWin {
    int64_t start;
    int32_t m;
    int32_t group;        // index of its length among the calibration lengths
};

struct PnLevel {
    int32_t anchor;       // owning anchor
    int32_t d;            // depth
    int64_t cap;          // min(nw, alpha 2^d): items allocated to this level
    int64_t item_off;     // first item of this level in the flat item space
    int64_t bucket_base;  // global bucket id of prefix 0 at this level
};
