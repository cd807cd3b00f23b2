// Emit-stage records and launch wrappers (Sec. 3.6, Algorithm 2).
#pragma once
#include "kernels.cuh"

// Row of the t-th tile of an nb x nb upper triangle enumerated row by row
// (row bu holds nb - bu tiles): the largest bu with bu nb - bu (bu - 1) / 2
// <= t, by bisection.
__host__ __device__ __forceinline__ uint32_t tri_row(uint32_t t, uint32_t nb) {
    uint32_t lo = 0, hi = nb - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if ((uint64_t)mid * nb - ((uint64_t)mid * (mid - 1)) / 2 <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

struct PnClass {          // one hot class: a final-depth bucket larger than R
    int32_t anchor;
    uint32_t lo;          // first sorted directory item of the bucket
    uint32_t size;        // members
    uint32_t moff;        // first member in the flat member space
};

struct PnSeed {           // a completion seed: cell (m, i) of a series and its neighbour j
    int32_t series;
    int32_t m;
    int64_t i;
    int64_t j;
};

struct PnSelGroup {       // one top-k selection group
    int64_t cell_off;     // first profile cell of the group
    int64_t ncell;        // cells in the group
    int32_t series;
    int32_t k;            // motifs wanted
    uint32_t need;        // pool size that must be covered: k (m_max + 1)
    int32_t _pad;
};

struct PnPoolEntry {
    double d;             // in-stream distance, then the FP64 verified and zero-snapped one
    uint32_t cell;        // cell offset inside the group ((m - m_min) n + i for a series group)
    uint32_t j;           // neighbour
};

struct PnPick {           // one selected motif
    int32_t series;
    int32_t m;
    int64_t i;
    int64_t j;
    double d;
};

namespace pn {
// topk_thr (device, one threshold per anchor, or null): the top-k sieve;
// focus_anchors (device, one word per anchor, or null) restricts it to the
// hot classes of the anchors whose word is nonzero; *improved (host) is set
// when it lowered a cell.
cudaError_t launch_sieve(const PnView &v, const int64_t *slot_off_dev, int64_t total_slots, int w, int exhaustive,
                         int grid_blocks, int a_max, cudaStream_t st, int32_t *n_classes_out,
                         const float *topk_thr = nullptr, const uint32_t *focus_anchors = nullptr,
                         int *improved = nullptr);
// nseeds: seeds in the array (host); nseeds_dev (device, may be null): how
// many of them the kernel takes.
cudaError_t launch_complete(const PnView &v, const PnSeed *seeds, int32_t nseeds, const int32_t *nseeds_dev, int dm,
                            int dp, int *improved, int grid_blocks, cudaStream_t st);
// Device-driven rounds (see emit.cu).
// Closes the round's gate when it had no work or lowered no cell; zeroes the
// work count (and *count2 when given).
cudaError_t launch_round_end(int *gate, int *flag, int32_t *count, int32_t *rounds, cudaStream_t st,
                             int32_t *count2 = nullptr);
// Sets each of the first *n_dev seeds' partner j to its cell's current
// neighbour (gated like the round it belongs to).
cudaError_t launch_seeds_refresh(const PnView &v, PnSeed *seeds, int32_t nmax, const int32_t *n_dev, cudaStream_t st);
cudaError_t launch_picks_to_seeds(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *seeds,
                                  int32_t *nseeds, const int *gate, cudaStream_t st);
cudaError_t launch_new_targets(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *done,
                               int32_t *ndone, int32_t done_cap, PnSeed *targets, int32_t *ntargets, const int *gate,
                               cudaStream_t st, PnSeed *near = nullptr, int32_t *nnear = nullptr, int32_t knear = 0);
// Exhaustive sieve of the mixed form on the tensor cores: every valid pair
// of each hot class estimated through an FP16 Gram block of the z-windows
// and only the pairs that can still lower a cell evaluated exactly
// (gram.cu); anchors of at most 192 samples.
bool sieve_gram_supported(int a_max);
// With topk_thr (per anchor), the top-k sieve: only pairs whose estimate can
// fall below their anchor's threshold (and below one of their cells) are evaluated, over the
// tiles that the pivot order leaves (nmem members in all classes).
cudaError_t launch_sieve_gram(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int64_t nmem,
                              int a_max, int grid_blocks, cudaStream_t st, const float *topk_thr = nullptr,
                              int *improved = nullptr);
// Exact row refinement: each target cell (series, m, i) scanned against
// every valid partner at its length; `improved` set when a cell decreased.
// max_windows bounds the partners of any target (the longest series).
cudaError_t launch_refine(const PnView &v, const PnSeed *tg, int32_t ntg, const int32_t *ntg_dev, int64_t max_windows,
                          int m_max, int *improved, int blocks_per_target, cudaStream_t st);
cudaError_t launch_select(const PnView &v, const PnSelGroup *grp_dev, int32_t ngrp, int64_t cell_begin,
                          int64_t cell_end, int32_t cap, double eps0, int32_t kmax, PnPick *out, int32_t *out_cnt,
                          int *overflow, int grid_blocks, cudaStream_t st);
}  // namespace pn
