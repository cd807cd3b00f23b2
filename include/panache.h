/*
 * panache.h -- C ABI of the B300 Panache pan-motif engine.
 *
 * Problem (Sec. 2, "Problem statement"): given a series T = (t_0..t_{n-1}),
 * a length interval [m_min, m_max] and a fixed exclusion zone excl, return
 * top-k pan-motifs: cells (m, i) of the pan matrix profile with a valid
 * neighbour j (|i - j| >= excl) and the exact z-normalised distance
 *   d_m(i, j) = || (T_{i,m} - mu_i) / sigma_i - (T_{j,m} - mu_j) / sigma_j ||_2,
 * ranked by distance, skipping any cell within m/2 (2|i - i'| <= m) of an
 * already accepted cell of the same length.  Distances below eps0 are
 * reported as 0 (Sec. 3.6).  Constant windows (max == min) are ignored.
 *
 * Method (Sec. 3, Algorithms 1-2): per anchor length a in
 * A = {m_min + r s} U {m_max}, every window's normalised non-DC spectrum
 * F = (X_1..X_K')/sigma is kept by a sliding DFT, hashed by SimHash into a
 * global-depth prefix directory with occupancy target alpha, searched with
 * multi-probe under the budget R = gamma alpha, filtered by the Parseval
 * bound LB <= d (Lemma 2) with a (1 - lambda) shrink, and verified exactly;
 * an emit stage runs the hot-class sieve and local completion before the
 * top-k.  Every reported distance is recomputed in FP64 from two-pass
 * moments.
 *
 * Conventions of every entry point:
 *  - Return 0 on success, a negative PANACHE_E* code on failure;
 *    panache_strerror() names it.  On failure no output is written except
 *    where stated (PANACHE_ETRUNC sets *out_len).
 *  - Ownership: the caller owns every input and output buffer; the library
 *    copies what it needs before returning and owns all device state behind
 *    a context or stream handle.
 *  - Series pointers are host memory unless the dtype carries
 *    PANACHE_DEVICE, in which case they are device pointers on the context's
 *    device and are read on the context's stream.
 *  - A context is not thread-safe: use one per host thread.  Calls on one
 *    context are serialised on its CUDA stream and are synchronous (they
 *    return after the results are on the host).
 *  - Results are deterministic for a given input, configuration and seed
 *    (Prop. 6): the profile each call builds is the minimum over the pairs
 *    its candidate rules admit, independent of the GPU schedule.
 *  - Limits: 3 <= m_min <= m_max <= 1024; n <= 2^26 - 1 samples per series;
 *    1 <= k; 1 <= excl; k * (m_max + 1) <= 3500 (selection pool).
 */
#ifndef PANACHE_H
#define PANACHE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define PANACHE_OK 0
#define PANACHE_EINVAL (-1)   /* bad argument (sizes, lengths, null pointers) */
#define PANACHE_ENOMEM (-2)   /* device or host allocation failed */
#define PANACHE_EBUDGET (-3)  /* request footprint above the context's HBM budget (admission refused) */
#define PANACHE_ECUDA (-4)    /* a CUDA call failed; the context should be destroyed */
#define PANACHE_ETRUNC (-5)   /* output capacity too small; *out_len holds the size needed */
#define PANACHE_ESTATE (-6)   /* call not valid in the handle's current state */
#define PANACHE_EPOOL (-7)    /* top-k pool overflow (massive exact ties); results withheld */
#define PANACHE_ENODEV (-8)   /* no CUDA device, or the device is not sm_103 */
#define PANACHE_ETIMEOUT (-9) /* a wait ran out of time before the result was ready */
#define PANACHE_EBUSY (-10)   /* refused at admission: the server's predicted wait exceeds its deadline */

/* ---- sample types (low byte) and pointer location flag ---- */
#define PANACHE_F32 1
#define PANACHE_F64 2
#define PANACHE_DEVICE 0x100

/* ---- precision forms ---- */
#define PANACHE_PLAIN_FP64 0  /* FP64 sliding-DFT state and FP64 in-stream distances */
#define PANACHE_MIXED 1       /* FP32 recurrence from tensor-core anchors, FP32 in-stream distances */

/* ---- top-k modes ---- */
#define PANACHE_TOPK_GLOBAL 0      /* k cells over the whole stack */
#define PANACHE_TOPK_PER_LENGTH 1  /* k cells for every length, ascending m */

/* ---- flags ---- */
#define PANACHE_FLAG_EXHAUSTIVE_SIEVE 0x1  /* every valid pair of a hot class, not only w sort-neighbours */
#define PANACHE_FLAG_SIEVE_GRAM 0x400      /* with the exhaustive sieve, mixed form, anchors of at most 192
                                              samples: estimate every pair of each 128 x 128 block of a class
                                              on the tensor cores (FP16 Gram block of the z-windows shifted by
                                              a reference window, tcgen05 kind::f16, with an error margin) and
                                              evaluate exactly only the pairs that can still lower a cell.
                                              Same rows as evaluating every pair, up to FP32 rounding; on the
                                              wafer-like prefix 1.9% of the pairs are evaluated, but the kernel
                                              is latency-bound (two 4-warp blocks per SM) and takes 143 ms
                                              against 58 ms for the dense CUDA-core tiles, so it is not the
                                              default */
#define PANACHE_FLAG_NO_SIEVE 0x2          /* skip the hot-class sieve (S_hot) */
#define PANACHE_FLAG_NO_COMPLETION 0x4     /* skip local completion (S_local) */
#define PANACHE_FLAG_TIMING 0x8            /* time each step with CUDA events on the context's stream */
#define PANACHE_FLAG_INDEX_ONLY 0x10       /* build features, keys and directories, then stop (no motifs) */
#define PANACHE_FLAG_FP64_ANCHORS 0x20     /* mixed form: chunk anchors by FP64 direct DFT instead of the
                                              tensor cores (3xTF32 tcgen05 contraction, the default) */
#define PANACHE_FLAG_GRAPH 0x40           /* capture a request into two CUDA graphs and replay them while
                                              requests keep the same shape (series lengths, dtypes, length
                                              intervals, k, excl): the index and search steps, and the emit
                                              stage after the hot-class sieve (completion rounds, row
                                              refinement and final selection, whose rounds are decided on
                                              the device); the sieve, which sizes its buffers from counts it
                                              reads back, runs between them.  The context keeps that
                                              request's buffers, copies each new request's samples into
                                              them and launches each graph once */
#define PANACHE_FLAG_HALF_FEATURES 0x80   /* mixed form: the feature-row cache (Sec. 3.2) held in half
                                              precision, 64 B per window and anchor instead of 128 B.  The
                                              rows are the FP32 rows rounded to nearest; the keys and the
                                              sieve order come from the FP32 rows before rounding.  Every
                                              Parseval bound read from half rows is tested with an additive
                                              margin 4 sqrt(m) 2^-11 (the absolute inflation bound in the
                                              proof of Lemma 5), so no pair is pruned that the FP32 rows'
                                              bound keeps.  The query's probe margins read its half row, so
                                              Hamming-1 probes may reorder where margins nearly tie.
                                              EINVAL with the plain form. */
#define PANACHE_FLAG_WARM_START 0x100     /* run a warm start before the search: every query evaluates exactly
                                              the candidate of smallest bound among the 32 most recent valid
                                              entries of its exact bucket (all of them candidates the search
                                              admits), so that candidate cells hold a distance when the search
                                              tests them against max(best_q, P[c]).  Results are the same either
                                              way.  It pays where candidate cells would otherwise still be
                                              empty (the planted walk: 64% fewer exact distances); on series
                                              whose cells mostly hold large distances (the wafer-like series)
                                              the bound passes the same pairs and the extra pass costs more
                                              than it saves, so it is off by default. */
#define PANACHE_FLAG_GRAM_SEARCH 0x800     /* mixed form: run the streaming search with a tensor-core Gram filter
                                              instead of the per-query Parseval test of Lemma 2.  Both evaluate
                                              exactly every listed pair that can still lower a cell, with the
                                              same FP32 arithmetic, so the profile rows and motifs are the same
                                              bit for bit.  The Gram search merges the lists of up to 16 queries
                                              that probe the same bucket first, estimates every listed pair's
                                              squared distance |z_q|^2 + |z_c|^2 - 2 <z_q, z_c> from FP16
                                              windows on the tensor cores (tcgen05, kind::f16) with an error
                                              margin 2^-9 (|z_q|^2 + |z_c|^2), and evaluates a pair only when
                                              that estimate can still lower a cell and is within twice the
                                              margin of its row's or column's best.  On the 200,000-sample
                                              wafer-like prefix it evaluates 8% fewer pairs but runs 3.6
                                              times slower (its block-wide merge, staging and MMA steps leave
                                              the SMs waiting on memory), so it is not the default.  Anchors
                                              longer than 192 samples, budgets above 128, the warm start and
                                              the plain form use the per-query search in any case. */
#define PANACHE_FLAG_TOPK_SIEVE 0x1000     /* mixed form, anchors of at most 192 samples: after the emit stage,
                                              estimate every pair of every hot class on the tensor cores (the
                                              Gram blocks of PANACHE_FLAG_SIEVE_GRAM) against the largest
                                              distance of the refined top lists, evaluate exactly the pairs
                                              that can fall below it and below one of their cells, and run
                                              the rest of the emit stage again.  It finds the near-copy pairs
                                              of large hot classes that the band of w sort neighbours misses;
                                              it and the emit stage after it run eagerly (no graph). */
#define PANACHE_FLAG_NO_FOCUS_SIEVE 0x2000 /* turn off the focused top-k sieve.  By default a global top-k
                                              request in the mixed form (anchors of at most 192 samples, with
                                              its directories: not pmp_from_rows) runs, after the emit stage,
                                              the top-k sieve of PANACHE_FLAG_TOPK_SIEVE restricted to the hot
                                              classes of the anchors next to the lengths of the refined lists'
                                              cells (per series, the largest anchor length <= m and the
                                              smallest >= m), against the largest distance of those lists,
                                              and then the rest of the emit stage again: the near-copy pairs
                                              where the lists live, which the band of w sort neighbours
                                              misses.  A pair below that distance at another anchor is not
                                              looked for (PANACHE_FLAG_TOPK_SIEVE looks at every anchor, and
                                              per-length requests take the sieve only with that flag).  With
                                              PANACHE_FLAG_GRAPH the first emit stage replays its graph and
                                              the sieve and the second emit stage run eagerly. */
#define PANACHE_FLAG_NO_REFINE 0x200      /* skip the exact row refinement of the top list.  After local
                                              completion, every cell of the top refine_mult*k list (per group)
                                              is scanned against all its valid partners at its length with the
                                              in-stream arithmetic and lowered to the smallest distance found;
                                              the list is reselected and new cells scanned until nothing
                                              changes, so every reported cell holds its exact nearest
                                              neighbour.  Not in the paper, whose emit stage never rescans a
                                              row: a row costs n m multiply-adds, tens of microseconds on the
                                              GPU. */

/* Tunables.  A zero field takes the paper's default (Sec. 4):
 * alpha 16, gamma 8 (R = 128), stride 2, K 16, B 24, d0 12, probe cap 8,
 * sieve width 8, (dm, dp) = (6, 4), 8 completion rounds, lambda 1e-4,
 * eps0 1e-6, batch beta = excl, chunk 256 slides per direct-DFT anchor,
 * seed_mult 2, grid_mult 8, refine_mult 4.  One exception: a zero stride is the paper's
 * s = 2 in global top-k mode but s = 1 in per-length mode, where every
 * length's own list must be exact (at s = 2 a length between anchors is
 * reached only through local completion, which can miss a cell whose best
 * pair no anchor's search found); panache_default_config leaves the stride
 * 0 and the context resolves it from the mode. */
typedef struct {
    uint32_t alpha;       /* occupancy target, the analyst's one knob ("budget") */
    uint32_t gamma;       /* R = gamma * alpha candidate inspections per query (R <= 512) */
    uint32_t stride;      /* anchor stride s (0: 2 for global top-k, 1 for per-length top-k) */
    uint32_t K;           /* spectral width, 2..16 (bins 1..K-1 kept) */
    uint32_t B;           /* signature bits, 1..24 */
    uint32_t d0;          /* probe reference depth */
    uint32_t probe_cap;   /* cap on Hamming-1 probes, 1..8 */
    uint32_t sieve_w;     /* sieve width w */
    uint32_t dm, dp;      /* completion radii in length and position (each <= 16) */
    uint32_t rounds;      /* completion rounds P_max */
    uint32_t precision;   /* PANACHE_PLAIN_FP64 or PANACHE_MIXED */
    uint32_t topk_mode;   /* PANACHE_TOPK_GLOBAL or PANACHE_TOPK_PER_LENGTH */
    uint32_t flags;       /* PANACHE_FLAG_* */
    uint32_t chunk;       /* slides per direct-DFT re-anchor (power of two, 16..4096) */
    uint32_t beta;        /* batch length of the streaming schedule (0: excl; capped at excl) */
    uint32_t seed_mult;   /* completion seeds per round: the top seed_mult*k cells (per length in per-length mode) */
    uint32_t grid_mult;   /* resident-block multiple of the search and sieve grids (blocks = SMs * grid_mult) */
    uint32_t refine_mult; /* the row refinement scans the top refine_mult*k cells of each selection group
                             (capped, like the completion seeds, so that the pool holds them) */
    uint32_t _reserved;
    uint64_t seed;        /* seed of the Gaussian projections */
    uint64_t hbm_budget_bytes; /* admission limit on a request's device footprint (0: none) */
    double lambda;        /* bound shrink */
    double eps0;          /* zero-snap threshold */
} panache_config;

/* One motif: cell (m, i) with neighbour j and its FP64 distance d. */
typedef struct {
    int32_t m;
    int32_t _pad;
    int64_t i;
    int64_t j;
    double d;
} panache_motif;

/* One series of a batched request.  Its motifs use the context's top-k mode. */
typedef struct {
    const void *series;
    int32_t dtype;
    int32_t _pad;
    int64_t n;
    int32_t m_min, m_max, k, excl;
} panache_request;

/* Counters of the last request (Sec. 3.7 cost terms). */
typedef struct {
    uint64_t queries;            /* windows searched at anchor lengths */
    uint64_t candidates;         /* candidates inspected (<= R per query) */
    uint64_t exact_stream;       /* exact evaluations in the streaming pass (bound survivors) */
    uint64_t exact_sieve;        /* exact evaluations of the hot-class sieve */
    uint64_t exact_completion;   /* exact evaluations of local completion */
    uint64_t hot_classes;        /* buckets larger than R at the final depth */
    uint64_t completion_rounds;  /* rounds run (stops early when nothing improves) */
    uint64_t device_bytes;       /* device footprint of the request (admission estimate) */
    uint64_t kernel_launches;    /* kernels launched by the request */
    uint64_t waves;              /* waves a batch was split into to fit the HBM budget */
    uint64_t refine_passes;      /* passes of the row refinement (reselect, scan new top cells) */
    uint64_t exact_refine;       /* exact evaluations of the row refinement */
    /* With PANACHE_FLAG_TIMING: device time of each step in ms (CUDA events on
     * the context's stream): 0 sample upload and conversion, 1 run lengths and
     * FP64 prefix moments, 2 features and keys, 3 ranks and directories,
     * 4 streaming search, 5 hot-class sieve, 6 completion rounds (with their
     * seed selections), 7 final selection and FP64 verification. */
    double step_ms[8];
} panache_stats;

typedef struct panache_ctx panache_ctx;
typedef struct panache_stream panache_stream;

/* Fills *cfg with the paper's defaults. */
int panache_default_config(panache_config *cfg);

/* Creates a context on the current CUDA device (which must be sm_103).
 * cfg may be null (defaults).  `panache_create(budget)` of the paper's
 * statement is a config with only alpha set.  Errors: EINVAL, ENODEV, ECUDA. */
int panache_create(const panache_config *cfg, panache_ctx **out);

/* Releases every device buffer of the context.  Null is ignored. */
void panache_destroy(panache_ctx *ctx);

/* Runs the context's work on `cuda_stream` (a cudaStream_t; null: the
 * context's own stream). */
int panache_set_stream(panache_ctx *ctx, void *cuda_stream);

/* One series: top-k pan-motifs into out[0..out_cap).  *out_len receives the
 * number written (fewer than k when fewer cells exist; k per length in
 * per-length mode).  ETRUNC when out_cap is too small (with *out_len set to
 * the count needed).  Errors: EINVAL, ENOMEM, EBUDGET, ECUDA, EPOOL. */
int panache_pmp(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min, int32_t m_max,
                int32_t k, int32_t excl, panache_motif *out, int64_t out_cap, int64_t *out_len);

/* Anchor sharding of one series across ranks, one process per GPU (Sec. 3.5:
 * every anchor owns its spectral state, directory and profile row and
 * shares nothing with the others).  panache_pmp_anchor_shard indexes,
 * searches and sieves only the anchors at positions p of
 * A = (m_min, m_min + s, ..., m_max) with p mod world == rank, and copies
 * the resulting profile rows (the layout of panache_profile_rows:
 * [m_max - m_min + 1][n] packed keys, empty cells all ones) into the host
 * array rows[0..cap).  The ranks' rows merge by the elementwise minimum of
 * the keys as unsigned 64-bit integers; panache_pmp_from_rows runs the rest
 * of the emit stage (local completion, row refinement, selection) on merged
 * host rows, with the series present, and writes the motifs as panache_pmp
 * does.  The motifs equal panache_pmp's on the same series and
 * configuration: the stream and sieve rows of a length come from its own
 * anchor alone, and the profile is the minimum over the admitted pairs
 * whatever the schedule.  Errors: EINVAL (rank outside [0, world), sizes),
 * ETRUNC (cap < L n), the others as panache_pmp. */
int panache_pmp_anchor_shard(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                             int32_t m_max, int32_t k, int32_t excl, int32_t rank, int32_t world, uint64_t *rows,
                             int64_t cap);
int panache_pmp_from_rows(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min, int32_t m_max,
                          int32_t k, int32_t excl, const uint64_t *rows, panache_motif *out, int64_t out_cap,
                          int64_t *out_len);

/* Many independent series in one set of launches (the batched form).  The
 * motifs of request r go to out[r * out_cap_per_req ...], their count to
 * out_len[r].  The batch runs in waves of consecutive series whose device
 * footprint fits hbm_budget_bytes (when unset: 60% of the free device
 * memory); each series' result does not depend on the split.  Errors as
 * panache_pmp; EBUDGET when a single series exceeds the budget. */
int panache_pmp_batch(panache_ctx *ctx, const panache_request *reqs, int32_t nreq, panache_motif *out,
                      int64_t out_cap_per_req, int64_t *out_len);

/* Streaming handles (Sec. 3.1): samples arrive by panache_append in chunks
 * of any size (host memory, or device memory with PANACHE_DEVICE; FP32 or
 * FP64; the call copies them).  The whole index stays resident on the
 * device until panache_stream_close: samples, FP64 prefix sums, features
 * and keys, directory levels and profile rows, laid out for a capacity that
 * grows to max(2 cap, 1.5 n) when an append outgrows it (the state is then
 * rebuilt from the samples).  An append computes the features of the new windows and
 * searches every query whose batch of beta samples it completes
 * (Algorithm 1: such a query's population, level and candidates are final).
 * panache_stream_topk searches the still-pending queries and runs the emit
 * stage (Algorithm 2) on a copy of the profile rows, so its result equals
 * panache_pmp on the samples received so far and the resident state does
 * not depend on when snapshots were taken.  Both calls run on the
 * context's stream and return when the work is done.  Errors as
 * panache_pmp; ETIMEOUT when a bounded device wait ran out.  Destroying the
 * context frees the device state of its open streams; their handles then
 * fail with ESTATE until panache_stream_close releases them. */
int panache_stream_open(panache_ctx *ctx, int32_t m_min, int32_t m_max, int32_t k, int32_t excl,
                        panache_stream **out);
int panache_append(panache_stream *h, const void *chunk, int32_t dtype, int64_t len);
int panache_stream_topk(panache_stream *h, panache_motif *out, int64_t out_cap, int64_t *out_len);
int64_t panache_stream_length(const panache_stream *h);
void panache_stream_close(panache_stream *h);
/* Checkpoint of a stream: its samples as FP64 (out[0..cap), *out_len set to
 * the length; ETRUNC when cap is smaller).  Every part of a stream's state
 * is a function of its samples and the context's configuration, so opening
 * a stream with the same parameters and appending the checkpoint (in one
 * chunk or any others) resumes it: later snapshots equal those of the
 * uninterrupted stream. */
int panache_stream_checkpoint(const panache_stream *h, double *out, int64_t cap, int64_t *out_len);

/* Counters of the context's last request. */
int panache_last_stats(const panache_ctx *ctx, panache_stats *out);

/* Copies the last request's profile rows of series `series_index`
 * (packed keys, layout [m_max - m_min + 1][n]: the IEEE-754 bits of the
 * in-stream distance with the low 26 bits replaced by the neighbour index;
 * 0xFFFFFFFFFFFFFFFF for an empty cell) into keys[0..cap).  ETRUNC when cap
 * is smaller than the row block.  The state is kept until the next request. */
int panache_profile_rows(const panache_ctx *ctx, int32_t series_index, uint64_t *keys, int64_t cap);

/* Copies anchor `anchor_index` (0-based in A of series `series_index`) of
 * the last request: its length, the feature rows [nw][32] as floats (bins
 * re, im interleaved / sigma, zero padded; the half rows widened under
 * PANACHE_FLAG_HALF_FEATURES) and the B-bit keys [nw].  Either
 * output may be null.  Used by the parity tests. */
int panache_anchor_state(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, int32_t *a_out,
                         float *features, uint32_t *keys, int64_t cap_windows);

/* Fault injection for tests of the failure paths (the paper has no
 * counterpart).  Arms one failure, made on the host, of a later operation of
 * the given kind in this process; `after` operations of that kind succeed
 * first, then one fails and the hook disarms itself:
 *   PANACHE_FAULT_ALLOC    a device allocation of a request's state: the
 *                          call returns ENOMEM
 *   PANACHE_FAULT_COPY     the upload of a request's samples: the call
 *                          returns ECUDA without the copy being issued
 *   PANACHE_FAULT_TC_WAIT  the next tensor-core anchor launch (mixed form)
 *                          issues no MMA and every CTA's bounded wait runs
 *                          out after a few tries: the kernel records the
 *                          timeout, zeroes its anchor rows, frees its tensor
 *                          memory and returns; the call returns ETIMEOUT
 *                          (never armed into a graph being captured)
 * PANACHE_FAULT_NONE disarms.  No GPU is faulted: the context stays usable
 * and its next request runs normally.  Errors: EINVAL. */
#define PANACHE_FAULT_NONE 0
#define PANACHE_FAULT_ALLOC 1
#define PANACHE_FAULT_COPY 2
#define PANACHE_FAULT_TC_WAIT 3
int panache_inject_fault(int32_t kind, int32_t after);

/* Device time of individual kernels in the last request made with
 * PANACHE_FLAG_TIMING (CUDA events on the context's stream around each
 * launch, summed; the last wave of a batch): ms[k] and launches[k] for
 * k = 0 tensor-core chunk anchors, 1 sliding DFT + normalisation + keys,
 * 2 streaming search, 3 hot-class sieve evaluation (without its sorts),
 * 4 local completion (without its seed selections), 5 selection (every
 * seed selection and the final top-k), 6 exact row refinement, 7 the
 * top-k sieve after the emit stage (focused or at every anchor, with its
 * pivot pre-pass).  Zero without the flag.  ETRUNC when cap < 8. */
#define PANACHE_KERNEL_TIMES 8
int panache_kernel_times(const panache_ctx *ctx, double *ms, uint64_t *launches, int32_t cap);

/* The budgeted candidate list (Sec. 3.4) each listed query window q[i] of
 * anchor `anchor_index` of series `series_index` in the last request is
 * searched with, built on the device by the search kernel's own code: the
 * exact d-bit prefix bucket of its key, then its Hamming-1 buckets in
 * increasing projection margin, each bucket's valid entries (start <=
 * q - excl, ascending) taken in full while the budget R allows, else the
 * evenly spaced half then the most recent half.  cand[i * cap ...] receives
 * up to cap window starts, counts[i] the list's length (-1 for a window the
 * search skips: constant, or q < excl).  Host arrays.  Used by the parity
 * tests.  Errors: EINVAL, ESTATE with no request yet. */
int panache_query_candidates(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, const int64_t *q,
                             int32_t nq, uint32_t *cand, int32_t cap, int32_t *counts);

/* Directory population and global depth that every window of anchor
 * `anchor_index` of series `series_index` in the last request is searched
 * with (Sec. 3.5 and Prop. 4): samples arrive in batches of beta, every
 * window a batch completes is inserted before the batch's searches, so the
 * query whose last sample is t sees the non-constant windows completed by
 * the end of t's batch; its depth is the smallest d with population <=
 * alpha 2^d, capped at B.  population[q] and depth[q] (q < nw, host arrays
 * of cap_windows entries) are -1 for windows the search skips (constant
 * windows, and q < excl).  The values are computed on the device by the
 * search kernel's own rule.  ETRUNC when cap_windows < nw; ESTATE with no
 * request yet.  Used by the parity tests. */
int panache_query_levels(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, int32_t *population,
                         int32_t *depth, int64_t cap_windows);

/* Spectral-width calibration (Sec. 3.2, "Spectral width selection"): the
 * width K is fixed before insertion as the smallest K in [2, 16] with
 *   E[(2/m^2) sum_{k<=K'(m)} |X^_k|^2] >= eta          (retained energy)
 *   n E[(1 - theta_K/pi)^B] <= 2 gamma alpha           (accidental collisions)
 * over sampled windows: up to 256 evenly spaced non-constant windows at each
 * of m_min, (m_min+m_max)/2 and m_max; angles theta_K between the K-width
 * features of two windows of one length, pairs whose full-width bound is
 * below 0.1 sqrt(2m) (near-duplicates) left out; K = 16 when no width
 * qualifies.  B, gamma and alpha come from the context's configuration; eta
 * 0 means 0.85.  *K_out receives K; energy[0..14] and collision_prob[0..14]
 * (either may be null) receive the two sample means E[...] for K = 2..16.
 * The series is host or device memory (dtype as panache_pmp).  Use K in the
 * configuration of the context that then runs the series.  Errors: EINVAL,
 * ENOMEM, ECUDA. */
int panache_calibrate_width(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                            int32_t m_max, double eta, int32_t *K_out, double *energy, double *collision_prob);

/* Writes the FP32 Gaussian projections g_{a,l} (l = 1..B+1, row-major
 * [B+1][32], dimensions >= 2(K-1) zero) that a context with configuration
 * cfg (null: defaults) draws for anchor length a (Sec. 3.4).  Host-only: no
 * device is needed.  ETRUNC when cap < (B+1)*32. */
int panache_projections(const panache_config *cfg, int32_t a, float *g, int64_t cap);

const char *panache_strerror(int code);

/* Measured throughput, in TFLOP/s, of one arithmetic pipe on the current
 * device: kind 0 FP32 fused multiply-add, 1 packed two-wide FP32 fused
 * multiply-add, 2 FP64 fused multiply-add (2 flop per multiply-add, one
 * launch of about 50 ms after a warm-up, CUDA events).  These are the
 * denominators of the per-kernel roofline fractions; the paper has no
 * counterpart.  Errors: EINVAL, ENODEV, ENOMEM, ECUDA. */
int panache_alu_peak(int32_t kind, double *tflops);

/* ---- request server (continuous batching under an HBM budget) ----
 *
 * A server runs `slots` worker threads, each with its own context and CUDA
 * stream, so requests of different slots overlap on the GPU.  A request
 * reserves its device footprint (the planner's estimate) from the budget
 * before it runs and releases it when its motifs are on the host; one larger
 * than the whole budget is refused at submission (EBUDGET), and one that
 * does not fit beside the live streams' reservations while no batch is
 * running is refused when it reaches the head of the queue (its wait returns
 * EBUDGET) rather than waiting for streams to close.  A free slot
 * takes, in arrival order, every queued request that fits the free budget
 * and the slot's share of it (budget / slots) and runs them as one batch.
 * Results do not depend on which requests share a batch or run alongside.
 * Latency is measured from submission to the motifs being on the host.
 * The server's contexts use cfg (the paper's defaults when null) and the
 * device current at creation.  All calls are thread-safe. */
typedef struct panache_server panache_server;

typedef struct {
    uint64_t submitted, completed, failed, queued, batches;
    uint64_t windows_lengths;      /* sum over completed requests and snapshots */
    uint64_t budget_bytes, peak_reserved_bytes;
    uint32_t max_concurrent_batches, _pad;
    double span_ms;                /* first submission to last completion */
    double p50_ms, p99_ms, mean_ms;   /* request latency of completed requests (snapshots apart) */
    uint64_t refused;              /* requests refused at submission by the deadline (EBUSY) */
    double snap_p50_ms, snap_p99_ms;  /* stream snapshot latency: call to motifs on the host */
    uint64_t refused_snapshots;    /* stream snapshots refused by the deadline (EBUSY) */
} panache_server_stats;

/* hbm_budget_bytes 0: 60% of the free device memory.  1 <= slots <= 64.
 * The server also runs max(4, 2 slots) stream worker threads. */
int panache_server_create(const panache_config *cfg, int32_t slots, uint64_t hbm_budget_bytes,
                          panache_server **out);
/* Drains the queue, stops the workers and frees everything. */
void panache_server_destroy(panache_server *sv);
/* Queues a host series (copied before returning); *ticket names the request. */
int panache_server_submit(panache_server *sv, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                          int32_t m_max, int32_t k, int32_t excl, uint64_t *ticket);
/* Waits up to timeout_ms (negative: forever, 0: poll) for a request; on
 * success copies its motifs and latency and forgets the ticket.  ETIMEOUT
 * when not ready; the request's own error code when it failed. */
int panache_server_wait(panache_server *sv, uint64_t ticket, int32_t timeout_ms, panache_motif *out, int64_t cap,
                        int64_t *out_len, double *latency_ms);
/* Live streams: each is a resident stream (panache_stream_open) on a
 * context and CUDA stream of its own, so its appends and snapshots overlap
 * one another and the slots' batches on the GPU.  panache_server_append
 * copies the chunk (host, FP32 or FP64) and queues it; stream worker
 * threads apply each stream's queued operations in order, a run of
 * consecutive appends as one append.  The resident state plus the row copy
 * a snapshot uses are reserved from the budget when the append is accepted;
 * an append that would grow them past it fails at the call with EBUDGET
 * (the stream keeps its samples).  A failure while an append is applied is
 * kept and returned by the stream's later appends and snapshots.
 * panache_server_stream_topk queues a top-k over every sample accepted
 * before it and returns its ticket for panache_server_wait (latency: from
 * the call to the motifs on the host).  ESTATE when the stream has no
 * samples.  panache_server_stream_close applies the stream's pending
 * operations, then frees it and its reservation. */
int panache_server_stream_open(panache_server *sv, int32_t m_min, int32_t m_max, int32_t k, int32_t excl,
                               uint64_t *stream_id);
int panache_server_append(panache_server *sv, uint64_t stream_id, const void *chunk, int32_t dtype, int64_t len);
int panache_server_stream_topk(panache_server *sv, uint64_t stream_id, uint64_t *ticket);
int panache_server_stream_close(panache_server *sv, uint64_t stream_id);
int panache_server_get_stats(panache_server *sv, panache_server_stats *out);
/* Deadline admission (0, the default: off).  A request whose predicted wait
 * -- the windows x lengths queued ahead of it plus its own, over the
 * server's measured request throughput (what completed in the last two
 * seconds; before that, a smoothed per-batch rate times the slots) --
 * exceeds three quarters of deadline_ms (the rest covers the estimate's
 * error) is refused at submission with EBUSY.  A stream
 * snapshot is refused with EBUSY when the snapshots queued ahead of it and
 * itself, at the measured time per snapshot spread over the stream workers,
 * exceed the deadline.  Above its capacity the server then sheds load
 * instead of letting the queues, and every latency, grow.  Errors: EINVAL. */
int panache_server_set_deadline(panache_server *sv, double deadline_ms);

/* Top-k motifs of ONE length row from profile keys already on the device,
 * with no device memory allocated by the call.  For callers that cannot call
 * cudaMalloc -- for example code that runs inside another framework's
 * memory pool or under a budget that forbids new device allocations.  The
 * paper has no counterpart: it is the selection step of panache_pmp offered
 * on its own.
 *
 *  x          device FP64 samples of the series, n of them
 *  m          the row's length (3 <= m <= min(n, 1024))
 *  keys       device row of n packed keys (layout of panache_profile_rows;
 *             cells past n - m and empty cells are 0xFFFFFFFFFFFFFFFF)
 *  k          motifs wanted; k * (m + 1) <= PANACHE_NOALLOC_NEED_MAX (6300)
 *  eps0       zero-snap threshold (the library's default is 1e-6)
 *  out        device array of at least k motifs (written)
 *  out_count  device int32 (written): the number of motifs, or
 *             PANACHE_EPOOL when massive exact ties overflowed the pool
 *  stream     cudaStream_t to run on (null: the legacy default stream)
 * Same rule and FP64 re-verification as panache_pmp's final selection.
 * Scratch: one fixed array of about 145 KB in device memory, defined in the
 * library and kept by every GPU that loads it until the process exits.  The
 * first call on each device looks up its address (with that device
 * current), so make that first call before any stream capture.  The call
 * only enqueues work: read out_count after synchronising the stream.  All
 * calls share the one array, so calls that overlap on the GPU (different
 * streams, or threads) race; serialise them.  Errors: EINVAL for sizes out
 * of range or null pointers, ENODEV, ECUDA.  When the calling thread
 * already has a CUDA error pending from earlier work, the call enqueues
 * nothing, returns ECUDA and leaves that error pending for its owner. */
#define PANACHE_NOALLOC_NEED_MAX 6300
int panache_topk_row_noalloc(const double *x, int64_t n, int32_t m, const uint64_t *keys, int32_t k, double eps0,
                             panache_motif *out, int32_t *out_count, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* PANACHE_H */
