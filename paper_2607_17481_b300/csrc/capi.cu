// Host runtime and C ABI: planning, admission, device buffers and the
// order of the steps (Algorithm 1 over all anchors, then Algorithm 2).
#include <algorithm>
#include <limits>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <set>
#include <new>
#include <tuple>
#include <vector>

#include "emit.cuh"
#include "kernels.cuh"
#include "panache.h"
#include "philox.h"
#include "prims.cuh"
#include "runtime.h"

namespace {

using SeriesIn = PnSeriesIn;

int from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return PANACHE_OK;
    if (e == cudaErrorMemoryAllocation) return PANACHE_ENOMEM;
    return PANACHE_ECUDA;
}

#define PN_TRY(expr)                         \
    do {                                     \
        int rc_ = (expr);                    \
        if (rc_ != PANACHE_OK) return rc_;   \
    } while (0)
#define PN_CU(expr) PN_TRY(from_cuda(expr))

// Host-side fault injection (panache_inject_fault): the armed kind and how
// many matching operations still succeed before it fires once.
std::atomic<int> g_fault_kind{PANACHE_FAULT_NONE};
std::atomic<int> g_fault_after{0};

bool fault_fires(int kind) {
    if (g_fault_kind.load() != kind) return false;
    if (g_fault_after.fetch_sub(1) > 0) return false;
    int k = kind;
    return g_fault_kind.compare_exchange_strong(k, PANACHE_FAULT_NONE);
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Sample conversion: raw host/device series -> FP64 and (hi, lo) float pairs.
struct PnConv {
    const void *src;
    int64_t n;
    int64_t x_off;
    int32_t dtype;
    int32_t _pad;
};

__global__ void k_convert(const PnConv *cv, int32_t ncv, int64_t total, double *x, float2 *xs, float *x1) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int c = pn_find(cv, ncv, t, [](const PnConv &e) { return e.x_off; });
    const PnConv &e = cv[c];
    int64_t i = t - e.x_off;
    double v = (e.dtype & 0xFF) == PANACHE_F32 ? (double)((const float *)e.src)[i] : ((const double *)e.src)[i];
    float hi = (float)v;
    x[t] = v;
    xs[t] = make_float2(hi, (float)(v - (double)hi));
    if (x1) x1[t] = hi;
}

// Stream samples: n values (FP32 or FP64) written at offset `off` as FP64 and
// as (hi, lo) float pairs.
__global__ void k_put(const void *src, int32_t dtype, int64_t n, int64_t off, double *x, float2 *xs) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    double v = (dtype & 0xFF) == PANACHE_F32 ? (double)((const float *)src)[t] : ((const double *)src)[t];
    float hi = (float)v;
    x[off + t] = v;
    xs[off + t] = make_float2(hi, (float)(v - (double)hi));
}

}  // namespace

// Device buffers of one selection group set: the groups, the picks
// [ngroups][kmax] and their counts, kept with the request so that the
// launches can be replayed.
struct SelBufs {
    PnSelGroup *dg = nullptr;
    PnPick *out = nullptr;
    int32_t *cnt = nullptr;
    int32_t ng = 0, kmax = 1, cap = 0;
};

// The emit stage after the sieve: its control words, the seed, refinement
// and final selection groups, and the seed and target lists.  Built once per
// request (kept with the request when the stage is replayed from a graph).
enum { C_GATE = 0, C_FLAG, C_NSEED, C_ROUNDS, R_GATE, R_FLAG, R_NTG, R_PASSES, OV_FINAL, OV_OTHER, R_NNEAR, C_WORDS };
struct EmitPlan {
    int32_t *ctl = nullptr;
    SelBufs sb, rb, fb;
    PnSeed *dseeds = nullptr, *dtg = nullptr, *ddone = nullptr, *dnear = nullptr;
    int32_t *ndone = nullptr;
    int32_t done_cap = 0;
    int32_t knear = 0;                 // picks per group whose new targets seed a completion
    int64_t max_windows = 0;
    int m_top = 3;
    bool completion = false, refine = false;
    void *pin = nullptr;               // graph replay: the pinned result buffer its copies write to
    ~EmitPlan() {
        if (pin) cudaFreeHost(pin);
    }
};

// ---------------------------------------------------------------------------
// One request: tables, device buffers and results.
// ---------------------------------------------------------------------------
struct PnRequest {
    std::vector<PnSeries> ser;
    std::vector<PnAnchor> anc;
    std::vector<PnLevel> lev;
    std::vector<int32_t> blk_anchor, blk_chunk0;
    std::vector<int32_t> tile_anchor, tile_row0;   // tensor-core anchor tiles (128 chunks each)
    int64_t total_chunks = 0;
    std::vector<int64_t> slot_off;
    int64_t total_samples = 0, total_windows = 0, total_rows = 0, total_items = 0, total_buckets = 0;
    int64_t total_cells = 0, total_slots = 0;
    int a_max = 0;
    size_t footprint = 0;

    std::vector<void *> allocs;
    cudaStream_t st = nullptr;
    PnSeries *d_ser = nullptr;
    PnAnchor *d_anc = nullptr;
    PnLevel *d_lev = nullptr;
    int32_t *d_blk_anchor = nullptr, *d_blk_chunk0 = nullptr;
    int32_t *d_tile_anchor = nullptr, *d_tile_row0 = nullptr;
    float *tca = nullptr;      // tensor-core chunk anchors
    float *twb = nullptr;      // their twiddle operand, [anchor][32][a_max]
    int *err = nullptr;
    int64_t *d_slot_off = nullptr;
    double *x = nullptr;
    float2 *xs = nullptr;
    float *x1 = nullptr;
    double2 *sq = nullptr;
    double *shift = nullptr;
    int32_t *runlen = nullptr;
    float *F = nullptr;
    __half *Fh = nullptr;      // half-precision rows (PANACHE_FLAG_HALF_FEATURES) in place of F
    float *sproj = nullptr;    // per-window sieve projections, from the FP32 rows
    uint32_t *sig = nullptr, *cnt = nullptr, *nclist = nullptr, *qorder = nullptr;
    float2 *wmf = nullptr;
    double2 *wmd = nullptr;
    float *g = nullptr, *gT = nullptr;
    uint32_t *dir_keys = nullptr, *dir_vals = nullptr, *bstart = nullptr;
    unsigned long long *prof = nullptr, *stats = nullptr;
    int *flagbuf = nullptr;
    EmitPlan *emit = nullptr;          // the emit stage's buffers, kept for graph replay

    // Buffers come from the stream-ordered pool of the request's stream and
    // go back to it in stream order, so requests on different streams never
    // synchronise the device through allocation.
    ~PnRequest() {
        for (void *p : allocs) cudaFreeAsync(p, st);
        delete emit;
    }

    template <class T>
    cudaError_t alloc(T *&p, int64_t count) {
        p = nullptr;
        if (fault_fires(PANACHE_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
        if (count <= 0) count = 1;
        cudaError_t e = cudaMallocAsync((void **)&p, sizeof(T) * (size_t)count, st);
        if (e == cudaSuccess) allocs.push_back(p);
        return e;
    }
};

struct panache_ctx {
    panache_config cfg;
    int device = 0;
    int sm_count = 148;
    cudaStream_t own = nullptr;
    cudaStream_t st = nullptr;
    PnRequest *last = nullptr;
    panache_stats stats;
    std::map<int, std::vector<float>> gcache;
    std::set<panache_stream *> streams;   // open streams: their state is freed with the context
    uint64_t launches = 0;
    PnKTimer kt;                          // per-kernel device time of the last request (PANACHE_FLAG_TIMING)
    // PANACHE_FLAG_GRAPH: the captured index + search steps of `last`, the
    // request shape they were captured for, and the persistent input staging
    cudaGraphExec_t gexec = nullptr;
    cudaGraphExec_t gexec_emit = nullptr;  // the emit stage after the sieve, same shape
    std::vector<PnSeriesIn> gshape;
    unsigned char *gstage = nullptr;
    std::vector<int64_t> gstage_off;
    uint64_t glaunches = 0, glaunches_emit = 0;
    // pinned host buffers the emit stage's results are copied into
    void *pin = nullptr;
    size_t pin_bytes = 0;

    void drop_graph() {
        if (gexec) cudaGraphExecDestroy(gexec);
        if (gexec_emit) cudaGraphExecDestroy(gexec_emit);
        gexec = nullptr;
        gexec_emit = nullptr;
        gshape.clear();
        gstage = nullptr;            // owned by `last` (allocated through it)
        gstage_off.clear();
    }

    int pinned(size_t bytes, void **out) {
        if (bytes > pin_bytes) {
            if (pin) cudaFreeHost(pin);
            pin = nullptr;
            pin_bytes = 0;
            if (cudaMallocHost(&pin, bytes) != cudaSuccess) return PANACHE_ENOMEM;
            pin_bytes = bytes;
        }
        *out = pin;
        return PANACHE_OK;
    }

    const std::vector<float> &proj(int a) {
        auto it = gcache.find(a);
        if (it != gcache.end()) return it->second;
        std::vector<float> g((size_t)(cfg.B + 1) * PN_FEAT);
        pn::projections(a, cfg.seed, (int)cfg.B, (int)cfg.K, g.data());
        return gcache.emplace(a, std::move(g)).first->second;
    }
};

// A live series whose whole index stays resident (Sec. 3.1): samples, prefix
// sums, features and keys, ranks, directory levels and profile rows, all laid
// out for `cap` samples.  Appends search only the queries whose batch the new
// samples complete; a snapshot searches the pending tail and runs Algorithm 2
// on a copy of the rows, so the resident state never depends on when
// snapshots were taken.
struct panache_stream {
    panache_ctx *ctx;
    int32_t m_min, m_max, k, excl;
    PnRequest *R = nullptr;
    int64_t len = 0, cap = 0;
    std::vector<int64_t> q_done;   // per anchor: queries [0, q_done) searched into the resident rows
    std::vector<int64_t> nw_feat;  // per anchor: windows whose features and keys are written
    ~panache_stream() { delete R; }
};

namespace {

// Zero fields take their defaults.  The anchor stride's default depends on
// the top-k mode, so panache_default_config leaves it 0 (`resolve` false)
// and the context resolves it: the paper's s = 2 for the top-k over the whole
// stack, s = 1 for per-length top-k, where every length's list must be
// exact and a length without an anchor of its own is reached only through
// local completion.
void fill_defaults(panache_config &c, bool resolve = true) {
    if (!c.alpha) c.alpha = 16;
    if (!c.gamma) c.gamma = 8;
    if (!c.stride && resolve) c.stride = c.topk_mode == PANACHE_TOPK_PER_LENGTH ? 1u : 2u;
    if (!c.K) c.K = 16;
    if (!c.B) c.B = 24;
    if (!c.d0) c.d0 = 12;
    if (!c.probe_cap) c.probe_cap = 8;
    if (!c.sieve_w) c.sieve_w = 8;
    if (!c.dm) c.dm = 6;
    if (!c.dp) c.dp = 4;
    if (!c.rounds) c.rounds = 8;
    if (!c.chunk) c.chunk = 256;
    if (!c.seed_mult) c.seed_mult = 2;
    if (!c.grid_mult) c.grid_mult = 8;
    if (!c.refine_mult) c.refine_mult = 4;
    if (c.lambda == 0.0) c.lambda = 1e-4;
    if (c.eps0 == 0.0) c.eps0 = 1e-6;
}

int check_config(const panache_config &c) {
    if (c.K < 2 || c.K > PN_MAXK || c.B < 1 || c.B > PN_MAXB) return PANACHE_EINVAL;
    if ((int)(c.gamma * c.alpha) > pn::search_max_budget() || c.alpha > (1u << 20)) return PANACHE_EINVAL;
    if (c.probe_cap < 1 || c.probe_cap > 8 || c.precision > 1 || c.topk_mode > 1) return PANACHE_EINVAL;
    if ((c.flags & PANACHE_FLAG_HALF_FEATURES) && c.precision != PANACHE_MIXED) return PANACHE_EINVAL;
    if (c.chunk < 16 || c.chunk > 4096 || (c.chunk & (c.chunk - 1))) return PANACHE_EINVAL;
    if (c.grid_mult > 64 || c.dm > 16 || c.dp > 16 || c.refine_mult > 64) return PANACHE_EINVAL;
    if (!(c.lambda > 0.0 && c.lambda < 1.0) || !(c.eps0 >= 0.0)) return PANACHE_EINVAL;
    return PANACHE_OK;
}

int check_series(const SeriesIn &s) {
    const int dt = s.dtype & 0xFF;
    if (!s.ptr && s.n > 0) return PANACHE_EINVAL;
    if ((dt != PANACHE_F32 && dt != PANACHE_F64) || (s.dtype & ~0x1FF)) return PANACHE_EINVAL;
    if (s.n < 0 || s.n > PN_MAX_SERIES_LEN) return PANACHE_EINVAL;
    if (s.m_min < 3 || s.m_max < s.m_min || s.m_max > 1024) return PANACHE_EINVAL;
    if (s.k < 1 || s.excl < 1) return PANACHE_EINVAL;
    return PANACHE_OK;
}

// Anchor sharding of one series across ranks (Sec. 3.5: each anchor owns its
// state and shares nothing): a rank indexes, searches and sieves the anchors
// at positions p of A with p mod world == rank and hands out its profile
// rows (rows_out); the merged rows (elementwise minimum over the ranks) come
// back through rows_in for the emit stage's completion, refinement and
// selection.
struct PnShard {
    int32_t rank = 0, world = 1;
    const uint64_t *rows_in = nullptr;   // emit only: the merged rows [L][n]
    uint64_t *rows_out = nullptr;        // shard: this rank's rows [L][n]
};

// Builds every table of a request and its device footprint.  With `caps`,
// series s is laid out for caps[s] >= n samples (a resident stream): every
// per-window array, feature block, directory level and profile row is sized
// for the capacity, while n, nw and the launches cover the samples present.
int plan(const panache_config &c, const std::vector<SeriesIn> &in, PnRequest &R,
         const std::vector<int64_t> *caps = nullptr, const PnShard *sh = nullptr) {
    const int C = (int)c.chunk;
    int64_t x_off = 0, row_off = 0;
    for (size_t s = 0; s < in.size(); ++s) {
        const SeriesIn &si = in[s];
        const int64_t ncap = caps ? (*caps)[s] : si.n;
        PnSeries S;
        memset(&S, 0, sizeof(S));
        S.x_off = x_off;
        S.n = si.n;
        S.row_off = row_off;
        S.ld = ncap;
        S.m_min = si.m_min;
        S.m_max = si.m_max;
        S.excl = si.excl;
        S.k = si.k;
        S.mode = (int32_t)c.topk_mode;
        S.anchor_begin = (int32_t)R.anc.size();
        std::vector<int> al;
        for (int a = si.m_min; a <= si.m_max; a += (int)c.stride) al.push_back(a);
        if (al.back() != si.m_max) al.push_back(si.m_max);
        if (sh && sh->world > 1) {
            std::vector<int> mine;
            for (size_t p = 0; p < al.size(); ++p)
                if ((int32_t)(p % (size_t)sh->world) == sh->rank) mine.push_back(al[p]);
            al.swap(mine);
        }
        for (int a : al) {
            const int64_t nwc = ncap - a + 1;             // windows at capacity
            if (nwc <= 0) continue;
            PnAnchor A;
            memset(&A, 0, sizeof(A));
            A.series = (int32_t)s;
            A.a = a;
            A.kp = pn_kprime(a, (int)c.K);
            A.nw = std::max<int64_t>(0, si.n - a + 1);
            A.dmax = pn_depth(nwc, (int)c.alpha, (int)c.B);
            A.win_off = R.total_windows;
            A.nchunk = (nwc + C - 1) / C;
            A.chunk_off = R.total_chunks;
            A.row_off = R.total_rows;
            A.item_off = R.total_items;
            A.bucket_base = R.total_buckets;
            A.level_begin = (int32_t)R.lev.size();
            A.nlevels = A.dmax + 1;
            for (int d = 0; d <= A.dmax; ++d) {
                PnLevel L;
                L.anchor = (int32_t)R.anc.size();
                L.d = d;
                L.cap = std::min<int64_t>(nwc, (int64_t)c.alpha << d);
                L.item_off = R.total_items;
                L.bucket_base = R.total_buckets;
                R.total_items += L.cap;
                R.total_buckets += (int64_t)1 << d;
                R.lev.push_back(L);
            }
            const int64_t nch_now = (A.nw + C - 1) / C;
            for (int64_t b = 0; b < nch_now; b += PN_FT_CHUNKS) {
                R.blk_anchor.push_back((int32_t)R.anc.size());
                R.blk_chunk0.push_back((int32_t)b);
            }
            for (int64_t b = 0; b < nch_now; b += 128) {
                R.tile_anchor.push_back((int32_t)R.anc.size());
                R.tile_row0.push_back((int32_t)b);
            }
            R.total_chunks += A.nchunk;
            R.slot_off.push_back(R.total_slots);
            R.total_slots += (int64_t)1 << A.dmax;
            R.total_windows += nwc;
            R.total_rows += A.nchunk * C;
            R.a_max = std::max(R.a_max, a);
            R.anc.push_back(A);
        }
        S.anchor_count = (int32_t)R.anc.size() - S.anchor_begin;
        R.ser.push_back(S);
        x_off += ncap;
        row_off += (int64_t)(si.m_max - si.m_min + 1) * ncap;
    }
    R.total_samples = x_off;
    R.total_cells = row_off;
    if (R.total_items >= 0xFFFFFFFFll || R.total_buckets >= 0xFFFFFFFEll || R.total_windows >= 0xFFFFFFFFll)
        return PANACHE_EBUDGET;
    // device footprint: resident arrays plus the largest transient (radix sort of the directory)
    size_t b = 0;
    b += (size_t)R.total_samples * (8 + 8 + 16 + 4 + 8);   // x, xs, sq, runlen, staging
    const bool half = (c.flags & PANACHE_FLAG_HALF_FEATURES) != 0;
    b += (size_t)R.total_rows * PN_FEAT * (half ? 2 : 4);   // features
    b += (size_t)R.total_windows * 4;                       // sieve projections
    b += (size_t)R.total_windows * (16 + 16);               // sig, cnt, nclist, qorder, moments
    b += (size_t)R.total_items * 8 * 2;                     // directory + sort scratch
    b += (size_t)R.total_buckets * 4 + (size_t)R.total_items / 4096 * 1024;
    b += (size_t)R.total_cells * 8;                         // profile rows
    b += (size_t)R.anc.size() * (c.B + 1) * PN_FEAT * 4;
    b += (size_t)R.total_chunks * PN_FEAT * 4;               // tensor-core anchors
    b += (size_t)R.anc.size() * 32 * R.a_max * 4;            // their twiddle operand
    R.footprint = b;
    if (c.hbm_budget_bytes && b > c.hbm_budget_bytes) return PANACHE_EBUDGET;
    return PANACHE_OK;
}

PnView make_view(panache_ctx *ctx, PnRequest &R) {
    const panache_config &c = ctx->cfg;
    PnView v;
    memset(&v, 0, sizeof(v));
    v.series = R.d_ser;
    v.anchors = R.d_anc;
    v.levels = R.d_lev;
    v.nseries = (int32_t)R.ser.size();
    v.nanchors = (int32_t)R.anc.size();
    v.nlevels = (int32_t)R.lev.size();
    v.B = (int32_t)c.B;
    v.K = (int32_t)c.K;
    v.C = (int32_t)c.chunk;
    v.cshift = 0;
    while ((1 << v.cshift) < v.C) ++v.cshift;
    v.alpha = (int32_t)c.alpha;
    v.R = (int32_t)(c.gamma * c.alpha);
    v.d0 = (int32_t)c.d0;
    v.probe_cap = (int32_t)c.probe_cap;
    v.beta = (int32_t)c.beta;
    v.lam = (float)c.lambda;
    v.precision = (int32_t)c.precision;
    v.x = R.x;
    v.xs = R.xs;
    v.x1 = R.x1;
    v.sq = R.sq;
    v.shift = R.shift;
    v.runlen = R.runlen;
    v.F = R.F;
    v.Fh = R.Fh;
    v.sproj = R.sproj;
    v.lb_eps = R.Fh ? 4.8828125e-4f : 0.0f;   // round to nearest half: relative error <= 2^-11
    v.sig = R.sig;
    v.cnt = R.cnt;
    v.nclist = R.nclist;
    v.qorder = R.qorder;
    v.wmf = R.wmf;
    v.wmd = R.wmd;
    v.g = R.g;
    v.gT = R.gT;
    v.anc = R.tca;
    v.twb = R.twb;
    v.twb_ld = R.a_max;
    v.err = R.err;
    v.dir_keys = R.dir_keys;
    v.dir_vals = R.dir_vals;
    v.bstart = R.bstart;
    v.prof = R.prof;
    v.stats = R.stats;
    v.kt = ctx->kt.on ? &ctx->kt : nullptr;
    return v;
}

struct GroupSet {
    std::vector<PnSelGroup> g;
    std::vector<int32_t> owner;  // series of each group
};

GroupSet make_groups(const PnRequest &R, int mode, const std::vector<int> &k_of_series) {
    GroupSet gs;
    for (size_t s = 0; s < R.ser.size(); ++s) {
        const PnSeries &S = R.ser[s];
        const int L = S.m_max - S.m_min + 1;
        if (mode == PANACHE_TOPK_GLOBAL) {
            PnSelGroup G;
            memset(&G, 0, sizeof(G));
            G.cell_off = S.row_off;
            G.ncell = (int64_t)L * S.ld;
            G.series = (int32_t)s;
            G.k = k_of_series[s];
            G.need = (uint32_t)((int64_t)G.k * (S.m_max + 1));
            gs.g.push_back(G);
            gs.owner.push_back((int32_t)s);
        } else {
            for (int r = 0; r < L; ++r) {
                PnSelGroup G;
                memset(&G, 0, sizeof(G));
                G.cell_off = S.row_off + (int64_t)r * S.ld;
                G.ncell = S.ld;
                G.series = (int32_t)s;
                G.k = k_of_series[s];
                G.need = (uint32_t)((int64_t)G.k * (S.m_min + r + 1));
                gs.g.push_back(G);
                gs.owner.push_back((int32_t)s);
            }
        }
    }
    return gs;
}

// Sizes the pool (k (m_max + 1) plus slack, capped at 8192 cells; EINVAL
// beyond that when strict) and uploads the groups.
int sel_prepare(PnRequest &R, const GroupSet &gs, bool strict, SelBufs &b) {
    b.ng = (int32_t)gs.g.size();
    if (!b.ng) return PANACHE_OK;
    uint32_t need_max = 0;
    b.kmax = 1;
    for (auto &G : gs.g) {
        need_max = std::max(need_max, G.need);
        b.kmax = std::max(b.kmax, G.k);
    }
    int64_t cap = next_pow2((int64_t)need_max + need_max / 4 + 256);
    if (cap > 8192) {
        if (strict) return PANACHE_EINVAL;
        cap = 8192;
    }
    b.cap = (int32_t)cap;
    PN_CU(R.alloc(b.dg, b.ng));
    PN_CU(R.alloc(b.out, (int64_t)b.ng * b.kmax));
    PN_CU(R.alloc(b.cnt, b.ng));
    PN_CU(cudaMemcpyAsync(b.dg, gs.g.data(), sizeof(PnSelGroup) * b.ng, cudaMemcpyHostToDevice, R.st));
    PN_CU(cudaMemsetAsync(b.cnt, 0, sizeof(int32_t) * b.ng, R.st));
    return PANACHE_OK;
}

// Enqueues one selection of `b` (its kernels honour v.gate).
int sel_launch(panache_ctx *ctx, PnRequest &R, const PnView &v, const SelBufs &b, int *overflow) {
    if (!b.ng) return PANACHE_OK;
    pn_kt_begin(v.kt, PN_KT_SELECT, R.st);
    PN_CU(pn::launch_select(v, b.dg, b.ng, 0, R.total_cells, b.cap, ctx->cfg.eps0, b.kmax, b.out, b.cnt, overflow,
                            ctx->sm_count * 8, R.st));
    pn_kt_end(v.kt, PN_KT_SELECT, R.st);
    ctx->launches += 10;
    return PANACHE_OK;
}

constexpr int kRefinePasses = 8;   // most row-refinement passes of one request

__global__ void k_fill_i32(int32_t *p, int32_t n, int32_t value) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) p[t] = value;
}

// CUDA events between the steps of a request (PANACHE_FLAG_TIMING).
struct StepTimer {
    bool on = false;
    cudaEvent_t ev[9] = {};
    cudaStream_t st = nullptr;
    ~StepTimer() {
        for (auto e : ev)
            if (e) cudaEventDestroy(e);
    }
    int start(bool enable, cudaStream_t s) {
        on = enable;
        st = s;
        if (!on) return PANACHE_OK;
        for (auto &e : ev) PN_CU(cudaEventCreate(&e));
        return mark(0);
    }
    int mark(int i) { return on ? from_cuda(cudaEventRecord(ev[i], st)) : PANACHE_OK; }
    int read(double *ms) {
        if (!on) return PANACHE_OK;
        PN_CU(cudaEventSynchronize(ev[8]));
        for (int i = 0; i < 8; ++i) {
            float t = 0.0f;
            PN_CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
            ms[i] = t;
        }
        return PANACHE_OK;
    }
};

// Device buffers of a planned request (or of a resident stream), its tables,
// projections and initial state: profile rows unset, counters and error word zero.
int alloc_state(panache_ctx *ctx, PnRequest &R, bool want_x1, bool full_tables, bool emit_only = false) {
    const panache_config &c = ctx->cfg;
    cudaStream_t st = R.st;
    const int64_t nser = (int64_t)R.ser.size(), nanc = emit_only ? 0 : (int64_t)R.anc.size();
    if (emit_only) {
        // the emit stage alone reads samples, prefix sums, run lengths and rows
        PN_CU(R.alloc(R.d_ser, nser));
        PN_CU(R.alloc(R.x, R.total_samples));
        PN_CU(R.alloc(R.xs, R.total_samples + PN_SAMPLE_PAD));
        if (want_x1) PN_CU(R.alloc(R.x1, R.total_samples + PN_SAMPLE_PAD));
        PN_CU(R.alloc(R.sq, R.total_samples + nser));
        PN_CU(cudaMemsetAsync(R.xs + R.total_samples, 0, sizeof(float2) * PN_SAMPLE_PAD, st));
        if (want_x1) PN_CU(cudaMemsetAsync(R.x1 + R.total_samples, 0, sizeof(float) * PN_SAMPLE_PAD, st));
        PN_CU(R.alloc(R.shift, nser));
        PN_CU(R.alloc(R.runlen, R.total_samples));
        PN_CU(R.alloc(R.prof, R.total_cells));
        PN_CU(R.alloc(R.stats, PN_ST_COUNT));
        PN_CU(R.alloc(R.flagbuf, 4));
        PN_CU(R.alloc(R.err, 1));
        PN_CU(cudaMemcpyAsync(R.d_ser, R.ser.data(), sizeof(PnSeries) * nser, cudaMemcpyHostToDevice, st));
        PN_CU(cudaMemsetAsync(R.stats, 0, sizeof(unsigned long long) * PN_ST_COUNT, st));
        PN_CU(cudaMemsetAsync(R.err, 0, sizeof(int), st));
        return PANACHE_OK;
    }
    PN_CU(R.alloc(R.d_ser, nser));
    PN_CU(R.alloc(R.d_anc, nanc));
    PN_CU(R.alloc(R.d_lev, (int64_t)R.lev.size()));
    PN_CU(R.alloc(R.d_slot_off, nanc));
    PN_CU(R.alloc(R.x, R.total_samples));
    PN_CU(R.alloc(R.xs, R.total_samples + PN_SAMPLE_PAD));
    if (want_x1) PN_CU(R.alloc(R.x1, R.total_samples + PN_SAMPLE_PAD));
    PN_CU(R.alloc(R.sq, R.total_samples + nser));
    PN_CU(cudaMemsetAsync(R.xs + R.total_samples, 0, sizeof(float2) * PN_SAMPLE_PAD, st));
    if (want_x1) PN_CU(cudaMemsetAsync(R.x1 + R.total_samples, 0, sizeof(float) * PN_SAMPLE_PAD, st));
    PN_CU(R.alloc(R.shift, nser));
    PN_CU(R.alloc(R.runlen, R.total_samples));
    if (c.flags & PANACHE_FLAG_HALF_FEATURES) PN_CU(R.alloc(R.Fh, R.total_rows * PN_FEAT));
    else PN_CU(R.alloc(R.F, R.total_rows * PN_FEAT));
    PN_CU(R.alloc(R.sproj, R.total_windows));
    PN_CU(R.alloc(R.sig, R.total_windows));
    PN_CU(R.alloc(R.cnt, R.total_windows));
    PN_CU(R.alloc(R.nclist, R.total_windows));
    PN_CU(R.alloc(R.qorder, R.total_windows));
    if (c.precision == PANACHE_PLAIN_FP64) PN_CU(R.alloc(R.wmd, R.total_windows));
    else PN_CU(R.alloc(R.wmf, R.total_windows));
    PN_CU(R.alloc(R.g, nanc * (c.B + 1) * PN_FEAT));
    PN_CU(R.alloc(R.gT, nanc * PN_FEAT * 32));
    PN_CU(R.alloc(R.dir_keys, R.total_items));
    PN_CU(R.alloc(R.dir_vals, R.total_items));
    PN_CU(R.alloc(R.bstart, R.total_buckets + 1));
    PN_CU(R.alloc(R.prof, R.total_cells));
    PN_CU(R.alloc(R.stats, PN_ST_COUNT));
    PN_CU(R.alloc(R.flagbuf, 4));
    PN_CU(R.alloc(R.err, 1));
    const bool tc_anchors = c.precision == PANACHE_MIXED && !(c.flags & PANACHE_FLAG_FP64_ANCHORS);
    if (tc_anchors) {
        PN_CU(R.alloc(R.tca, R.total_chunks * PN_FEAT));
        PN_CU(R.alloc(R.twb, nanc * 32 * (int64_t)std::max(1, R.a_max)));
    }
    if (full_tables) {
        PN_CU(R.alloc(R.d_blk_anchor, (int64_t)R.blk_anchor.size()));
        PN_CU(R.alloc(R.d_blk_chunk0, (int64_t)R.blk_chunk0.size()));
        if (tc_anchors) {
            PN_CU(R.alloc(R.d_tile_anchor, (int64_t)R.tile_anchor.size()));
            PN_CU(R.alloc(R.d_tile_row0, (int64_t)R.tile_row0.size()));
        }
    }
    std::vector<float> hg((size_t)nanc * (c.B + 1) * PN_FEAT);
    for (int64_t a = 0; a < nanc; ++a) {
        const std::vector<float> &g = ctx->proj(R.anc[a].a);
        std::copy(g.begin(), g.end(), hg.begin() + a * (c.B + 1) * PN_FEAT);
    }
    // transposed copy: element (t, l) = dimension t of projection l, so that
    // lane l of a warp reads its projection's dimensions with coalesced loads
    std::vector<float> hgT((size_t)nanc * PN_FEAT * 32, 0.0f);
    for (int64_t a = 0; a < nanc; ++a)
        for (int l = 0; l <= (int)c.B; ++l)
            for (int t = 0; t < PN_FEAT; ++t)
                hgT[(a * PN_FEAT + t) * 32 + l] = hg[(a * (c.B + 1) + l) * PN_FEAT + t];
    PN_CU(cudaMemcpyAsync(R.d_ser, R.ser.data(), sizeof(PnSeries) * nser, cudaMemcpyHostToDevice, st));
    if (nanc) {
        PN_CU(cudaMemcpyAsync(R.d_anc, R.anc.data(), sizeof(PnAnchor) * nanc, cudaMemcpyHostToDevice, st));
        PN_CU(cudaMemcpyAsync(R.d_lev, R.lev.data(), sizeof(PnLevel) * R.lev.size(), cudaMemcpyHostToDevice, st));
        PN_CU(cudaMemcpyAsync(R.d_slot_off, R.slot_off.data(), 8 * nanc, cudaMemcpyHostToDevice, st));
        if (full_tables) {
            PN_CU(cudaMemcpyAsync(R.d_blk_anchor, R.blk_anchor.data(), 4 * R.blk_anchor.size(),
                                  cudaMemcpyHostToDevice, st));
            PN_CU(cudaMemcpyAsync(R.d_blk_chunk0, R.blk_chunk0.data(), 4 * R.blk_chunk0.size(),
                                  cudaMemcpyHostToDevice, st));
            if (tc_anchors) {
                PN_CU(cudaMemcpyAsync(R.d_tile_anchor, R.tile_anchor.data(), 4 * R.tile_anchor.size(),
                                      cudaMemcpyHostToDevice, st));
                PN_CU(cudaMemcpyAsync(R.d_tile_row0, R.tile_row0.data(), 4 * R.tile_row0.size(),
                                      cudaMemcpyHostToDevice, st));
            }
        }
        PN_CU(cudaMemcpyAsync(R.g, hg.data(), 4 * hg.size(), cudaMemcpyHostToDevice, st));
        PN_CU(cudaMemcpyAsync(R.gT, hgT.data(), 4 * hgT.size(), cudaMemcpyHostToDevice, st));
    }
    if (tc_anchors && nanc) {
        PN_CU(pn::launch_twiddles(R.d_anc, (int32_t)nanc, R.a_max, R.twb, st));
        ctx->launches += 1;
    }
    PN_CU(cudaMemsetAsync(R.prof, 0xFF, sizeof(unsigned long long) * std::max<int64_t>(1, R.total_cells), st));
    PN_CU(cudaMemsetAsync(R.stats, 0, sizeof(unsigned long long) * PN_ST_COUNT, st));
    PN_CU(cudaMemsetAsync(R.err, 0, sizeof(int), st));
    return PANACHE_OK;
}

// Buffers and uploads of the emit stage after the sieve (no launches).
int emit_prepare(panache_ctx *ctx, PnRequest &R, const GroupSet &seed_groups, const GroupSet &ref_groups,
                 const GroupSet &out_groups, EmitPlan &E) {
    const panache_config &c = ctx->cfg;
    PN_CU(R.alloc(E.ctl, C_WORDS));
    E.completion = !(c.flags & PANACHE_FLAG_NO_COMPLETION) && c.rounds > 0;
    E.refine = !(c.flags & PANACHE_FLAG_NO_REFINE);
    if (E.completion) {
        PN_TRY(sel_prepare(R, seed_groups, false, E.sb));
        if (E.sb.ng) PN_CU(R.alloc(E.dseeds, (int64_t)E.sb.ng * E.sb.kmax));
    }
    if (E.refine) {
        PN_TRY(sel_prepare(R, ref_groups, false, E.rb));
        if (E.rb.ng) {
            E.done_cap = E.rb.kmax * kRefinePasses;
            PN_CU(R.alloc(E.dtg, (int64_t)E.rb.ng * E.rb.kmax));
            if (E.completion) PN_CU(R.alloc(E.dnear, (int64_t)E.rb.ng * E.rb.kmax));
            // global lists: the completion seeds' count (seed_mult k); per-length
            // lists: k per length
            E.knear = c.topk_mode == PANACHE_TOPK_GLOBAL && E.completion && E.sb.ng
                          ? E.sb.kmax
                          : (int32_t)std::max<int64_t>(1, E.rb.kmax / std::max<uint32_t>(1, c.refine_mult));
            PN_CU(R.alloc(E.ddone, (int64_t)E.rb.ng * E.done_cap));
            PN_CU(R.alloc(E.ndone, E.rb.ng));
        }
        for (auto &S : R.ser) {
            E.max_windows = std::max<int64_t>(E.max_windows, S.n - S.m_min + 1);
            E.m_top = std::max(E.m_top, (int)S.m_max);
        }
    }
    PN_TRY(sel_prepare(R, out_groups, true, E.fb));
    return PANACHE_OK;
}

// Every launch of the emit stage after the sieve, with the results copied
// to the pinned host buffers: no host wait, so it can be captured.
// Algorithm 2's rounds are driven on the device: every round is enqueued,
// and a gate word in device memory closes the remaining rounds once the
// seeds run out or nothing improves.  Control words: 0-3 completion (gate,
// improved, seeds, rounds run), 4-7 refinement (gate, improved, targets,
// passes run), 8 the final selection's pool overflow, 9 the others'
// (ignored).
// With `batch` > 0 (not while capturing) the rounds are enqueued `batch` at
// a time and the host reads the gate between batches, so a request whose
// rounds end early does not launch the rest.
int gate_open(cudaStream_t st, const int32_t *gate, int32_t *host, bool *open) {
    PN_CU(cudaMemcpyAsync(host, gate, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    PN_CU(cudaStreamSynchronize(st));
    *open = *host != 0;
    return PANACHE_OK;
}

int emit_launch(panache_ctx *ctx, PnRequest &R, const PnView &v, StepTimer &tm, EmitPlan &E, PnPick *hout,
                int32_t *hcnt, int32_t *hctl, int batch) {
    const panache_config &c = ctx->cfg;
    cudaStream_t st = R.st;
    const int grid = ctx->sm_count * (int)c.grid_mult;
    int32_t *ctl = E.ctl;
    PN_CU(cudaMemsetAsync(ctl, 0, sizeof(int32_t) * C_WORDS, st));
    if (E.completion && E.sb.ng) {
        const int32_t nmax = E.sb.ng * E.sb.kmax;
        k_fill_i32<<<1, 32, 0, st>>>(ctl + C_GATE, 1, 1);
        PnView vg = v;
        vg.gate = ctl + C_GATE;
        for (uint32_t round = 0; round < c.rounds; ++round) {
            if (batch > 0 && round > 0 && round % batch == 0) {
                bool open = true;
                PN_TRY(gate_open(st, ctl + C_GATE, hctl + C_GATE, &open));
                if (!open) break;
            }
            PN_TRY(sel_launch(ctx, R, vg, E.sb, ctl + OV_OTHER));
            PN_CU(pn::launch_picks_to_seeds(E.sb.out, E.sb.cnt, E.sb.ng, E.sb.kmax, E.dseeds, ctl + C_NSEED,
                                            ctl + C_GATE, st));
            pn_kt_begin(v.kt, PN_KT_COMPLETE, st);
            PN_CU(pn::launch_complete(vg, E.dseeds, nmax, ctl + C_NSEED, (int)c.dm, (int)c.dp, ctl + C_FLAG, grid, st));
            pn_kt_end(v.kt, PN_KT_COMPLETE, st);
            PN_CU(pn::launch_round_end(ctl + C_GATE, ctl + C_FLAG, ctl + C_NSEED, ctl + C_ROUNDS, st));
            ctx->launches += 3;
        }
    }
    // Exact row refinement of the top list (refine.cu): the top
    // refine_mult*k cells of every selection group are each scanned against
    // all valid partners at their length; the list is reselected and cells
    // not scanned before are scanned, until a pass finds no new cell or
    // lowers none.  The final top-k is a prefix of that list (the same
    // greedy rule), so every reported cell ends with its exact nearest
    // neighbour.  Each pass then completes around the refined pairs of its
    // targets among the first k picks of their group (partners read back from
    // the cells): a row brought into the list by its exact neighbour has a box
    // no completion round has seen, and a cell that box lowers enters the next
    // pass's list.
    if (E.refine && E.rb.ng) {
        const int32_t nmax = E.rb.ng * E.rb.kmax;
        PN_CU(cudaMemsetAsync(E.ndone, 0, sizeof(int32_t) * E.rb.ng, st));
        k_fill_i32<<<1, 32, 0, st>>>(ctl + R_GATE, 1, 1);
        PnView vr = v;
        vr.gate = ctl + R_GATE;
        for (int pass = 0; pass < kRefinePasses; ++pass) {
            if (batch > 0 && pass > 0 && pass % batch == 0) {
                bool open = true;
                PN_TRY(gate_open(st, ctl + R_GATE, hctl + R_GATE, &open));
                if (!open) break;
            }
            PN_TRY(sel_launch(ctx, R, vr, E.rb, ctl + OV_OTHER));
            PN_CU(pn::launch_new_targets(E.rb.out, E.rb.cnt, E.rb.ng, E.rb.kmax, E.ddone, E.ndone, E.done_cap, E.dtg,
                                         ctl + R_NTG, ctl + R_GATE, st, E.completion ? E.dnear : nullptr,
                                         ctl + R_NNEAR, E.knear));
            pn_kt_begin(v.kt, PN_KT_REFINE, st);
            PN_CU(pn::launch_refine(vr, E.dtg, nmax, ctl + R_NTG, E.max_windows, E.m_top, ctl + R_FLAG,
                                    ctx->sm_count * 2, st));
            pn_kt_end(v.kt, PN_KT_REFINE, st);
            if (E.completion) {
                PN_CU(pn::launch_seeds_refresh(vr, E.dnear, nmax, ctl + R_NNEAR, st));
                pn_kt_begin(v.kt, PN_KT_COMPLETE, st);
                PN_CU(pn::launch_complete(vr, E.dnear, nmax, ctl + R_NNEAR, (int)c.dm, (int)c.dp, ctl + R_FLAG, grid,
                                          st));
                pn_kt_end(v.kt, PN_KT_COMPLETE, st);
                ctx->launches += 2;
            }
            PN_CU(pn::launch_round_end(ctl + R_GATE, ctl + R_FLAG, ctl + R_NTG, ctl + R_PASSES, st, ctl + R_NNEAR));
            ctx->launches += 3;
        }
    }
    PN_TRY(tm.mark(7));
    PN_TRY(sel_launch(ctx, R, v, E.fb, ctl + OV_FINAL));
    if (E.fb.ng) {
        PN_CU(cudaMemcpyAsync(hout, E.fb.out, sizeof(PnPick) * (size_t)E.fb.ng * E.fb.kmax, cudaMemcpyDeviceToHost,
                              st));
        PN_CU(cudaMemcpyAsync(hcnt, E.fb.cnt, sizeof(int32_t) * E.fb.ng, cudaMemcpyDeviceToHost, st));
    }
    PN_CU(cudaMemcpyAsync(hctl, ctl, sizeof(int32_t) * C_WORDS, cudaMemcpyDeviceToHost, st));
    return PANACHE_OK;
}

enum { PN_EMIT_SIEVE = 1, PN_EMIT_REST = 2, PN_EMIT_ALL = 3 };

int read_counters(panache_ctx *ctx, PnRequest &R) {
    unsigned long long hs[PN_ST_COUNT];
    int herr = 0;
    PN_CU(cudaMemcpyAsync(hs, R.stats, sizeof(hs), cudaMemcpyDeviceToHost, R.st));
    PN_CU(cudaMemcpyAsync(&herr, R.err, sizeof(int), cudaMemcpyDeviceToHost, R.st));
    PN_CU(cudaStreamSynchronize(R.st));
    if (herr) return PANACHE_ETIMEOUT;
    ctx->stats.queries = hs[PN_ST_QUERIES];
    ctx->stats.candidates = hs[PN_ST_CANDIDATES];
    ctx->stats.exact_stream = hs[PN_ST_LB_PASSED];
    ctx->stats.exact_sieve = hs[PN_ST_EXACT_SIEVE];
    ctx->stats.exact_completion = hs[PN_ST_EXACT_COMPLETION];
    ctx->stats.exact_refine = hs[PN_ST_EXACT_REFINE];
    ctx->stats.kernel_launches = ctx->launches;
    ctx->stats.waves = 1;
    return PANACHE_OK;
}

int run_emit(panache_ctx *ctx, PnRequest &R, const PnView &v, StepTimer &tm,
             std::vector<std::vector<panache_motif>> &res, int stages = PN_EMIT_ALL) {
    const panache_config &c = ctx->cfg;
    cudaStream_t st = R.st;
    const int64_t nser = (int64_t)R.ser.size();
    const int grid = ctx->sm_count * (int)c.grid_mult;
    int32_t ncls = 0;
    if ((stages & PN_EMIT_SIEVE) && !(c.flags & PANACHE_FLAG_NO_SIEVE)) {
        // exhaustive sieve: 1 with the tensor-core Gram filter, 2 every pair exactly
        const int exhaustive = !(c.flags & PANACHE_FLAG_EXHAUSTIVE_SIEVE) ? 0
                               : (c.flags & PANACHE_FLAG_SIEVE_GRAM) ? 1 : 2;
        PN_CU(pn::launch_sieve(v, R.d_slot_off, R.total_slots, (int)c.sieve_w, exhaustive, grid, R.a_max, st,
                               &ncls));
        ctx->launches += 6 + (ncls ? 4 + 2 * 12 : 0);
    }
    ctx->stats.hot_classes = (uint64_t)ncls;
    if (!(stages & PN_EMIT_REST)) {
        for (int t = 6; t <= 8; ++t) PN_TRY(tm.mark(t));
        PN_TRY(tm.read(ctx->stats.step_ms));
        ctx->kt.collect();
        res.assign(nser, {});
        return read_counters(ctx, R);
    }
    PN_TRY(tm.mark(6));
    // seeds and refinement targets per group, capped so that k (m_max + 1)
    // stays within the selection pool
    std::vector<int> kser(nser), kseed(nser), kref(nser);
    for (int64_t s = 0; s < nser; ++s) {
        kser[s] = R.ser[s].k;
        const int64_t cap = 6000 / (R.ser[s].m_max + 1);
        kseed[s] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c.seed_mult * R.ser[s].k, cap));
        kref[s] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)c.refine_mult * R.ser[s].k, cap));
    }
    const GroupSet out_groups = make_groups(R, (int)c.topk_mode, kser);
    // Seeds: the top-kseed cells in the output's mode.  In per-length mode
    // this already holds the global top-kseed: suppression acts within one
    // length, so the global greedy list restricted to a length is a
    // prefix of that length's own greedy list, and no length contributes
    // more than kseed cells to it.
    const GroupSet seed_mode = make_groups(R, (int)c.topk_mode, kseed);
    // The rest of Algorithm 2 (completion rounds, the row refinement, the
    // final selection) runs without the host: buffers first, then the
    // launches, replayed from a captured graph when the request's shape
    // repeats, then one wait for the results.
    const bool gram_ok = c.precision == PANACHE_MIXED && !(c.flags & PANACHE_FLAG_NO_SIEVE) &&
                         pn::sieve_gram_supported(R.a_max);
    // the top-k sieves need the request's own directories (not rows handed
    // in from other ranks); the focused one runs for global requests unless
    // turned off
    const bool own_dirs = (stages & PN_EMIT_SIEVE) != 0;
    const bool topk_sieve = (c.flags & PANACHE_FLAG_TOPK_SIEVE) && gram_ok && own_dirs;
    const bool focus_sieve = !topk_sieve && !(c.flags & PANACHE_FLAG_NO_FOCUS_SIEVE) && c.topk_mode == 0 && gram_ok &&
                             own_dirs;
    const bool graph = (c.flags & PANACHE_FLAG_GRAPH) && !(c.flags & (PANACHE_FLAG_TIMING | PANACHE_FLAG_INDEX_ONLY)) &&
                       ctx->last == &R && !topk_sieve;
    if (!R.emit || !graph) {
        delete R.emit;
        R.emit = new (std::nothrow) EmitPlan();
        if (!R.emit) return PANACHE_ENOMEM;
        PN_TRY(emit_prepare(ctx, R, seed_mode, make_groups(R, (int)c.topk_mode, kref), out_groups, *R.emit));
    }
    EmitPlan &E = *R.emit;
    const size_t out_bytes = sizeof(PnPick) * (size_t)E.fb.ng * E.fb.kmax;
    const size_t pin_bytes = out_bytes + sizeof(int32_t) * ((size_t)E.fb.ng + C_WORDS);
    void *pin = nullptr;
    if (graph) {
        // the captured copies write to a buffer of the plan's own, which
        // lives as long as the graph
        if (!E.pin && cudaMallocHost(&E.pin, std::max<size_t>(pin_bytes, 64)) != cudaSuccess) return PANACHE_ENOMEM;
        pin = E.pin;
    } else {
        PN_TRY(ctx->pinned(std::max<size_t>(pin_bytes, 64), &pin));
    }
    PnPick *hout = static_cast<PnPick *>(pin);
    int32_t *hcnt = reinterpret_cast<int32_t *>(static_cast<unsigned char *>(pin) + out_bytes);
    int32_t *hctl = hcnt + E.fb.ng;
    if (graph && ctx->gexec_emit) {
        PN_CU(cudaGraphLaunch(ctx->gexec_emit, st));
        ctx->launches += ctx->glaunches_emit;
    } else if (graph) {
        // capture once; later requests of the same shape launch it
        const uint64_t l0 = ctx->launches;
        cudaGraph_t g = nullptr;
        PN_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = emit_launch(ctx, R, v, tm, E, hout, hcnt, hctl, 0);
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (rc == PANACHE_OK) rc = from_cuda(ec);
        if (rc == PANACHE_OK) rc = from_cuda(cudaGraphInstantiate(&ctx->gexec_emit, g, 0));
        if (g) cudaGraphDestroy(g);
        if (rc != PANACHE_OK) {
            ctx->drop_graph();
            return rc;
        }
        ctx->glaunches_emit = ctx->launches - l0;
        PN_CU(cudaGraphLaunch(ctx->gexec_emit, st));
    } else {
        PN_TRY(emit_launch(ctx, R, v, tm, E, hout, hcnt, hctl, 2));
    }
    PN_CU(cudaStreamSynchronize(st));
    if (hctl[OV_FINAL]) return PANACHE_EPOOL;
    if (topk_sieve || focus_sieve) {
        // The top-k sieve: every hot class's pairs estimated on the tensor
        // cores against the largest distance of the refined lists (the
        // reported lists when there is no refinement), the pairs that can
        // enter a list evaluated exactly, then the rest of the emit stage
        // once more on the lowered cells.  Focused: only the classes that
        // hold a window of a listed cell, at the anchors next to its length.
        const SelBufs &lb = E.refine && E.rb.ng ? E.rb : E.fb;
        std::vector<PnPick> lp((size_t)lb.ng * lb.kmax);
        std::vector<int32_t> lc((size_t)lb.ng);
        if (lb.ng) {
            PN_CU(cudaMemcpyAsync(lp.data(), lb.out, sizeof(PnPick) * lp.size(), cudaMemcpyDeviceToHost, st));
            PN_CU(cudaMemcpyAsync(lc.data(), lb.cnt, sizeof(int32_t) * lc.size(), cudaMemcpyDeviceToHost, st));
            PN_CU(cudaStreamSynchronize(st));
        }
        // each anchor's threshold: the largest last distance of the lists that
        // can take its pairs (a global list: every anchor of its series; a
        // per-length list: the anchors next to its length); a short list
        // takes any pair (no threshold)
        auto next_anchors = [&](const PnSeries &S, int m, int &below, int &above) {
            below = above = -1;
            for (int32_t k = S.anchor_begin; k < S.anchor_begin + S.anchor_count; ++k) {
                const int a = R.anc[k].a;
                if (a <= m && (below < 0 || a > R.anc[below].a)) below = k;
                if (a >= m && (above < 0 || a < R.anc[above].a)) above = k;
            }
        };
        std::vector<float> thr(R.anc.size(), 0.0f);
        for (int32_t gi = 0; gi < lb.ng; ++gi) {
            if (lc[gi] <= 0) continue;
            const PnPick &last = lp[(size_t)gi * lb.kmax + lc[gi] - 1];
            const float t = lc[gi] < lb.kmax ? std::numeric_limits<float>::max() : (float)last.d;
            const PnSeries &S = R.ser[last.series];
            if (S.mode == 0) {
                for (int32_t k = S.anchor_begin; k < S.anchor_begin + S.anchor_count; ++k) thr[k] = std::max(thr[k], t);
            } else {
                int below, above;
                next_anchors(S, last.m, below, above);
                if (below >= 0) thr[below] = std::max(thr[below], t);
                if (above >= 0) thr[above] = std::max(thr[above], t);
            }
        }
        // focused: the anchors next to the length of every listed cell (the
        // largest anchor length <= m and the smallest >= m of its series)
        std::vector<uint32_t> fa;
        if (focus_sieve) {
            fa.assign(R.anc.size(), 0u);
            for (int32_t gi = 0; gi < lb.ng; ++gi) {
                for (int32_t t = 0; t < lc[gi]; ++t) {
                    const PnPick &pk = lp[(size_t)gi * lb.kmax + t];
                    int below, above;
                    next_anchors(R.ser[pk.series], pk.m, below, above);
                    if (below >= 0) fa[below] = 1u;
                    if (above >= 0) fa[above] = 1u;
                }
            }
        }
        uint32_t *dfa = nullptr;
        float *dthr = nullptr;
        if (!fa.empty()) {
            PN_CU(cudaMallocAsync((void **)&dfa, sizeof(uint32_t) * fa.size(), st));
            PN_CU(cudaMemcpyAsync(dfa, fa.data(), sizeof(uint32_t) * fa.size(), cudaMemcpyHostToDevice, st));
        }
        PN_CU(cudaMallocAsync((void **)&dthr, sizeof(float) * thr.size(), st));
        PN_CU(cudaMemcpyAsync(dthr, thr.data(), sizeof(float) * thr.size(), cudaMemcpyHostToDevice, st));
        int32_t ncls2 = 0;
        int improved = 0;
        const cudaError_t es = pn::launch_sieve(v, R.d_slot_off, R.total_slots, (int)c.sieve_w, 0, grid, R.a_max, st,
                                                &ncls2, dthr, dfa, &improved);
        if (dfa) cudaFreeAsync(dfa, st);
        cudaFreeAsync(dthr, st);
        PN_CU(es);
        ctx->launches += 6 + (ncls2 ? 4 + 2 * 12 + 6 : 0);
        if (improved) {
            // the rest of the emit stage once more, on the lowered cells
            PN_TRY(emit_launch(ctx, R, v, tm, E, hout, hcnt, hctl, 2));
            PN_CU(cudaStreamSynchronize(st));
            if (hctl[OV_FINAL]) return PANACHE_EPOOL;
        }
    }
    ctx->stats.completion_rounds = (uint64_t)hctl[C_ROUNDS];
    ctx->stats.refine_passes = (uint64_t)hctl[R_PASSES];
    const SelBufs &fb = E.fb;
    std::vector<std::vector<PnPick>> picks(fb.ng);
    for (int32_t gi = 0; gi < fb.ng; ++gi)
        picks[gi].assign(hout + (size_t)gi * fb.kmax, hout + (size_t)gi * fb.kmax + hcnt[gi]);
    PN_TRY(tm.mark(8));
    PN_TRY(tm.read(ctx->stats.step_ms));
    ctx->kt.collect();
    res.assign(nser, {});
    for (size_t gi = 0; gi < picks.size(); ++gi) {
        for (auto &p : picks[gi]) {
            panache_motif mo;
            mo.m = p.m;
            mo._pad = 0;
            mo.i = p.i;
            mo.j = p.j;
            mo.d = p.d;
            res[out_groups.owner[gi]].push_back(mo);
        }
    }
    return read_counters(ctx, R);
}

bool same_shape(const std::vector<SeriesIn> &a, const std::vector<SeriesIn> &b) {
    if (a.size() != b.size()) return false;
    for (size_t s = 0; s < a.size(); ++s) {
        if (a[s].n != b[s].n || (a[s].dtype & 0xFF) != (b[s].dtype & 0xFF) || a[s].m_min != b[s].m_min ||
            a[s].m_max != b[s].m_max || a[s].k != b[s].k || a[s].excl != b[s].excl)
            return false;
    }
    return true;
}

// Copies every series of `in` into the persistent staging buffer of the
// captured graph (host or device sources; the graph reads fixed addresses).
int stage_inputs(panache_ctx *ctx, const std::vector<SeriesIn> &in) {
    for (size_t s = 0; s < in.size(); ++s) {
        const size_t es = (in[s].dtype & 0xFF) == PANACHE_F32 ? 4 : 8;
        if (!in[s].n) continue;
        const cudaMemcpyKind kind = (in[s].dtype & PANACHE_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        PN_CU(cudaMemcpyAsync(ctx->gstage + ctx->gstage_off[s], in[s].ptr, (size_t)in[s].n * es, kind, ctx->st));
    }
    return PANACHE_OK;
}

// The tensor-core Gram search when asked for and supported (mixed form,
// anchors of at most 192 samples, R <= 128, no warm start).
bool use_gram_search(const panache_ctx *ctx, const PnView &v, int a_max) {
    const uint32_t f = ctx->cfg.flags;
    return (f & PANACHE_FLAG_GRAM_SEARCH) && !(f & PANACHE_FLAG_WARM_START) && pn::search_gram_supported(v, a_max);
}

// The streaming search over the query order (Algorithm 1 phase B): the Gram
// search when `qkeys` (the sorted bucket keys, freed here) is given, else the
// per-query Parseval search.
int run_search(panache_ctx *ctx, const PnView &v, int64_t total, int a_max, cudaStream_t st, uint32_t *qkeys) {
    const panache_config &c = ctx->cfg;
    pn_kt_begin(v.kt, PN_KT_SEARCH, st);
    cudaError_t e;
    if (qkeys) {
        e = pn::launch_search_gram(v, qkeys, total, ctx->sm_count, a_max, st);
        const cudaError_t ef = cudaFreeAsync(qkeys, st);
        if (e == cudaSuccess) e = ef;
        ctx->launches += 7;
    } else {
        e = pn::launch_search(v, total, ctx->sm_count * (int)c.grid_mult, a_max, st,
                              (c.flags & PANACHE_FLAG_WARM_START) != 0);
        ctx->launches += 1 + ((c.flags & PANACHE_FLAG_WARM_START) ? 1 : 0);
    }
    pn_kt_end(v.kt, PN_KT_SEARCH, st);
    PN_CU(e);
    return PANACHE_OK;
}

// Algorithm 1 over every anchor of every series (conversion of the staged
// samples, moments, anchors, features and keys, ranks, directory, query
// order) and the streaming search: the part of a request whose launches
// depend only on its shape.
int index_and_search(panache_ctx *ctx, PnRequest &R, const PnView &v, const PnConv *dcv, int32_t ncv,
                     StepTimer &tm, bool search) {
    cudaStream_t st = R.st;
    if (R.total_samples > 0) {
        k_convert<<<(unsigned)((R.total_samples + 255) / 256), 256, 0, st>>>(dcv, ncv, R.total_samples, R.x, R.xs,
                                                                            R.x1);
        PN_CU(cudaGetLastError());
        ctx->launches += 1;
    }
    PN_TRY(tm.mark(1));
    PN_CU(pn::launch_runlen(v, R.total_samples, st));
    PN_CU(pn::launch_moments(v, R.total_samples, R.sq, st));
    PN_CU(pn::launch_moment_table(v, R.total_windows, st));
    PN_TRY(tm.mark(2));
    if (R.tca) {
        // an injected wait fault never fires into a graph being captured
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        PN_CU(cudaStreamIsCapturing(st, &cs));
        PnView va = v;
        va.tc_fault = (cs == cudaStreamCaptureStatusNone && fault_fires(PANACHE_FAULT_TC_WAIT)) ? 1 : 0;
        pn_kt_begin(v.kt, PN_KT_ANCHOR_TC, st);
        PN_CU(pn::launch_anchor_tc(va, R.d_tile_anchor, R.d_tile_row0, (int32_t)R.tile_anchor.size(), st));
        pn_kt_end(v.kt, PN_KT_ANCHOR_TC, st);
        ctx->launches += 1;
    }
    pn_kt_begin(v.kt, PN_KT_FEATURES, st);
    PN_CU(pn::launch_features(v, R.d_blk_anchor, R.d_blk_chunk0, (int32_t)R.blk_anchor.size(), R.a_max, st));
    pn_kt_end(v.kt, PN_KT_FEATURES, st);
    PN_TRY(tm.mark(3));
    PN_CU(pn::launch_ranks(v, R.total_windows, st));
    PN_CU(pn::launch_directory(v, R.total_items, R.total_buckets, st));
    const bool gram = search && use_gram_search(ctx, v, R.a_max);
    uint32_t *qkeys = nullptr;
    PN_CU(pn::launch_query_order(v, R.total_windows, R.total_buckets, st, nullptr, 0, gram ? &qkeys : nullptr));
    const int mrc = tm.mark(4);
    if (mrc != PANACHE_OK) {
        if (qkeys) cudaFreeAsync(qkeys, st);
        return mrc;
    }
    ctx->launches += 3 + 5 + 1 + 5 + 2 + 4 * 3;
    if (!search) return PANACHE_OK;
    return run_search(ctx, v, R.total_windows, R.a_max, st, qkeys);
}

// The whole path for a list of series; results per series.
int run_request(panache_ctx *ctx, const std::vector<SeriesIn> &in, std::vector<std::vector<panache_motif>> &res,
                const PnShard *sh = nullptr) {
    const panache_config &c = ctx->cfg;
    for (auto &s : in) PN_TRY(check_series(s));
    const bool emit_only = sh && sh->rows_in;
    const bool graph = !sh && (c.flags & PANACHE_FLAG_GRAPH) &&
                       !(c.flags & (PANACHE_FLAG_INDEX_ONLY | PANACHE_FLAG_TIMING));
    if (graph && ctx->gexec && ctx->last && same_shape(ctx->gshape, in)) {
        // replay: new samples into the kept buffers, one graph launch, then Algorithm 2
        memset(&ctx->stats, 0, sizeof(ctx->stats));
        ctx->kt.reset(false);
        ctx->launches = ctx->glaunches;
        PnRequest &R = *ctx->last;
        ctx->stats.device_bytes = R.footprint;
        PN_TRY(stage_inputs(ctx, in));
        PN_CU(cudaGraphLaunch(ctx->gexec, R.st));
        StepTimer tm;
        PN_TRY(tm.start(false, R.st));
        return run_emit(ctx, R, make_view(ctx, R), tm, res);
    }
    ctx->drop_graph();
    delete ctx->last;
    ctx->last = nullptr;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->kt.reset((c.flags & PANACHE_FLAG_TIMING) != 0);
    ctx->launches = 0;
    PnRequest *Rp = new (std::nothrow) PnRequest();
    if (!Rp) return PANACHE_ENOMEM;
    ctx->last = Rp;
    PnRequest &R = *Rp;
    cudaStream_t st = ctx->st;
    R.st = st;
    PN_TRY(plan(ctx->cfg, in, R, nullptr, sh));
    ctx->stats.device_bytes = R.footprint;
    const int64_t nser = (int64_t)R.ser.size();
    bool all_f32 = true;
    for (auto &si : in) all_f32 = all_f32 && (si.dtype & 0xFF) == PANACHE_F32;
    PN_TRY(alloc_state(ctx, R, all_f32 && c.precision == PANACHE_MIXED, true, emit_only));
    StepTimer tm;
    PN_TRY(tm.start((c.flags & PANACHE_FLAG_TIMING) != 0, st));

    // samples: host inputs go through one staging buffer; device inputs are
    // read in place (with the graph, every input is staged at a fixed address)
    std::vector<PnConv> cv(nser);
    int64_t stage_bytes = 0;
    std::vector<int64_t> stage_off(nser, -1);
    for (int64_t s = 0; s < nser; ++s) {
        const int es = (in[s].dtype & 0xFF) == PANACHE_F32 ? 4 : 8;
        if (graph || !(in[s].dtype & PANACHE_DEVICE)) {
            stage_off[s] = stage_bytes;
            stage_bytes += ((in[s].n * es + 15) / 16) * 16;
        }
    }
    unsigned char *stage = nullptr;
    if (stage_bytes) {
        if (graph) PN_CU(R.alloc(stage, stage_bytes));
        else PN_CU(cudaMallocAsync((void **)&stage, stage_bytes, st));
    }
    for (int64_t s = 0; s < nser; ++s) {
        const int es = (in[s].dtype & 0xFF) == PANACHE_F32 ? 4 : 8;
        cv[s].n = in[s].n;
        cv[s].x_off = R.ser[s].x_off;
        cv[s].dtype = in[s].dtype & 0xFF;
        if (stage_off[s] < 0) {
            cv[s].src = in[s].ptr;
        } else {
            cv[s].src = stage + stage_off[s];
            if (in[s].n) {
                const cudaMemcpyKind kind =
                    (in[s].dtype & PANACHE_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
                if (fault_fires(PANACHE_FAULT_COPY)) {          // as if the copy had been refused
                    if (!graph) cudaFreeAsync(stage, st);
                    return PANACHE_ECUDA;
                }
                PN_CU(cudaMemcpyAsync(stage + stage_off[s], in[s].ptr, in[s].n * es, kind, st));
            }
        }
    }
    PnConv *dcv = nullptr;
    PN_CU(R.alloc(dcv, std::max<int64_t>(1, nser)));
    PN_CU(cudaMemcpyAsync(dcv, cv.data(), sizeof(PnConv) * nser, cudaMemcpyHostToDevice, st));
    PnView v = make_view(ctx, R);
    const bool search = !(c.flags & PANACHE_FLAG_INDEX_ONLY);
    if (emit_only) {
        // samples, run lengths and prefix sums; the given rows; then the emit
        // stage after the sieve (each rank sieved its own anchors)
        if (R.total_samples > 0) {
            k_convert<<<(unsigned)((R.total_samples + 255) / 256), 256, 0, st>>>(dcv, (int32_t)nser, R.total_samples,
                                                                                R.x, R.xs, R.x1);
            PN_CU(cudaGetLastError());
        }
        PN_CU(pn::launch_runlen(v, R.total_samples, st));
        PN_CU(pn::launch_moments(v, R.total_samples, R.sq, st));
        ctx->launches += 1 + 3 + 5;
        PN_CU(cudaMemcpyAsync(R.prof, sh->rows_in, sizeof(uint64_t) * (size_t)R.total_cells, cudaMemcpyHostToDevice,
                              st));
        if (stage) cudaFreeAsync(stage, st);
        for (int t = 1; t <= 5; ++t) PN_TRY(tm.mark(t));
        return run_emit(ctx, R, v, tm, res, PN_EMIT_REST);
    }
    if (graph) {
        // capture once; this and every later request of the same shape launch it
        cudaGraph_t g = nullptr;
        PN_CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        int rc = from_cuda(cudaMemsetAsync(R.prof, 0xFF, sizeof(unsigned long long) *
                                                               std::max<int64_t>(1, R.total_cells), st));
        if (rc == PANACHE_OK) rc = from_cuda(cudaMemsetAsync(R.stats, 0, sizeof(unsigned long long) * PN_ST_COUNT, st));
        if (rc == PANACHE_OK) rc = from_cuda(cudaMemsetAsync(R.err, 0, sizeof(int), st));
        StepTimer off;
        if (rc == PANACHE_OK) rc = index_and_search(ctx, R, v, dcv, (int32_t)nser, off, true);
        const cudaError_t ec = cudaStreamEndCapture(st, &g);
        if (rc == PANACHE_OK) rc = from_cuda(ec);
        if (rc == PANACHE_OK) rc = from_cuda(cudaGraphInstantiate(&ctx->gexec, g, 0));
        if (g) cudaGraphDestroy(g);
        if (rc != PANACHE_OK) {
            ctx->drop_graph();
            return rc;
        }
        ctx->gshape = in;
        ctx->gstage = stage;
        ctx->gstage_off = stage_off;
        ctx->glaunches = ctx->launches;
        PN_CU(cudaGraphLaunch(ctx->gexec, st));
    } else {
        int rc = index_and_search(ctx, R, v, dcv, (int32_t)nser, tm, search);
        if (stage) cudaFreeAsync(stage, st);
        PN_TRY(rc);
    }
    if (!search) {
        for (int t = 5; t <= 8; ++t) PN_TRY(tm.mark(t));
        PN_TRY(tm.read(ctx->stats.step_ms));
        ctx->kt.collect();
        int herr = 0;
        PN_CU(cudaMemcpyAsync(&herr, R.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        PN_CU(cudaStreamSynchronize(st));
        if (herr) return PANACHE_ETIMEOUT;
        res.assign(nser, {});
        ctx->stats.kernel_launches = ctx->launches;
        ctx->stats.waves = 1;
        return PANACHE_OK;
    }
    PN_TRY(tm.mark(5));
    if (sh && sh->rows_out) {
        // this rank's rows after its anchors' search and sieve
        PN_TRY(run_emit(ctx, R, v, tm, res, PN_EMIT_SIEVE));
        PN_CU(cudaMemcpyAsync(sh->rows_out, R.prof, sizeof(uint64_t) * (size_t)R.total_cells, cudaMemcpyDeviceToHost,
                              st));
        PN_CU(cudaStreamSynchronize(st));
        return PANACHE_OK;
    }
    return run_emit(ctx, R, v, tm, res);
}

// ---------------------------------------------------------------------------
// Resident streams
// ---------------------------------------------------------------------------

// Fresh resident state for `cap` samples (none present yet).
int stream_alloc(panache_stream *h, int64_t cap, PnRequest *&out) {
    out = nullptr;
    panache_ctx *ctx = h->ctx;
    PnRequest *R = new (std::nothrow) PnRequest();
    if (!R) return PANACHE_ENOMEM;
    R->st = ctx->st;
    static const double none = 0.0;
    std::vector<SeriesIn> in{SeriesIn{&none, PANACHE_F64 | PANACHE_DEVICE, 0, h->m_min, h->m_max, h->k, h->excl}};
    std::vector<int64_t> caps{cap};
    int rc = plan(ctx->cfg, in, *R, &caps);
    if (rc == PANACHE_OK) rc = alloc_state(ctx, *R, false, false);
    if (rc != PANACHE_OK) {
        delete R;
        return rc;
    }
    out = R;
    return PANACHE_OK;
}

// Copies a host table into a stream-ordered temporary of the request's stream.
template <class T>
int upload_tmp(cudaStream_t st, const std::vector<T> &h, T *&d) {
    d = nullptr;
    if (h.empty()) return PANACHE_OK;
    PN_CU(cudaMallocAsync((void **)&d, sizeof(T) * h.size(), st));
    PN_CU(cudaMemcpyAsync(d, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, st));
    return PANACHE_OK;
}

// Searches queries [q_lo[a], q_hi[a]) of every anchor into `v.prof`.
int stream_search(panache_ctx *ctx, PnRequest &R, const PnView &v, const std::vector<int64_t> &q_lo,
                  const std::vector<int64_t> &q_hi) {
    std::vector<PnQRange> rng;
    int64_t total = 0;
    for (size_t ai = 0; ai < R.anc.size(); ++ai) {
        if (q_hi[ai] <= q_lo[ai]) continue;
        rng.push_back(PnQRange{total, q_lo[ai], (int32_t)ai, 0});
        total += q_hi[ai] - q_lo[ai];
    }
    if (!total) return PANACHE_OK;
    PnQRange *drng = nullptr;
    PN_TRY(upload_tmp(R.st, rng, drng));
    uint32_t *qkeys = nullptr;
    const bool gram = use_gram_search(ctx, v, R.a_max);
    PN_CU(pn::launch_query_order(v, total, R.total_buckets, R.st, drng, (int32_t)rng.size(), gram ? &qkeys : nullptr));
    ctx->launches += 1 + 4 * 3;
    const int rc = run_search(ctx, v, total, R.a_max, R.st, qkeys);
    PN_CU(cudaFreeAsync(drng, R.st));
    return rc;
}

// Brings the resident index up to the samples present: moments, features of
// the chunks that gained windows, ranks, directory, and the search of every
// query whose batch of beta samples is now complete (its population, and so
// its level and candidates, can no longer change).
int stream_advance(panache_stream *h) {
    panache_ctx *ctx = h->ctx;
    const panache_config &c = ctx->cfg;
    PnRequest &R = *h->R;
    cudaStream_t st = R.st;
    const int64_t n = h->len;
    const int C = (int)c.chunk;
    R.ser[0].n = n;
    for (auto &A : R.anc) A.nw = std::max<int64_t>(0, n - A.a + 1);
    PN_CU(cudaMemcpyAsync(R.d_ser, R.ser.data(), sizeof(PnSeries), cudaMemcpyHostToDevice, st));
    PN_CU(cudaMemcpyAsync(R.d_anc, R.anc.data(), sizeof(PnAnchor) * R.anc.size(), cudaMemcpyHostToDevice, st));
    PN_CU(cudaMemsetAsync(R.stats, 0, sizeof(unsigned long long) * PN_ST_COUNT, st));
    ctx->kt.reset(false);
    PnView v = make_view(ctx, R);
    PN_CU(pn::launch_runlen(v, n, st));
    PN_CU(pn::launch_moments(v, n, R.sq, st));
    PN_CU(pn::launch_moment_table(v, R.total_windows, st));
    std::vector<int32_t> ba, bc, ta, tc;
    for (size_t ai = 0; ai < R.anc.size(); ++ai) {
        const PnAnchor &A = R.anc[ai];
        const int64_t c_lo = h->nw_feat[ai] / C, c_hi = (A.nw + C - 1) / C;
        for (int64_t b = c_lo; b < c_hi; b += PN_FT_CHUNKS) {
            ba.push_back((int32_t)ai);
            bc.push_back((int32_t)b);
        }
        // tensor-core tiles keep the request's 128-chunk alignment
        for (int64_t b = c_lo / 128 * 128; b < c_hi; b += 128) {
            ta.push_back((int32_t)ai);
            tc.push_back((int32_t)b);
        }
    }
    if (!ba.empty()) {
        int32_t *dba = nullptr, *dbc = nullptr, *dta = nullptr, *dtc = nullptr;
        PN_TRY(upload_tmp(st, ba, dba));
        PN_TRY(upload_tmp(st, bc, dbc));
        if (R.tca) {
            PN_TRY(upload_tmp(st, ta, dta));
            PN_TRY(upload_tmp(st, tc, dtc));
            PN_CU(pn::launch_anchor_tc(v, dta, dtc, (int32_t)ta.size(), st));
            PN_CU(cudaFreeAsync(dta, st));
            PN_CU(cudaFreeAsync(dtc, st));
            ctx->launches += 1;
        }
        PN_CU(pn::launch_features(v, dba, dbc, (int32_t)ba.size(), R.a_max, st));
        PN_CU(cudaFreeAsync(dba, st));
        PN_CU(cudaFreeAsync(dbc, st));
    }
    for (size_t ai = 0; ai < R.anc.size(); ++ai) h->nw_feat[ai] = R.anc[ai].nw;
    PN_CU(pn::launch_ranks(v, R.total_windows, st));
    PN_CU(pn::launch_directory(v, R.total_items, R.total_buckets, st));
    ctx->launches += 3 + 5 + 1 + 5 + 2 + 4 * 3;
    const int beta = (c.beta > 0 && (int)c.beta < h->excl) ? (int)c.beta : h->excl;
    const int64_t nb = n / beta * beta;                // samples of complete batches
    std::vector<int64_t> q_ready(R.anc.size());
    for (size_t ai = 0; ai < R.anc.size(); ++ai) {
        const PnAnchor &A = R.anc[ai];
        q_ready[ai] = std::max(h->q_done[ai], std::min<int64_t>(A.nw, std::max<int64_t>(0, nb - A.a + 1)));
    }
    PN_TRY(stream_search(ctx, R, v, h->q_done, q_ready));
    h->q_done = q_ready;
    unsigned long long hs[PN_ST_COUNT];
    int herr = 0;
    PN_CU(cudaMemcpyAsync(hs, R.stats, sizeof(hs), cudaMemcpyDeviceToHost, st));
    PN_CU(cudaMemcpyAsync(&herr, R.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    PN_CU(cudaStreamSynchronize(st));
    // counters of this append: the queries it searched and their candidates
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->stats.queries = hs[PN_ST_QUERIES];
    ctx->stats.candidates = hs[PN_ST_CANDIDATES];
    ctx->stats.exact_stream = hs[PN_ST_LB_PASSED];
    ctx->stats.device_bytes = R.footprint;
    ctx->stats.kernel_launches = ctx->launches;
    return herr ? PANACHE_ETIMEOUT : PANACHE_OK;
}

int copy_out(const std::vector<panache_motif> &m, panache_motif *out, int64_t cap, int64_t *out_len) {
    if (out_len) *out_len = (int64_t)m.size();
    if ((int64_t)m.size() > cap) return PANACHE_ETRUNC;
    if (!m.empty()) {
        if (!out) return PANACHE_EINVAL;
        memcpy(out, m.data(), sizeof(panache_motif) * m.size());
    }
    return PANACHE_OK;
}

}  // namespace

namespace pn_rt {
int64_t stream_capacity(const panache_stream *h) { return h ? h->cap : 0; }

int64_t grow_capacity(int64_t cap, int64_t need) {
    if (need <= cap) return cap;
    return std::min<int64_t>(PN_MAX_SERIES_LEN, std::max<int64_t>(std::max<int64_t>(cap * 2, need + need / 2), 4096));
}

int run(panache_ctx *ctx, const std::vector<PnSeriesIn> &in, std::vector<std::vector<panache_motif>> &res) {
    return run_request(ctx, in, res);
}

int footprint(panache_ctx *ctx, const PnSeriesIn &s_in, uint64_t *bytes) {
    PnSeriesIn s = s_in;
    if (!s.ptr) s.ptr = bytes;          // planning reads sizes only, never the samples
    PN_TRY(check_series(s));
    PnRequest one;
    panache_config unbounded = ctx->cfg;      // read only: safe while ctx runs a request
    unbounded.hbm_budget_bytes = 0;
    PN_TRY(plan(unbounded, std::vector<SeriesIn>{s}, one));
    *bytes = one.footprint;
    return PANACHE_OK;
}
}  // namespace pn_rt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace {

// Appends `len` samples; when they outgrow the capacity the state is rebuilt
// at `cap_to` (when it holds them) or at grow_capacity's choice.
int stream_append(panache_stream *h, const void *chunk, int32_t dtype, int64_t len, int64_t cap_to) {
    if (!h || len < 0 || (len > 0 && !chunk)) return PANACHE_EINVAL;
    const int dt = dtype & 0xFF;
    if ((dt != PANACHE_F32 && dt != PANACHE_F64) || (dtype & ~0x1FF)) return PANACHE_EINVAL;
    if (len == 0) return PANACHE_OK;
    if (h->len + len > PN_MAX_SERIES_LEN) return PANACHE_EINVAL;
    panache_ctx *ctx = h->ctx;
    if (!ctx) return PANACHE_ESTATE;
    cudaStream_t st = ctx->st;
    ctx->launches = 0;
    if (h->len + len > h->cap) {
        // grow: a fresh state at twice the capacity, rebuilt from the samples
        // (every step is a function of the samples, so the rebuilt state
        // equals the one the appends would have produced)
        const int64_t nc = cap_to >= h->len + len && cap_to <= PN_MAX_SERIES_LEN
                               ? cap_to : pn_rt::grow_capacity(h->cap, h->len + len);
        PnRequest *R2 = nullptr;
        PN_TRY(stream_alloc(h, nc, R2));
        if (h->len) {
            k_put<<<(unsigned)((h->len + 255) / 256), 256, 0, st>>>(h->R->x, PANACHE_F64, h->len, 0, R2->x, R2->xs);
            PN_CU(cudaGetLastError());
        }
        delete h->R;
        h->R = R2;
        h->cap = nc;
        h->q_done.assign(R2->anc.size(), 0);
        h->nw_feat.assign(R2->anc.size(), 0);
    }
    PnRequest &R = *h->R;
    const int es = dt == PANACHE_F32 ? 4 : 8;
    const void *src = chunk;
    void *stage = nullptr;
    if (!(dtype & PANACHE_DEVICE)) {
        PN_CU(cudaMallocAsync(&stage, (size_t)len * es, st));
        PN_CU(cudaMemcpyAsync(stage, chunk, (size_t)len * es, cudaMemcpyHostToDevice, st));
        src = stage;
    }
    k_put<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(src, dtype, len, h->len, R.x, R.xs);
    PN_CU(cudaGetLastError());
    if (stage) PN_CU(cudaFreeAsync(stage, st));
    h->len += len;
    return stream_advance(h);
}

}  // namespace

namespace pn_rt {
int append_to(panache_stream *h, const void *chunk, int32_t dtype, int64_t len, int64_t cap) {
    return stream_append(h, chunk, dtype, len, cap);
}
}  // namespace pn_rt

extern "C" {

int panache_default_config(panache_config *cfg) {
    if (!cfg) return PANACHE_EINVAL;
    memset(cfg, 0, sizeof(*cfg));
    fill_defaults(*cfg, false);
    return PANACHE_OK;
}

int panache_create(const panache_config *cfg, panache_ctx **out) {
    if (!out) return PANACHE_EINVAL;
    *out = nullptr;
    panache_config c;
    if (cfg) c = *cfg; else memset(&c, 0, sizeof(c));
    fill_defaults(c);
    PN_TRY(check_config(c));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PANACHE_ENODEV;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return PANACHE_ENODEV;
    if (prop.major != 10 || prop.minor != 3) return PANACHE_ENODEV;
    panache_ctx *ctx = new (std::nothrow) panache_ctx();
    if (!ctx) return PANACHE_ENOMEM;
    ctx->cfg = c;
    ctx->device = dev;
    ctx->sm_count = prop.multiProcessorCount;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    if (cudaStreamCreateWithFlags(&ctx->own, cudaStreamNonBlocking) != cudaSuccess) {
        delete ctx;
        return PANACHE_ECUDA;
    }
    ctx->st = ctx->own;
    *out = ctx;
    return PANACHE_OK;
}

void panache_destroy(panache_ctx *ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    // streams still open lose their device state; their handles stay valid
    // for panache_stream_close (and fail with ESTATE otherwise)
    for (panache_stream *h : ctx->streams) {
        delete h->R;
        h->R = nullptr;
        h->ctx = nullptr;
    }
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    ctx->drop_graph();
    delete ctx->last;
    if (ctx->pin) cudaFreeHost(ctx->pin);
    if (ctx->own) cudaStreamDestroy(ctx->own);
    delete ctx;
}

int panache_set_stream(panache_ctx *ctx, void *stream) {
    if (!ctx) return PANACHE_EINVAL;
    ctx->st = stream ? (cudaStream_t)stream : ctx->own;
    return PANACHE_OK;
}

int panache_pmp(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min, int32_t m_max,
                int32_t k, int32_t excl, panache_motif *out, int64_t out_cap, int64_t *out_len) {
    if (!ctx || !out_len) return PANACHE_EINVAL;
    std::vector<SeriesIn> in{SeriesIn{series, dtype, n, m_min, m_max, k, excl}};
    std::vector<std::vector<panache_motif>> res;
    PN_TRY(run_request(ctx, in, res));
    return copy_out(res[0], out, out_cap, out_len);
}

int panache_pmp_anchor_shard(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                             int32_t m_max, int32_t k, int32_t excl, int32_t rank, int32_t world, uint64_t *rows,
                             int64_t cap) {
    if (!ctx || !rows || world < 1 || rank < 0 || rank >= world) return PANACHE_EINVAL;
    SeriesIn si{series, dtype, n, m_min, m_max, k, excl};
    PN_TRY(check_series(si));
    if (cap < (int64_t)(m_max - m_min + 1) * n) return PANACHE_ETRUNC;
    PnShard sh;
    sh.rank = rank;
    sh.world = world;
    sh.rows_out = rows;
    std::vector<std::vector<panache_motif>> res;
    return run_request(ctx, std::vector<SeriesIn>{si}, res, &sh);
}

int panache_pmp_from_rows(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min, int32_t m_max,
                          int32_t k, int32_t excl, const uint64_t *rows, panache_motif *out, int64_t out_cap,
                          int64_t *out_len) {
    if (!ctx || !rows || !out_len) return PANACHE_EINVAL;
    SeriesIn si{series, dtype, n, m_min, m_max, k, excl};
    PN_TRY(check_series(si));
    PnShard sh;
    sh.rows_in = rows;
    std::vector<std::vector<panache_motif>> res;
    PN_TRY(run_request(ctx, std::vector<SeriesIn>{si}, res, &sh));
    return copy_out(res[0], out, out_cap, out_len);
}

int panache_pmp_batch(panache_ctx *ctx, const panache_request *reqs, int32_t nreq, panache_motif *out,
                      int64_t out_cap_per_req, int64_t *out_len) {
    if (!ctx || !reqs || nreq <= 0 || !out_len || out_cap_per_req < 0) return PANACHE_EINVAL;
    std::vector<SeriesIn> in;
    for (int32_t r = 0; r < nreq; ++r) {
        in.push_back(SeriesIn{reqs[r].series, reqs[r].dtype, reqs[r].n, reqs[r].m_min, reqs[r].m_max, reqs[r].k,
                              reqs[r].excl});
        PN_TRY(check_series(in.back()));
    }
    // Waves: consecutive series whose summed footprint fits the budget (the
    // configured one, else 60% of the free device memory) and the 32-bit
    // index spaces of one request.
    size_t budget = ctx->cfg.hbm_budget_bytes;
    if (!budget) {
        size_t fr = 0, tot = 0;
        PN_CU(cudaMemGetInfo(&fr, &tot));
        budget = (size_t)(0.6 * (double)fr);
    }
    std::vector<std::pair<int32_t, int32_t>> waves;
    {
        int32_t w0 = 0;
        size_t acc = 0;
        int64_t items = 0, buckets = 0, wins = 0;
        for (int32_t r = 0; r < nreq; ++r) {
            PnRequest one;
            panache_config unbounded = ctx->cfg;
            unbounded.hbm_budget_bytes = 0;
            PN_TRY(plan(unbounded, std::vector<SeriesIn>{in[r]}, one));
            if (one.footprint > budget) return PANACHE_EBUDGET;
            const bool full = acc + one.footprint > budget || items + one.total_items >= 0xFFFFFFFFll ||
                              buckets + one.total_buckets >= 0xFFFFFFFEll || wins + one.total_windows >= 0xFFFFFFFFll;
            if (r > w0 && full) {
                waves.push_back({w0, r});
                w0 = r;
                acc = 0;
                items = buckets = wins = 0;
            }
            acc += one.footprint;
            items += one.total_items;
            buckets += one.total_buckets;
            wins += one.total_windows;
        }
        waves.push_back({w0, nreq});
    }
    panache_stats total;
    memset(&total, 0, sizeof(total));
    int rc = PANACHE_OK;
    for (auto &wv : waves) {
        std::vector<SeriesIn> part(in.begin() + wv.first, in.begin() + wv.second);
        std::vector<std::vector<panache_motif>> res;
        PN_TRY(run_request(ctx, part, res));
        const panache_stats &st = ctx->stats;
        total.queries += st.queries;
        total.candidates += st.candidates;
        total.exact_stream += st.exact_stream;
        total.exact_sieve += st.exact_sieve;
        total.exact_completion += st.exact_completion;
        total.hot_classes += st.hot_classes;
        total.completion_rounds = std::max(total.completion_rounds, st.completion_rounds);
        total.device_bytes = std::max(total.device_bytes, st.device_bytes);
        total.kernel_launches += st.kernel_launches;
        total.refine_passes = std::max(total.refine_passes, st.refine_passes);
        total.exact_refine += st.exact_refine;
        for (int t = 0; t < 8; ++t) total.step_ms[t] += st.step_ms[t];
        for (int32_t r = wv.first; r < wv.second; ++r) {
            int e = copy_out(res[r - wv.first], out ? out + (int64_t)r * out_cap_per_req : nullptr, out_cap_per_req,
                             &out_len[r]);
            if (e != PANACHE_OK) rc = e;
        }
    }
    total.waves = waves.size();
    ctx->stats = total;
    return rc;
}

int panache_stream_open(panache_ctx *ctx, int32_t m_min, int32_t m_max, int32_t k, int32_t excl,
                        panache_stream **out) {
    if (!ctx || !out) return PANACHE_EINVAL;
    *out = nullptr;
    SeriesIn probe{nullptr, PANACHE_F64, 0, m_min, m_max, k, excl};
    PN_TRY(check_series(probe));
    panache_stream *h = new (std::nothrow) panache_stream();
    if (!h) return PANACHE_ENOMEM;
    h->ctx = ctx;
    h->m_min = m_min;
    h->m_max = m_max;
    h->k = k;
    h->excl = excl;
    ctx->streams.insert(h);
    *out = h;
    return PANACHE_OK;
}

int panache_append(panache_stream *h, const void *chunk, int32_t dtype, int64_t len) {
    return stream_append(h, chunk, dtype, len, 0);
}

int panache_stream_topk(panache_stream *h, panache_motif *out, int64_t out_cap, int64_t *out_len) {
    if (!h || !out_len) return PANACHE_EINVAL;
    if (!h->ctx) return PANACHE_ESTATE;
    if (h->len == 0 || !h->R) {
        *out_len = 0;
        return PANACHE_OK;
    }
    panache_ctx *ctx = h->ctx;
    PnRequest &R = *h->R;
    cudaStream_t st = R.st;
    memset(&ctx->stats, 0, sizeof(ctx->stats));
    ctx->kt.reset((ctx->cfg.flags & PANACHE_FLAG_TIMING) != 0);
    ctx->launches = 0;
    ctx->stats.device_bytes = R.footprint;
    PN_CU(cudaMemsetAsync(R.stats, 0, sizeof(unsigned long long) * PN_ST_COUNT, st));
    // Algorithm 2 and the pending tail run on a copy of the rows
    unsigned long long *rows = nullptr;
    const size_t bytes = sizeof(unsigned long long) * (size_t)std::max<int64_t>(1, R.total_cells);
    PN_CU(cudaMallocAsync((void **)&rows, bytes, st));
    PN_CU(cudaMemcpyAsync(rows, R.prof, bytes, cudaMemcpyDeviceToDevice, st));
    PnView v = make_view(ctx, R);
    v.prof = rows;
    std::vector<int64_t> q_end(R.anc.size());
    for (size_t ai = 0; ai < R.anc.size(); ++ai) q_end[ai] = R.anc[ai].nw;
    int rc = stream_search(ctx, R, v, h->q_done, q_end);
    std::vector<std::vector<panache_motif>> res;
    StepTimer tm;
    if (rc == PANACHE_OK) rc = tm.start(false, st);
    if (rc == PANACHE_OK) rc = run_emit(ctx, R, v, tm, res);
    cudaFreeAsync(rows, st);
    if (rc != PANACHE_OK) return rc;
    return copy_out(res[0], out, out_cap, out_len);
}

int64_t panache_stream_length(const panache_stream *h) { return h ? h->len : -1; }

int panache_stream_checkpoint(const panache_stream *h, double *out, int64_t cap, int64_t *out_len) {
    if (!h || !out_len) return PANACHE_EINVAL;
    *out_len = h->len;
    if (cap < h->len) return PANACHE_ETRUNC;
    if (!h->len) return PANACHE_OK;
    if (!out) return PANACHE_EINVAL;
    if (!h->ctx || !h->R) return PANACHE_ESTATE;
    PN_CU(cudaMemcpyAsync(out, h->R->x, sizeof(double) * h->len, cudaMemcpyDeviceToHost, h->R->st));
    PN_CU(cudaStreamSynchronize(h->R->st));
    return PANACHE_OK;
}

void panache_stream_close(panache_stream *h) {
    if (!h) return;
    if (h->ctx) {
        if (h->ctx->st) cudaStreamSynchronize(h->ctx->st);
        h->ctx->streams.erase(h);
    }
    delete h;
}

int panache_last_stats(const panache_ctx *ctx, panache_stats *out) {
    if (!ctx || !out) return PANACHE_EINVAL;
    *out = ctx->stats;
    return PANACHE_OK;
}

int panache_profile_rows(const panache_ctx *ctx, int32_t series_index, uint64_t *keys, int64_t cap) {
    if (!ctx || !keys) return PANACHE_EINVAL;
    if (!ctx->last) return PANACHE_ESTATE;
    const PnRequest &R = *ctx->last;
    if (series_index < 0 || series_index >= (int32_t)R.ser.size()) return PANACHE_EINVAL;
    const PnSeries &S = R.ser[series_index];
    const int64_t cells = (int64_t)(S.m_max - S.m_min + 1) * S.n;
    if (cap < cells) return PANACHE_ETRUNC;
    PN_CU(cudaMemcpy(keys, R.prof + S.row_off, 8 * cells, cudaMemcpyDeviceToHost));
    return PANACHE_OK;
}

int panache_anchor_state(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, int32_t *a_out,
                         float *features, uint32_t *keys, int64_t cap_windows) {
    if (!ctx) return PANACHE_EINVAL;
    if (!ctx->last) return PANACHE_ESTATE;
    const PnRequest &R = *ctx->last;
    if (series_index < 0 || series_index >= (int32_t)R.ser.size()) return PANACHE_EINVAL;
    const PnSeries &S = R.ser[series_index];
    if (anchor_index < 0 || anchor_index >= S.anchor_count) return PANACHE_EINVAL;
    const PnAnchor &A = R.anc[S.anchor_begin + anchor_index];
    if (a_out) *a_out = A.a;
    if ((features || keys) && cap_windows < A.nw) return PANACHE_ETRUNC;
    const int C = (int)ctx->cfg.chunk;
    if (features) {
        std::vector<float> blk((size_t)A.nchunk * C * PN_FEAT);
        if (R.Fh) {
            std::vector<__half> hb(blk.size());
            PN_CU(cudaMemcpy(hb.data(), R.Fh + A.row_off * PN_FEAT, sizeof(__half) * hb.size(),
                             cudaMemcpyDeviceToHost));
            for (size_t t = 0; t < hb.size(); ++t) blk[t] = __half2float(hb[t]);
        } else {
            PN_CU(cudaMemcpy(blk.data(), R.F + A.row_off * PN_FEAT, 4 * blk.size(), cudaMemcpyDeviceToHost));
        }
        for (int64_t q = 0; q < A.nw; ++q)
            memcpy(features + q * PN_FEAT, blk.data() + pn_row(q, C, A.nchunk) * PN_FEAT, 4 * PN_FEAT);
    }
    if (keys) PN_CU(cudaMemcpy(keys, R.sig + A.win_off, 4 * A.nw, cudaMemcpyDeviceToHost));
    return PANACHE_OK;
}

int panache_inject_fault(int32_t kind, int32_t after) {
    if (kind < PANACHE_FAULT_NONE || kind > PANACHE_FAULT_TC_WAIT || after < 0) return PANACHE_EINVAL;
    g_fault_kind.store(PANACHE_FAULT_NONE);
    g_fault_after.store(after);
    g_fault_kind.store(kind);
    return PANACHE_OK;
}

static_assert(PN_KT_COUNT == PANACHE_KERNEL_TIMES, "kernel timer slots and the header's count differ");

int panache_kernel_times(const panache_ctx *ctx, double *ms, uint64_t *launches, int32_t cap) {
    if (!ctx || cap < 0 || (cap > 0 && (!ms || !launches))) return PANACHE_EINVAL;
    if (cap < PN_KT_COUNT) return PANACHE_ETRUNC;
    for (int k = 0; k < PN_KT_COUNT; ++k) {
        ms[k] = ctx->kt.ms[k];
        launches[k] = ctx->kt.launches[k];
    }
    return PANACHE_OK;
}

int panache_query_candidates(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, const int64_t *q,
                             int32_t nq, uint32_t *cand, int32_t cap, int32_t *counts) {
    if (!ctx || nq < 0 || cap < 1 || (nq > 0 && (!q || !cand || !counts))) return PANACHE_EINVAL;
    if (!ctx->last) return PANACHE_ESTATE;
    PnRequest &R = *ctx->last;
    if (series_index < 0 || series_index >= (int32_t)R.ser.size()) return PANACHE_EINVAL;
    const PnSeries &S = R.ser[series_index];
    if (anchor_index < 0 || anchor_index >= S.anchor_count) return PANACHE_EINVAL;
    if (nq == 0) return PANACHE_OK;
    const int32_t ai = S.anchor_begin + anchor_index;
    cudaStream_t st = ctx->st;
    int64_t *dq = nullptr;
    uint32_t *dc = nullptr;
    int32_t *dn = nullptr;
    PN_CU(cudaMallocAsync((void **)&dq, sizeof(int64_t) * nq, st));
    PN_CU(cudaMallocAsync((void **)&dc, sizeof(uint32_t) * (size_t)nq * cap, st));
    PN_CU(cudaMallocAsync((void **)&dn, sizeof(int32_t) * nq, st));
    int rc = from_cuda(cudaMemcpyAsync(dq, q, sizeof(int64_t) * nq, cudaMemcpyHostToDevice, st));
    const PnView v = make_view(const_cast<panache_ctx *>(ctx), R);
    if (rc == PANACHE_OK) rc = from_cuda(pn::launch_query_candidates(v, ai, dq, nq, dc, cap, dn, st));
    if (rc == PANACHE_OK)
        rc = from_cuda(cudaMemcpyAsync(cand, dc, sizeof(uint32_t) * (size_t)nq * cap, cudaMemcpyDeviceToHost, st));
    if (rc == PANACHE_OK) rc = from_cuda(cudaMemcpyAsync(counts, dn, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(dq, st);
    cudaFreeAsync(dc, st);
    cudaFreeAsync(dn, st);
    if (rc == PANACHE_OK) rc = from_cuda(cudaStreamSynchronize(st));
    return rc;
}

int panache_query_levels(const panache_ctx *ctx, int32_t series_index, int32_t anchor_index, int32_t *population,
                         int32_t *depth, int64_t cap_windows) {
    if (!ctx || !population || !depth) return PANACHE_EINVAL;
    if (!ctx->last) return PANACHE_ESTATE;
    PnRequest &R = *ctx->last;
    if (series_index < 0 || series_index >= (int32_t)R.ser.size()) return PANACHE_EINVAL;
    const PnSeries &S = R.ser[series_index];
    if (anchor_index < 0 || anchor_index >= S.anchor_count) return PANACHE_EINVAL;
    const int32_t ai = S.anchor_begin + anchor_index;
    const int64_t nw = R.anc[ai].nw;
    if (cap_windows < nw) return PANACHE_ETRUNC;
    if (nw <= 0) return PANACHE_OK;
    cudaStream_t st = ctx->st;
    int32_t *dp = nullptr;
    PN_CU(cudaMallocAsync((void **)&dp, sizeof(int32_t) * 2 * (size_t)nw, st));
    const PnView v = make_view(const_cast<panache_ctx *>(ctx), R);
    int rc = from_cuda(pn::launch_query_levels(v, ai, nw, dp, dp + nw, st));
    if (rc == PANACHE_OK) rc = from_cuda(cudaMemcpyAsync(population, dp, 4 * nw, cudaMemcpyDeviceToHost, st));
    if (rc == PANACHE_OK) rc = from_cuda(cudaMemcpyAsync(depth, dp + nw, 4 * nw, cudaMemcpyDeviceToHost, st));
    cudaFreeAsync(dp, st);
    if (rc == PANACHE_OK) rc = from_cuda(cudaStreamSynchronize(st));
    return rc;
}

int panache_calibrate_width(panache_ctx *ctx, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                            int32_t m_max, double eta, int32_t *K_out, double *energy, double *collisions) {
    if (!ctx || !K_out) return PANACHE_EINVAL;
    SeriesIn si{series, dtype, n, m_min, m_max, 1, 1};
    PN_TRY(check_series(si));
    if (eta == 0.0) eta = 0.85;
    if (!(eta > 0.0 && eta <= 1.0)) return PANACHE_EINVAL;
    const panache_config &c = ctx->cfg;
    cudaStream_t st = ctx->st;
    // sample: at m_min, the midpoint and m_max, up to 256 evenly spaced starts each
    std::vector<int> lengths;
    for (int m : {m_min, (m_min + m_max) / 2, m_max})
        if (std::find(lengths.begin(), lengths.end(), m) == lengths.end()) lengths.push_back(m);
    std::vector<PnCalWin> win;
    std::vector<int> g_off, g_cnt, row_g, row_a;
    for (size_t g = 0; g < lengths.size(); ++g) {
        const int m = lengths[g];
        const int64_t nw = n - m + 1;
        g_off.push_back((int)win.size());
        if (nw > 0) {
            const int64_t S = std::min<int64_t>(256, nw);
            int64_t last = -1;
            for (int64_t t = 0; t < S; ++t) {
                const int64_t s0 = S == 1 ? 0 : t * (nw - 1) / (S - 1);
                if (s0 == last) continue;
                last = s0;
                win.push_back(PnCalWin{s0, m, (int32_t)g});
            }
        }
        g_cnt.push_back((int)win.size() - g_off.back());
        for (int a = 0; a + 1 < g_cnt.back(); ++a) {
            row_g.push_back((int)g);
            row_a.push_back(a);
        }
    }
    // the series as FP64 on the device
    const int dt = dtype & 0xFF;
    const size_t es = dt == PANACHE_F32 ? 4 : 8;
    void *stage = nullptr;
    double *x = nullptr;
    PnCalWin *dwin = nullptr;
    int *dgo = nullptr, *dgc = nullptr, *drg = nullptr, *dra = nullptr;
    double *dout = nullptr;
    std::vector<double> hout(2 * (PN_MAXK - 1) + 1, 0.0);
    int rc = PANACHE_OK;
    do {
        const void *src = series;
        if (!(dtype & PANACHE_DEVICE) && n) {
            if ((rc = from_cuda(cudaMallocAsync(&stage, (size_t)n * es, st)))) break;
            if ((rc = from_cuda(cudaMemcpyAsync(stage, series, (size_t)n * es, cudaMemcpyHostToDevice, st)))) break;
            src = stage;
        }
        if ((rc = from_cuda(cudaMallocAsync((void **)&x, sizeof(double) * std::max<int64_t>(1, n), st)))) break;
        float2 *scratch = nullptr;
        if ((rc = from_cuda(cudaMallocAsync((void **)&scratch, sizeof(float2) * std::max<int64_t>(1, n), st)))) break;
        if (n) k_put<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(src, dtype, n, 0, x, scratch);
        cudaFreeAsync(scratch, st);
        if ((rc = upload_tmp(st, win, dwin))) break;
        if ((rc = upload_tmp(st, g_off, dgo))) break;
        if ((rc = upload_tmp(st, g_cnt, dgc))) break;
        if ((rc = upload_tmp(st, row_g, drg))) break;
        if ((rc = upload_tmp(st, row_a, dra))) break;
        if ((rc = from_cuda(cudaMallocAsync((void **)&dout, sizeof(double) * hout.size(), st)))) break;
        if ((rc = from_cuda(pn::launch_calibration(x, dwin, (int)win.size(), dgo, dgc, drg, dra, (int)row_g.size(),
                                                   (int)c.B, dout, st))))
            break;
        if ((rc = from_cuda(cudaMemcpyAsync(hout.data(), dout, sizeof(double) * hout.size(), cudaMemcpyDeviceToHost,
                                            st))))
            break;
        rc = from_cuda(cudaStreamSynchronize(st));
    } while (false);
    for (void *p : {(void *)stage, (void *)x, (void *)dwin, (void *)dgo, (void *)dgc, (void *)drg, (void *)dra,
                    (void *)dout})
        if (p) cudaFreeAsync(p, st);
    PN_TRY(rc);
    // the smallest width meeting both conditions, else the largest
    const int nk = PN_MAXK - 1;
    int K = PN_MAXK;
    for (int t = 0; t < nk; ++t) {
        if (hout[t] >= eta && (double)n * hout[nk + t] <= 2.0 * (double)c.gamma * (double)c.alpha) {
            K = t + 2;
            break;
        }
    }
    *K_out = K;
    if (energy) memcpy(energy, hout.data(), sizeof(double) * nk);
    if (collisions) memcpy(collisions, hout.data() + nk, sizeof(double) * nk);
    return PANACHE_OK;
}

int panache_projections(const panache_config *cfg, int32_t a, float *g, int64_t cap) {
    if (!g || a < 1) return PANACHE_EINVAL;
    panache_config c;
    if (cfg) c = *cfg; else memset(&c, 0, sizeof(c));
    fill_defaults(c);
    PN_TRY(check_config(c));
    const int64_t need = (int64_t)(c.B + 1) * PN_FEAT;
    if (cap < need) return PANACHE_ETRUNC;
    pn::projections(a, c.seed, (int)c.B, (int)c.K, g);
    return PANACHE_OK;
}

const char *panache_strerror(int code) {
    switch (code) {
        case PANACHE_OK: return "ok";
        case PANACHE_EINVAL: return "invalid argument";
        case PANACHE_ENOMEM: return "out of memory";
        case PANACHE_EBUDGET: return "request exceeds the HBM budget (admission refused)";
        case PANACHE_ECUDA: return "CUDA error";
        case PANACHE_ETRUNC: return "output buffer too small";
        case PANACHE_ESTATE: return "invalid state for this call";
        case PANACHE_EPOOL: return "top-k selection pool overflow";
        case PANACHE_ENODEV: return "no sm_103 CUDA device";
        case PANACHE_ETIMEOUT: return "a wait ran out of time";
        case PANACHE_EBUSY: return "refused at admission: the predicted wait exceeds the server's deadline";
        default: return "unknown error";
    }
}

}  // extern "C"
