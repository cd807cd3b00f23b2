// Streaming candidate search at the anchor lengths (Sec. 3.4-3.5,
// Algorithm 1 phase B), one warp per query window.
//
// For query q of anchor a the directory population is the number of
// non-constant windows inserted by the end of q's batch (batches of beta
// samples of stream time), which fixes the global depth d and so the level
// to probe.  Probes: the exact d-bit prefix bucket, then 1 + max(0, d - d0)
// Hamming-1 buckets (capped by d and the probe cap) in increasing
// |<g_{a,l}, F_q>|.  Candidates are earlier windows c <= q - excl; a bucket
// with more valid entries than the remaining budget r gives ceil(r/2) of its
// most recent entries and floor(r/2) evenly spaced ones.  A candidate is
// evaluated exactly iff (1 - lambda) LB < max(best_q, P[c]) (Lemma 2, the
// threshold of Algorithm 1), where best_q also takes the live value of the
// query's own cell; both cells receive the distance by packed atomicMin.
// The test is taken on squares, (1 - lambda)^2 LB^2 < threshold^2, with no
// root: FP32 rounding of either form is far inside the lambda slack.
//
// The final profile does not depend on the schedule: a pair is skipped only
// when its distance exceeds, by the factor 1/(1 - lambda), the current value
// of both cells it could lower, and cells only decrease, so every pair whose
// key would win a cell is evaluated.
//
// Queries run in the order of the bucket they probe first (qorder), so warps
// active at the same time share candidate rows in L2.  The query's
// z-normalised window is staged once in shared memory; each surviving
// candidate streams its own window against it.
#include "distance.cuh"
#include "zops.cuh"
#include "evalbatch.cuh"
#include "search.cuh"

namespace pn {
namespace {

constexpr int SR_WARPS = 8;
constexpr int SR_THREADS = SR_WARPS * 32;
constexpr int SR_MAXR = 512;   // largest supported budget R

// HALF: the rows are read from the half-precision copy, and every bound test
// carries the rounding margin of pn_row_margin.
//
// WARM: the warm start that runs before the search.  Each query takes the
// SR_WARM most recent valid entries of its exact bucket -- a subset of the
// candidates the search admits, whatever the budget split -- bounds them and
// evaluates the one of smallest bound exactly, updating both cells.  Queries
// run grouped by bucket, not in stream order, so without it many candidate
// cells are still empty when a query tests them and the threshold
// max(best_q, P[c]) rejects nothing; after it, nearly every cell holds the
// exact distance of an admitted pair.  The final profile is unchanged (it
// is the minimum over the admitted pairs); only the number of pairs the
// bound lets through drops.
#ifndef PN_SR_TILE
#define PN_SR_TILE 8
#endif
constexpr int SR_TILE = PN_SR_TILE;   // queries a warp takes from the work queue at a time

// A persistent kernel: SMs x grid_mult blocks, and each warp takes the next
// SR_TILE queries of the query order from a global work counter until the
// order is exhausted, so warps that draw cheap queries take more of them.
#ifndef PN_SR_MINB
#define PN_SR_MINB 5
#endif

// Byte offsets of the search kernel's per-block dynamic shared memory: each
// array holds SR_WARPS per-warp slices, every array 16-byte aligned.
template <class Z>
struct SrLayout {
    size_t snap, zq, cand, mom, sum, bytes;
    __host__ __device__ SrLayout(int R, int zcap) {
        auto up = [](size_t b) { return (b + 15) & ~(size_t)15; };
        snap = 0;
        zq = up(snap + sizeof(unsigned long long) * (size_t)R * SR_WARPS);
        cand = up(zq + sizeof(typename Z::Q) * (size_t)zcap * SR_WARPS);
        mom = up(cand + sizeof(uint32_t) * (size_t)R * SR_WARPS);
        sum = up(mom + sizeof(typename Z::M) * (size_t)R * SR_WARPS);
        bytes = up(sum + sizeof(typename Z::T) * (size_t)R * SR_WARPS);
    }
};

template <class Z, bool HALF, bool WARM>
__global__ void __launch_bounds__(SR_THREADS, PN_SR_MINB) k_search(PnView v, int64_t total, int zcap,
                                                        unsigned long long *work) {
    using ZT = typename Z::T;
    __shared__ __align__(16) float sF[SR_WARPS][PN_FEAT];
    __shared__ unsigned long long s_stat[3];
    __shared__ uint32_t sprobe[SR_WARPS][32];
    extern __shared__ __align__(16) unsigned char dsm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int R = v.R;
    using ZQ = typename Z::Q;
    using ZM = typename Z::M;
    // per warp: survivor snapshots, staged query window, candidate list
    // (survivors compacted at its front), survivor moments and sums
    const SrLayout<Z> lay(R, zcap);
    unsigned long long *snap = reinterpret_cast<unsigned long long *>(dsm + lay.snap) + warp * R;
    ZQ *zq = reinterpret_cast<ZQ *>(dsm + lay.zq) + warp * zcap;
    uint32_t *scand = reinterpret_cast<uint32_t *>(dsm + lay.cand) + warp * R;
    ZM *smom = reinterpret_cast<ZM *>(dsm + lay.mom) + warp * R;
    ZT *ssum = reinterpret_cast<ZT *>(dsm + lay.sum) + warp * R;
    const auto *xb = Z::samples(v, 0);
    if (threadIdx.x < 3) s_stat[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long n_q = 0, n_c = 0, n_lb = 0;
    const int dims = 2 * (v.K - 1);
    const float shrink = 1.0f - v.lam;
    const float shrink2 = shrink * shrink;
    // anchor of the previous query and its window range [a_lo, a_hi): the
    // query order keeps each anchor's queries together, so the search over
    // the anchor table is mostly skipped
    int ai = 0;
    int64_t a_lo = 1, a_hi = 0;

    int64_t tile = 0, tile_end = 0;
    for (int64_t it = 0;; ++it) {
        if (it >= tile_end) {                              // warp-uniform: next tile of the queue
            unsigned long long t0 = 0;
            if (lane == 0) t0 = atomicAdd(work, (unsigned long long)SR_TILE);
            tile = (int64_t)__shfl_sync(0xffffffffu, t0, 0);
            if (tile >= total) break;
            it = tile;
            tile_end = min(total, tile + SR_TILE);
        }
        const int64_t w = v.qorder[it];
        if (w < a_lo || w >= a_hi) {
            ai = pn_find(v.anchors, v.nanchors, w, [](const PnAnchor &A) { return A.win_off; });
            a_lo = v.anchors[ai].win_off;
            a_hi = ai + 1 < v.nanchors ? v.anchors[ai + 1].win_off : INT64_MAX;
        }
        const PnAnchor &A = v.anchors[ai];
        const int s = A.series;
        const PnSeries &S = v.series[s];
        const int64_t q = w - A.win_off;
        const int a = A.a;
        if (v.runlen[S.x_off + q] >= a) continue;          // constant window
        if (q < S.excl) continue;                          // no valid earlier window
        // population seen by q: everything inserted by the end of its batch
        const uint32_t P = pn_query_population(v, A, S, q);
        const int d = pn_depth_dev(P, (uint32_t)v.alpha, v.B);

        const void *Fa = pn_rows<HALF>(v, A.row_off);
        const uint32_t nch = (uint32_t)A.nchunk;
        const int taken = sr_candidates<HALF, WARM>(v, ai, A, S, w, q, d, lane, sF[warp], sprobe[warp], scand, Fa, nch,
                                                    dims, R);
        __syncwarp();
        if (!WARM) {
            n_q += 1;
            n_c += taken;
        }
        if (taken == 0) continue;

        // z-normalised query window, staged once
        {
            const auto mq = Z::load(v, w);
            const auto *xq = Z::samples(v, S.x_off + q);
            for (int r = lane; r < a; r += 32) zq[r] = Z::stage(Z::z(mq, xq[r]));
        }
        __syncwarp();
        unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
        const auto *xs = xb + S.x_off;
        const float4 fq = reinterpret_cast<const float4 *>(sF[warp])[lane & 7];
        const float2 nfxy = make_float2(-fq.x, -fq.y), nfzw = make_float2(-fq.z, -fq.w);
        unsigned long long bestkey = PN_EMPTY_KEY;
        const float lbscale = 2.0f / (float)a;
        const ZT lbmargin = HALF ? (ZT)(shrink * pn_row_margin(v.lb_eps, a)) : (ZT)0;
        // Bounds of 32 candidates at a time: lane l owns candidate l of the
        // block; its row is read by the 8 lanes of a group (4 rows per step,
        // 8 steps, every load issued before the sums need it), the 8 partial
        // sums of a lane are reduced across its group by a transposed
        // butterfly (7 shuffles), and one more shuffle hands each lane its
        // own candidate's bound.  Survivors are compacted in place at the
        // front of scand (never past a candidate not yet read), with their
        // cell snapshots in snap.
        int nsurv = 0, head = 0;
        for (int b32 = 0; b32 < taken; b32 += 32) {
            const int nblk = min(32, taken - b32);
            uint32_t c = 0, roff = 0;
            if (lane < nblk) {
                c = scand[b32 + lane];
                roff = pn_row32(c, v.cshift, nch);
            }
            float4 fc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = 4 * j + (lane >> 3);
                const uint32_t ro = __shfl_sync(0xffffffffu, roff, k);
                fc[j] = k < nblk ? pn_row_quad<HALF>(Fa, ro, lane & 7) : fq;
            }
            // squared differences of a quarter row, packed two-wide: (c - q) is
            // the exact negation of (q - c); the four squares are summed as
            // (dx^2 + dz^2) + (dy^2 + dw^2)
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float2 dxy = __fadd2_rn(make_float2(fc[j].x, fc[j].y), nfxy);
                const float2 dzw = __fadd2_rn(make_float2(fc[j].z, fc[j].w), nfzw);
                const float2 s2 = __ffma2_rn(dxy, dxy, __fmul2_rn(dzw, dzw));
                acc[j] = s2.x + s2.y;
            }
            // transposed reduction over the 8 lanes of a group: afterwards lane L
            // holds the sum of candidate 4 (L & 7) + (L >> 3)
            const bool b2 = (lane & 4) != 0, b1 = (lane & 2) != 0, b0 = (lane & 1) != 0;
            float r4[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float send = b2 ? acc[i] : acc[i + 4];
                r4[i] = (b2 ? acc[i + 4] : acc[i]) + __shfl_xor_sync(0xffffffffu, send, 4);
            }
            float r2[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const float send = b1 ? r4[i] : r4[i + 2];
                r2[i] = (b1 ? r4[i + 2] : r4[i]) + __shfl_xor_sync(0xffffffffu, send, 2);
            }
            const float tot = (b0 ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, b0 ? r2[0] : r2[1], 1);
            const float lbsq = __shfl_sync(0xffffffffu, tot, ((lane & 3) << 3) | (lane >> 2));
            unsigned long long kc = 0;
            float lbs = __int_as_float(0x7f800000);
            if (lane < nblk) {
                kc = __ldcg(&prow[c]);
                lbs = shrink2 * (lbscale * lbsq);            // ((1 - lambda) LB)^2
            }
            const ZT cq = Z::cell(__ldcg(&prow[q]));
            // best-first start: while the query has no distance yet, the block's
            // smallest bound is evaluated before the others are tested, so the
            // query's threshold is tight from the first block on
            if (bestkey == PN_EMPTY_KEY) {
                float bm = lbs;
                int bl = lane;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float om = __shfl_xor_sync(0xffffffffu, bm, o);
                    const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
                    if (om < bm || (om == bm && ol < bl)) {
                        bm = om;
                        bl = ol;
                    }
                }
                const uint32_t cb = __shfl_sync(0xffffffffu, c, bl);
                const unsigned long long kb = __shfl_sync(0xffffffffu, kc, bl);
                ZT tb = Z::fmx(Z::fmn(Z::cell(bestkey), cq), Z::cell(kb));
                if constexpr (HALF) tb += lbmargin;
                if (bl < nblk && (ZT)bm < tb * tb) {
                    eval_one<Z>(v, zq, cb, kb, S.x_off, A.win_off, a, (uint32_t)q, prow, bestkey, lane);
                    n_lb += 1;
                }
                if (lane == bl) lbs = __int_as_float(0x7f800000);   // done: not retested
            }
            if constexpr (WARM) break;                      // the warm start evaluates one pair
            bool surv = false;
            if (lane < nblk) {
                ZT tc = Z::fmx(Z::fmn(Z::cell(bestkey), cq), Z::cell(kc));
                if constexpr (HALF) tc += lbmargin;
                surv = (ZT)lbs < tc * tc;
            }
            const uint32_t sm = __ballot_sync(0xffffffffu, surv);
            __syncwarp();
            if (surv) {
                const int rank = __popc(sm & ((1u << lane) - 1u));
                scand[nsurv + rank] = c;
                snap[nsurv + rank] = kc;
                smom[nsurv + rank] = Z::load(v, A.win_off + c);
            }
            nsurv += __popc(sm);
            __syncwarp();
            // full batches of four now; a remainder waits for the next block
            const int h0 = head;
            while (nsurv - head >= 4) {
                eval_sums<Z>(zq, xs, scand + head, smom + head, 4, a, ssum + head, lane);
                head += 4;
            }
            __syncwarp();
            if (head > h0) eval_finish<Z>(ssum, scand, snap, smom, h0, head, (uint32_t)q, prow, bestkey, lane);
        }
        if (nsurv > head) {
            eval_sums<Z>(zq, xs, scand + head, smom + head, nsurv - head, a, ssum + head, lane);
            __syncwarp();
            eval_finish<Z>(ssum, scand, snap, smom, head, nsurv, (uint32_t)q, prow, bestkey, lane);
        }
        n_lb += nsurv;
        if (lane == 0 && bestkey != PN_EMPTY_KEY) atomicMin(&prow[q], bestkey);
        __syncwarp();
    }
    if (lane == 0) {
        atomicAdd(&s_stat[0], n_q);
        atomicAdd(&s_stat[1], n_c);
        atomicAdd(&s_stat[2], n_lb);
    }
    __syncthreads();
    if (threadIdx.x == 0 && v.stats) {
        atomicAdd(&v.stats[PN_ST_QUERIES], s_stat[0]);
        atomicAdd(&v.stats[PN_ST_CANDIDATES], s_stat[1]);
        atomicAdd(&v.stats[PN_ST_LB_PASSED], s_stat[2]);
    }
}

template <class Z, bool HALF, bool WARM>
cudaError_t launch_one(const PnView &v, int64_t total, int grid_blocks, int a_max, cudaStream_t st,
                       unsigned long long *work) {
    const int zcap = (a_max + 3) & ~3;
    const size_t sm = SrLayout<Z>(v.R, zcap).bytes;
    cudaError_t e = pn_allow_smem(k_search<Z, HALF, WARM>, sm);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    int64_t need = (total + SR_WARPS * SR_TILE - 1) / (SR_WARPS * SR_TILE);
    unsigned g = (unsigned)(need < grid_blocks ? need : grid_blocks);
    k_search<Z, HALF, WARM><<<g, SR_THREADS, sm, st>>>(v, total, zcap, work);
    return cudaGetLastError();
}

template <class Z, bool HALF>
cudaError_t launch_t(const PnView &v, int64_t total, int grid_blocks, int a_max, cudaStream_t st, bool warm) {
    unsigned long long *work = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&work, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (warm) e = launch_one<Z, HALF, true>(v, total, grid_blocks, a_max, st, work + 1);
    if (e == cudaSuccess) e = launch_one<Z, HALF, false>(v, total, grid_blocks, a_max, st, work);
    cudaFreeAsync(work, st);
    return e;
}

// Introspection: the population and depth of every window of one anchor,
// taken exactly as k_search takes them.
__global__ void k_query_levels(PnView v, int32_t anchor, int64_t nw, int32_t *population, int32_t *depth) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nw) return;
    const PnAnchor &A = v.anchors[anchor];
    const PnSeries &S = v.series[A.series];
    if (v.runlen[S.x_off + q] >= A.a || q < S.excl) {
        population[q] = -1;
        depth[q] = -1;
        return;
    }
    const uint32_t P = pn_query_population(v, A, S, q);
    population[q] = (int32_t)P;
    depth[q] = pn_depth_dev(P, (uint32_t)v.alpha, v.B);
}

// Introspection: the candidate list of each listed query of one anchor, by
// the search's own list building (one warp per query); count -1 for a
// window the search skips.
__global__ void k_query_candidates(PnView v, int32_t anchor, const int64_t *qs, int32_t nq, uint32_t *cand,
                                   int32_t cap, int32_t *counts) {
    __shared__ __align__(16) float frow[PN_FEAT];
    __shared__ uint32_t probe[32];
    __shared__ uint32_t lst[SR_MAXR];
    const int lane = threadIdx.x & 31;
    const int qi = blockIdx.x;
    if (qi >= nq) return;
    const PnAnchor &A = v.anchors[anchor];
    const PnSeries &S = v.series[A.series];
    const int64_t q = qs[qi];
    if (q < 0 || q >= A.nw || v.runlen[S.x_off + q] >= A.a || q < S.excl) {
        if (lane == 0) counts[qi] = -1;
        return;
    }
    const uint32_t P = pn_query_population(v, A, S, q);
    const int d = pn_depth_dev(P, (uint32_t)v.alpha, v.B);
    const int dims = 2 * (v.K - 1);
    const uint32_t nch = (uint32_t)A.nchunk;
    int taken;
    if (v.Fh)
        taken = sr_candidates<true, false>(v, anchor, A, S, A.win_off + q, q, d, lane, frow, probe, lst,
                                           pn_rows<true>(v, A.row_off), nch, dims, v.R);
    else
        taken = sr_candidates<false, false>(v, anchor, A, S, A.win_off + q, q, d, lane, frow, probe, lst,
                                            pn_rows<false>(v, A.row_off), nch, dims, v.R);
    for (int t = lane; t < taken && t < cap; t += 32) cand[(int64_t)qi * cap + t] = lst[t];
    if (lane == 0) counts[qi] = taken;
}

}  // namespace

int search_max_budget() { return SR_MAXR; }

cudaError_t launch_query_candidates(const PnView &v, int32_t anchor, const int64_t *qs, int32_t nq, uint32_t *cand,
                                    int32_t cap, int32_t *counts, cudaStream_t st) {
    if (nq <= 0) return cudaSuccess;
    k_query_candidates<<<nq, 32, 0, st>>>(v, anchor, qs, nq, cand, cap, counts);
    return cudaGetLastError();
}

cudaError_t launch_query_levels(const PnView &v, int32_t anchor, int64_t nw, int32_t *population, int32_t *depth,
                                cudaStream_t st) {
    if (nw <= 0) return cudaSuccess;
    k_query_levels<<<(unsigned)((nw + 255) / 256), 256, 0, st>>>(v, anchor, nw, population, depth);
    return cudaGetLastError();
}

cudaError_t launch_search(const PnView &v, int64_t total, int grid_blocks, int a_max, cudaStream_t st, bool warm) {
    if (total <= 0) return cudaSuccess;
    if (v.precision == 0) return launch_t<ZPlain, false>(v, total, grid_blocks, a_max, st, warm);
    if (v.Fh)   // half rows: the mixed form only (checked at configuration)
        return v.x1 ? launch_t<ZMix1, true>(v, total, grid_blocks, a_max, st, warm)
                    : launch_t<ZMix2, true>(v, total, grid_blocks, a_max, st, warm);
    return v.x1 ? launch_t<ZMix1, false>(v, total, grid_blocks, a_max, st, warm)
                : launch_t<ZMix2, false>(v, total, grid_blocks, a_max, st, warm);
}

}  // namespace pn
