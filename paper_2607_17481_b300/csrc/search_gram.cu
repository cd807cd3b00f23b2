// Streaming candidate search of the mixed form with a tensor-core Gram
// filter (Sec. 3.4-3.5, Algorithm 1 phase B); opt-in (PANACHE_FLAG_GRAM_SEARCH).
//
// The admitted pairs are those of the per-query search: each query's
// budgeted list over its exact prefix bucket and its Hamming-1 probes, built
// by the same device function (sr_candidates), at the depth its batch's
// population fixes.  Every admitted pair that can still lower one of its two
// cells is evaluated exactly with the per-query search's own FP32 arithmetic
// (eval_batch), so the profile rows are the same bit for bit: a cell is the
// minimum packed key over its admitted pairs whatever test decides which
// pairs are evaluated.  What differs is that test.  The per-query search
// rejects a pair by the Parseval bound of Lemma 2 over the 30 stored
// feature floats.  Here the queries that probe the same bucket first
// (consecutive in the query order) are taken GQ at a time, their lists are
// merged, and the z-normalised windows of the merged candidates and of the
// queries, rounded to FP16, are multiplied on the tensor cores:
// tcgen05.mma kind::f16, M = 128 candidates x N = 16 queries x K = window
// length (zero-padded to 16), FP32 accumulator in tensor memory.  That gives
// every listed pair an estimate d~^2 = |z_q|^2 + |z_c|^2 - 2 <z_q, z_c>~ of
// its squared distance.
//
// Error of the estimate.  z is the FP32 z-value the exact pass uses, z~ its
// FP16 rounding (|z| <= sqrt(a) < 14, far inside FP16's range), |z~ - z| <=
// 2^-11 |z| + 2^-25, so |z~_q z~_c - z_q z_c| <= (2^-10 + 2^-22) |z_q z_c|
// plus a subnormal term below a 2^-20 in total.  FP16 products are exact in
// FP32 and the tensor core's FP32 accumulation of a <= 192 of them adds at
// most a 2^-23 of their magnitudes.  Cauchy-Schwarz gives sum |z_q z_c| <=
// (|z_q|^2 + |z_c|^2) / 2, the norms are FP32 sums (relative error
// <= a 2^-24) and the exact pass's own FP32 sum of squares is within
// a 2^-24 of <= 2 (|z_q|^2 + |z_c|^2).  Together |d~^2 - d_f^2| <=
// 2^-9.9 (|z_q|^2 + |z_c|^2) =: e(q, c), where d_f is the distance the exact
// pass would store; the test uses M = 2^-9 (|z_q|^2 + |z_c|^2) > e.
//
// Which pairs are evaluated.  Pair (c, q) is evaluated iff
//   [d~^2 - M < P[c]^2 and d~^2 <= rowmin(c) + 2 M_row]  or
//   [d~^2 - M < P[q]^2 and d~^2 <= colmin(q) + 2 M_col],
// with P the cells' current values (a stale, larger value only keeps more
// pairs), rowmin(c) the smallest estimate over c's listed pairs with the
// group's queries, colmin(q) the smallest over q's listed pairs in this
// 128-candidate tile, and M_row, M_col margins with the row's (column's)
// own norm and the largest norm on the other side.  A pair failing the first
// part of a clause has d_f > P (strictly), so it cannot lower that cell; a
// pair failing the second part has d_f larger than the row's (column's)
// best pair, which wins the cell against it.  So every pair whose key could
// end in a cell is evaluated.
//
// Merging.  The group's lists (<= GQ R entries) go into an open-addressing
// hash table in shared memory keyed by window start, with a bit per query
// that lists the window; the table is compacted into the tile's rows.  On
// the wafer-like series 16 queries list ~2,000 pairs over ~500 distinct
// windows, so each window is staged once for four listed pairs.
//
// Measured on the 200,000-sample wafer-like prefix: the filter keeps 8% fewer pairs than
// the Parseval bound (near-equal distances among repeated template windows
// sit inside the FP16 margin, and the best pair of every merged window whose
// cell can still drop must be evaluated), while the group-wide steps (list
// building, merge, staging, MMA, evaluation, each behind a block barrier,
// two 8-warp blocks per SM) leave the SMs waiting on memory: 3.6 times the
// per-query search's time.  Hence opt-in.
//
// Layouts.  Both operands are K-major with the 128-byte swizzle: a row's
// 64 FP16 values of one K atom fill one 128-byte line whose 16-byte chunks
// are permuted by (row mod 8), eight rows per 1024-byte block, atoms of 64
// samples one after the other; a warp writes one line per store, with no
// bank conflict.  The MMA's K step (16 samples, 32 bytes) advances the
// descriptor's start address inside the atom.
//
// Every wait on the tensor core is bounded: on timeout the kernel records
// the error word, waits once more (bounded), frees its tensor memory and
// returns; the request reports ETIMEOUT.
#include <cuda_fp16.h>

#include "evalbatch.cuh"
#include "prims.cuh"
#include "search.cuh"
#include "tcgen05.cuh"
#include "zops.cuh"

namespace pn {
namespace {

constexpr int GS_GQ = 16;               // queries per group (MMA N)
constexpr int GS_M = 128;               // merged candidates per tile (MMA M)
constexpr int GS_WARPS = 8;
constexpr int GS_THREADS = GS_WARPS * 32;
constexpr int GS_HT = 2048;             // hash slots (>= GS_GQ * GS_RMAX distinct windows)
constexpr int GS_RMAX = 128;            // largest budget R served by this kernel
constexpr int GS_AMAX = 192;            // longest anchor served (three K atoms)
constexpr int GS_SQ = 32;               // survivor slots per query and round
constexpr int GS_SPIN = 1 << 22;        // try_wait iterations before giving up
constexpr uint32_t GS_EMPTY = 0xFFFFFFFFu;
constexpr int GS_TMEM_COLS = 32;

static_assert(GS_GQ * GS_RMAX <= GS_HT, "the table holds every listed window");
static_assert(GS_GQ * GS_SQ * 12 <= GS_GQ * GS_RMAX * 4, "survivor queues fit in the list area");

__device__ __forceinline__ uint32_t gs_hash(uint32_t c) { return (c * 2654435761u) >> (32 - 11); }

__device__ __forceinline__ float gs_warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// Query keys in sorted order -> group starts: a group is at most GS_GQ
// consecutive queries of one key (one first-probed bucket), cut from the
// start of the key's run.  flag[t] = 1 where a group starts.
__global__ void k_group_flags(const uint32_t *keys, int64_t total, uint32_t *flag) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const uint32_t k = keys[t];
    uint32_t f = 0;
    if (k != GS_EMPTY) {
        int64_t lo = 0, hi = t;                      // first index holding key k
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < k) lo = mid + 1; else hi = mid;
        }
        f = ((t - lo) % GS_GQ) == 0 ? 1u : 0u;
    }
    flag[t] = f;
}

// After the exclusive scan of the flags: gstart[g] = start of group g.
__global__ void k_group_fill(const uint32_t *keys, const uint32_t *off, int64_t total, const uint32_t *ngroups,
                             uint32_t *gstart) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    const uint32_t next = t + 1 < total ? off[t + 1] : *ngroups;
    if (next != off[t] && keys[t] != GS_EMPTY) gstart[off[t]] = (uint32_t)t;
}

struct GsShared {
    float sF[GS_WARPS][PN_FEAT];                     // sr_candidates scratch, per warp
    uint32_t sprobe[GS_WARPS][32];
    float rowmin[2][GS_M];                           // per column half
    float nc[GS_M];                                  // |z_c|^2 of the tile's rows
    float sc[GS_M];                                  // 1/sigma of the tile's rows (0: degenerate)
    int colmin[GS_GQ];                               // float bits, >= 0
    float nq[GS_GQ];                                 // |z_q|^2
    float tq[GS_GQ];                                 // the query cell's current distance
    unsigned long long qbest[GS_GQ];                 // best key of each query in this group
    uint32_t q[GS_GQ];                               // query window (index within its anchor)
    int cnt[GS_GQ];                                  // list length
    int qn[GS_GQ];                                   // survivors queued in this pass
    int ncmax, nqmax;                                // float bits
    int nu, G, ai;
    uint32_t g;
    int fail;
    uint32_t taddr;
    __align__(8) uint64_t mbar;
    unsigned long long stat[3];
};

template <class Z, bool HALF>
__global__ void __launch_bounds__(GS_THREADS, 2) k_search_gram(PnView v, const uint32_t *keys, int64_t total,
                                                               const uint32_t *gstart, const uint32_t *ngroups,
                                                               unsigned int *work, int kpad_max, int zcap) {
    using ZQ = typename Z::Q;
    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    __shared__ GsShared sh;
    // dynamic layout: A tile | B tile | staged query windows | lists + table
    unsigned char *gsm = gsm_raw + ((1024 - (smem_u32(gsm_raw) & 1023)) & 1023);
    const int atoms_max = (kpad_max + 63) >> 6;
    unsigned char *tA = gsm;
    unsigned char *tB = tA + atoms_max * GS_M * 128;
    ZQ *zq = reinterpret_cast<ZQ *>(tB + atoms_max * GS_GQ * 128);
    uint32_t *lists = reinterpret_cast<uint32_t *>(zq + GS_GQ * zcap);
    uint32_t *htk = lists + GS_GQ * GS_RMAX;
    uint32_t *htm = htk + GS_HT;
    // survivor queues reuse the list area once the lists are merged
    uint32_t *qc = lists;                                               // [GS_GQ][GS_SQ]
    unsigned long long *qk = reinterpret_cast<unsigned long long *>(lists + GS_GQ * GS_SQ);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        sh.fail = 0;
        sh.stat[0] = sh.stat[1] = sh.stat[2] = 0ull;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.taddr)),
                     "r"(GS_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = sh.taddr;
    const uint32_t idesc = umma_idesc_f16(GS_M, GS_GQ);
    const int dims = 2 * (v.K - 1);
    const int R = v.R;
    const uint32_t ng = *ngroups;
    uint32_t phase = 0;
    unsigned long long n_q = 0, n_c = 0, n_ex = 0;
    const float inf = __int_as_float(0x7f800000);

    for (;;) {
        __syncthreads();                                // the previous group is finished everywhere
        if (tid == 0) sh.g = atomicAdd(work, 1u);
        for (int s = tid; s < GS_HT; s += GS_THREADS) {
            htk[s] = GS_EMPTY;
            htm[s] = 0u;
        }
        __syncthreads();
        const uint32_t g = sh.g;
        if (g >= ng || sh.fail) break;
        const uint32_t gs = gstart[g];
        if (warp == 0) {
            const uint32_t k0 = keys[gs];
            const bool same = lane < GS_GQ && (int64_t)gs + lane < total && keys[gs + lane] == k0;
            const uint32_t bal = __ballot_sync(0xffffffffu, same);
            if (lane == 0) {
                sh.G = __popc(bal);                      // a prefix: the keys are sorted
                const int64_t w0 = v.qorder[gs];
                sh.ai = pn_find(v.anchors, v.nanchors, w0, [](const PnAnchor &A) { return A.win_off; });
                sh.ncmax = 0;
                sh.nqmax = 0;
            }
        }
        __syncthreads();
        const int G = sh.G;
        const int ai = sh.ai;
        const PnAnchor &A = v.anchors[ai];
        const PnSeries &S = v.series[A.series];
        const int a = A.a;
        const int kp = (a + 15) & ~15;
        unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
        const void *Fa = pn_rows<HALF>(v, A.row_off);
        const uint32_t nch = (uint32_t)A.nchunk;

        // ---- lists, staged query windows (FP32 for the exact pass, FP16 for the MMA), norms
        for (int j = warp; j < G; j += GS_WARPS) {
            const int64_t w = v.qorder[gs + j];
            const int64_t q = w - A.win_off;
            const uint32_t P = pn_query_population(v, A, S, q);
            const int d = pn_depth_dev(P, (uint32_t)v.alpha, v.B);
            const int taken = sr_candidates<HALF, false>(v, ai, A, S, w, q, d, lane, sh.sF[warp], sh.sprobe[warp],
                                                         lists + j * GS_RMAX, Fa, nch, dims, R);
            const auto mq = Z::load(v, w);
            const auto *xq = Z::samples(v, S.x_off + q);
            ZQ *zj = zq + j * zcap;
            for (int r = lane; r < a; r += 32) zj[r] = Z::stage(Z::z(mq, xq[r]));
            float nrm = 0.0f;
            for (int k = 2 * lane; k < kp; k += 64) {
                const float z0 = k < a ? Z::z(mq, xq[k]) : 0.0f;
                const float z1 = k + 1 < a ? Z::z(mq, xq[k + 1]) : 0.0f;
                nrm = fmaf(z0, z0, fmaf(z1, z1, nrm));
                *reinterpret_cast<__half2 *>(tB + sw128_off(j, k, GS_GQ)) = __floats2half2_rn(z0, z1);
            }
            nrm = pn_warp_sum(nrm);
            if (lane == 0) {
                sh.cnt[j] = taken;
                sh.q[j] = (uint32_t)q;
                sh.nq[j] = nrm;
                sh.tq[j] = pn_key_distf(__ldcg(&prow[q]));
                sh.qbest[j] = PN_EMPTY_KEY;
                sh.qn[j] = 0;
                atomicMax(&sh.nqmax, __float_as_int(nrm));
                n_q += 1;
                n_c += (unsigned long long)taken;
            }
        }
        __syncthreads();

        // ---- merge the lists: window -> bit mask of the queries listing it
        for (int e = tid; e < G * GS_RMAX; e += GS_THREADS) {
            const int j = e / GS_RMAX, i = e - j * GS_RMAX;
            if (i >= sh.cnt[j]) continue;
            const uint32_t c = lists[j * GS_RMAX + i];
            uint32_t s = gs_hash(c);
            for (int probe = 0; probe < GS_HT; ++probe) {
                const uint32_t prev = atomicCAS(&htk[s], GS_EMPTY, c);
                if (prev == GS_EMPTY || prev == c) {
                    atomicOr(&htm[s], 1u << j);
                    break;
                }
                s = (s + 1) & (GS_HT - 1);
            }
        }
        __syncthreads();
        // compact the table in slot order into htk/htm[0, nu)
        {
            constexpr int PER = GS_HT / GS_THREADS;
            uint32_t kk[PER], mm[PER];
            int cnt = 0;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                kk[i] = htk[tid * PER + i];
                mm[i] = htm[tid * PER + i];
                cnt += kk[i] != GS_EMPTY ? 1 : 0;
            }
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            __shared__ int wsum[GS_WARPS];
            if (lane == 31) wsum[warp] = incl;
            __syncthreads();                             // every slot is read before any is written
            int base = 0;
            for (int w2 = 0; w2 < warp; ++w2) base += wsum[w2];
            int pos = base + incl - cnt;
#pragma unroll
            for (int i = 0; i < PER; ++i)
                if (kk[i] != GS_EMPTY) {
                    htk[pos] = kk[i];
                    htm[pos] = mm[i];
                    ++pos;
                }
            if (tid == GS_THREADS - 1) sh.nu = pos;
        }
        __syncthreads();
        const int nu = sh.nu;
        const int nq_max_bits = sh.nqmax;

        // ---- tiles of 128 merged windows
        for (int u0 = 0; u0 < nu; u0 += GS_M) {
            const int rows = min(GS_M, nu - u0);
            if (tid < GS_GQ) sh.colmin[tid] = 0x7f800000;
            for (int i = warp; i < rows; i += GS_WARPS) {
                const uint32_t c = htk[u0 + i];
                const auto m = Z::load(v, A.win_off + c);
                const auto *xc = Z::samples(v, S.x_off + c);
                float nrm = 0.0f;
                for (int k = 2 * lane; k < kp; k += 64) {
                    const float z0 = k < a ? Z::z(m, xc[k]) : 0.0f;
                    const float z1 = k + 1 < a ? Z::z(m, xc[k + 1]) : 0.0f;
                    nrm = fmaf(z0, z0, fmaf(z1, z1, nrm));
                    *reinterpret_cast<__half2 *>(tA + sw128_off(i, k, GS_M)) = __floats2half2_rn(z0, z1);
                }
                nrm = pn_warp_sum(nrm);
                if (lane == 0) {
                    sh.nc[i] = nrm;
                    sh.sc[i] = m.x;
                    if (m.x != 0.0f) atomicMax(&sh.ncmax, __float_as_int(nrm));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t a0 = smem_u32(tA), b0 = smem_u32(tB);
                for (int s = 0; s < kp / 16; ++s) {
                    const uint32_t ao = a0 + (uint32_t)((s >> 2) * GS_M * 128 + (s & 3) * 32);
                    const uint32_t bo = b0 + (uint32_t)((s >> 2) * GS_GQ * 128 + (s & 3) * 32);
                    const uint64_t ad = sw128_desc(ao), bd = sw128_desc(bo);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                                 ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&sh.mbar))
                             : "memory");
            }
            if (!mbar_wait(smem_u32(&sh.mbar), phase, GS_SPIN)) {
                if (lane == 0) atomicExch(&sh.fail, 1);
            }
            phase ^= 1u;
            __syncthreads();
            if (sh.fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

            // ---- estimates: warp w reads rows 32 (w mod 4) .. +31, columns 8 (w / 4) .. +7
            const int quarter = warp & 3, half = warp >> 2;
            const int i = quarter * 32 + lane;
            const int j0 = half * 8;
            uint32_t r[8];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(taddr + ((uint32_t)(quarter * 32) << 16) + (uint32_t)j0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const bool valid = i < rows && sh.sc[i] != 0.0f;
            const uint32_t c = valid ? htk[u0 + i] : 0u;
            const uint32_t mk = valid ? ((htm[u0 + i] >> j0) & 0xFFu) : 0u;
            const unsigned long long snap = valid ? __ldcg(&prow[c]) : PN_EMPTY_KEY;
            const float tc = pn_key_distf(snap);
            const float ncv = valid ? sh.nc[i] : 0.0f;
            float dd[8];
            float rmin = inf;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                dd[jj] = inf;
                if ((mk >> jj) & 1u) dd[jj] = fmaxf(0.0f, ncv + sh.nq[j0 + jj] - 2.0f * __uint_as_float(r[jj]));
                rmin = fminf(rmin, dd[jj]);
            }
            sh.rowmin[half][i] = rmin;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                const float m = gs_warp_min(dd[jj]);
                if (lane == 0 && m < inf) atomicMin(&sh.colmin[j0 + jj], __float_as_int(m));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            const float rowmin = fminf(sh.rowmin[0][i], sh.rowmin[1][i]);
            const float ncmax = __int_as_float(sh.ncmax), nqmax = __int_as_float(nq_max_bits);
            const float tol_row = 0.00390625f * (ncv + nqmax);         // 2 M_row, 2^-8 (|z_c|^2 + max |z_q|^2)
            const float tc2 = tc * tc;
            uint32_t bits = 0;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                if (!(dd[jj] < inf)) continue;
                const int j = j0 + jj;
                const float nqj = sh.nq[j];
                const float M = 0.001953125f * (ncv + nqj);              // 2^-9 (|z_c|^2 + |z_q|^2)
                const float tol_col = 0.00390625f * (nqj + ncmax);
                const float tq = sh.tq[j];
                const bool keep_c = dd[jj] - M < tc2 && dd[jj] <= rowmin + tol_row;
                const bool keep_q = dd[jj] - M < tq * tq && dd[jj] <= __int_as_float(sh.colmin[j]) + tol_col;
                if (keep_c || keep_q) bits |= 1u << jj;
            }
            // ---- exact distances of the kept pairs, per query, in rounds of GS_SQ
            while (__syncthreads_or(bits != 0u)) {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    if (!((bits >> jj) & 1u)) continue;
                    const int j = j0 + jj;
                    const int pos = atomicAdd(&sh.qn[j], 1);
                    if (pos < GS_SQ) {
                        qc[j * GS_SQ + pos] = c;
                        qk[j * GS_SQ + pos] = snap;
                        bits &= ~(1u << jj);
                    }
                }
                __syncthreads();
                for (int j = warp; j < G; j += GS_WARPS) {
                    const int n = min(sh.qn[j], GS_SQ);
                    if (n == 0) continue;
                    unsigned long long best = PN_EMPTY_KEY;
                    for (int e = 0; e < n; e += 4)
                        eval_batch<Z>(v, zq + j * zcap, qc + j * GS_SQ + e, qk + j * GS_SQ + e, min(4, n - e), S.x_off,
                                      A.win_off, a, sh.q[j], prow, best, lane);
                    if (lane == 0) {
                        if (best < sh.qbest[j]) {
                            sh.qbest[j] = best;
                            sh.tq[j] = fminf(sh.tq[j], pn_key_distf(best));
                        }
                        n_ex += (unsigned long long)n;
                    }
                }
                __syncthreads();
                if (tid < GS_GQ) sh.qn[tid] = 0;
            }
        }
        if (sh.fail) break;
        __syncthreads();
        if (tid < G && sh.qbest[tid] != PN_EMPTY_KEY) atomicMin(&prow[sh.q[tid]], sh.qbest[tid]);
    }
    __syncthreads();
    if (sh.fail && tid == 0) {
        atomicExch(v.err, PN_ERR_TC_TIMEOUT);
        mbar_wait(smem_u32(&sh.mbar), phase ^ 1u, GS_SPIN);      // an MMA still in flight finishes (bounded)
    }
    if (lane == 0) {
        atomicAdd(&sh.stat[0], n_q);
        atomicAdd(&sh.stat[1], n_c);
        atomicAdd(&sh.stat[2], n_ex);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(GS_TMEM_COLS));
    if (tid == 0 && v.stats) {
        atomicAdd(&v.stats[PN_ST_QUERIES], sh.stat[0]);
        atomicAdd(&v.stats[PN_ST_CANDIDATES], sh.stat[1]);
        atomicAdd(&v.stats[PN_ST_LB_PASSED], sh.stat[2]);
    }
}

inline unsigned gs_grid(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

template <class Z, bool HALF>
cudaError_t gram_t(const PnView &v, const uint32_t *keys, int64_t total, int grid_blocks, int a_max,
                   cudaStream_t st) {
    const int kpad = (a_max + 15) & ~15;
    const int atoms = (kpad + 63) >> 6;
    const int zcap = kpad;
    const size_t sm = 1024 + (size_t)atoms * (GS_M + GS_GQ) * 128 + sizeof(typename Z::Q) * (size_t)GS_GQ * zcap +
                      sizeof(uint32_t) * ((size_t)GS_GQ * GS_RMAX + 2 * GS_HT);
    cudaError_t e = pn_allow_smem(k_search_gram<Z, HALF>, sm);
    if (e != cudaSuccess) return e;
    uint32_t *flag = nullptr, *gstart = nullptr, *cnt = nullptr;
    e = cudaMallocAsync((void **)&flag, sizeof(uint32_t) * (size_t)total, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&gstart, sizeof(uint32_t) * (size_t)total, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cnt, 2 * sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 2 * sizeof(uint32_t), st);
    if (e == cudaSuccess) {
        k_group_flags<<<gs_grid(total, 256), 256, 0, st>>>(keys, total, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(flag, flag, total, cnt, st);
    if (e == cudaSuccess) {
        k_group_fill<<<gs_grid(total, 256), 256, 0, st>>>(keys, flag, total, cnt, gstart);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_search_gram<Z, HALF><<<(unsigned)grid_blocks, GS_THREADS, sm, st>>>(v, keys, total, gstart, cnt, cnt + 1,
                                                                               kpad, zcap);
        e = cudaGetLastError();
    }
    for (void *p : {(void *)flag, (void *)gstart, (void *)cnt})
        if (p) cudaFreeAsync(p, st);
    return e;
}

}  // namespace

bool search_gram_supported(const PnView &v, int a_max) {
    return v.precision == 1 && a_max <= GS_AMAX && v.R <= GS_RMAX;
}

cudaError_t launch_search_gram(const PnView &v, const uint32_t *keys, int64_t total, int sm_count, int a_max,
                               cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    const int grid = 2 * sm_count;
    if (v.Fh)
        return v.x1 ? gram_t<ZMix1, true>(v, keys, total, grid, a_max, st)
                    : gram_t<ZMix2, true>(v, keys, total, grid, a_max, st);
    return v.x1 ? gram_t<ZMix1, false>(v, keys, total, grid, a_max, st)
                : gram_t<ZMix2, false>(v, keys, total, grid, a_max, st);
}

}  // namespace pn
