// Emit stage (Sec. 3.6, Algorithm 2): hot-class sieve, local completion and
// the zero-snapped top-k selection with FP64 re-verification.
#include <algorithm>
#include <type_traits>

#include "distance.cuh"
#include "emit.cuh"
#include "zops.cuh"
#include "evalbatch.cuh"
#include "prims.cuh"

namespace pn {
namespace {

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// Hot classes: buckets of an anchor's final directory (depth(N)) that hold
// more than R entries -- classes no budgeted scan covered (Sec. 3.6).
// ---------------------------------------------------------------------------
__global__ void k_hot_flags(PnView v, const int64_t *slot_off, int64_t total, uint32_t *flag, uint32_t *size,
                            const uint32_t *anchor_on) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int ai = pn_find(slot_off, v.nanchors, t, [](int64_t o) { return o; });
    if (anchor_on && !anchor_on[ai]) {           // an anchor the focused sieve leaves out
        flag[t] = 0;
        size[t] = 0;
        return;
    }
    const PnAnchor &A = v.anchors[ai];
    uint32_t N = A.nw > 0 ? v.cnt[A.win_off + A.nw - 1] : 0u;
    int D = pn_depth(N, v.alpha, v.B);
    int64_t b = t - slot_off[ai];
    uint32_t f = 0, sz = 0;
    if (b < ((int64_t)1 << D)) {
        const PnLevel &L = v.levels[A.level_begin + D];
        int64_t gb = L.bucket_base + b;
        uint32_t c = v.bstart[gb + 1] - v.bstart[gb];
        if ((int)c > v.R) {
            f = 1;
            sz = c;
        }
    }
    flag[t] = f;
    size[t] = sz;
}

__global__ void k_hot_compact(PnView v, const int64_t *slot_off, int64_t total, const uint32_t *flag,
                              const uint32_t *cid, const uint32_t *moff, PnClass *cls) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total || !flag[t]) return;
    int ai = pn_find(slot_off, v.nanchors, t, [](int64_t o) { return o; });
    const PnAnchor &A = v.anchors[ai];
    uint32_t N = A.nw > 0 ? v.cnt[A.win_off + A.nw - 1] : 0u;
    int D = pn_depth(N, v.alpha, v.B);
    const PnLevel &L = v.levels[A.level_begin + D];
    int64_t gb = L.bucket_base + (t - slot_off[ai]);
    PnClass c;
    c.anchor = ai;
    c.lo = v.bstart[gb];
    c.size = v.bstart[gb + 1] - v.bstart[gb];
    c.moff = moff[t];
    cls[cid[t]] = c;
}

// A class's members in directory order, one block per class (the top-k
// sieves order them themselves).
__global__ void k_class_members(PnView v, const PnClass *cls, uint32_t *vals) {
    const PnClass c = cls[blockIdx.x];
    for (uint32_t t = threadIdx.x; t < c.size; t += blockDim.x) vals[(int64_t)c.moff + t] = v.dir_vals[c.lo + t];
}

// Sort key of a member: its projection on the sieve direction g_{a,B+1},
// stored per window by the feature kernel (one 4-byte read, not a row).
__global__ void k_sieve_keys(PnView v, const PnClass *cls, int32_t ncls, int64_t total, uint32_t *keys,
                             uint32_t *vals) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int ci = pn_find(cls, ncls, t, [](const PnClass &c) { return (int64_t)c.moff; });
    const PnClass &c = cls[ci];
    const PnAnchor &A = v.anchors[c.anchor];
    uint32_t x = v.dir_vals[c.lo + (t - c.moff)];
    keys[t] = pn_float_order(v.sproj[A.win_off + x]);
    vals[t] = (uint32_t)t;
}

// After the projection sort: re-key by class (second stable sort) and carry the start.
__global__ void k_sieve_rekey(PnView v, const PnClass *cls, int32_t ncls, int64_t total, uint32_t *keys,
                              uint32_t *vals) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= total) return;
    uint32_t t = vals[p];
    int ci = pn_find(cls, ncls, (int64_t)t, [](const PnClass &c) { return (int64_t)c.moff; });
    const PnClass &c = cls[ci];
    keys[p] = (uint32_t)ci;
    vals[p] = v.dir_vals[c.lo + (t - c.moff)];
}

// One warp per sorted member u: pairs (u, v) with u < v <= u + w (or every
// v > u in the exhaustive variant), valid pairs only (|x_u - x_v| >= excl),
// bound-filtered, exact.  The same machinery as the streaming search: u's
// z-normalised window staged once, bounds of up to 32 neighbours with each
// row read by 8 lanes, threshold tests lane-parallel, survivors evaluated
// four at a time against the staged window, both cells updated.  HALF: rows
// read from the half-precision copy, every bound test with its rounding margin.
template <class Z, bool HALF>
__global__ void __launch_bounds__(256, 3) k_sieve_pairs(PnView v, const PnClass *cls, int64_t total,
                                                        const uint32_t *member_class, const uint32_t *members, int w,
                                                        int exhaustive, int zcap) {
    using ZT = typename Z::T;
    extern __shared__ __align__(16) unsigned char zsm[];
    __shared__ __align__(16) float sF[8][PN_FEAT];
    __shared__ uint32_t scand[8][32];
    __shared__ unsigned long long snap[8][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    typename Z::Q *zu = reinterpret_cast<typename Z::Q *>(zsm) + warp * zcap;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const float shrink = 1.0f - v.lam;
    unsigned long long n_ex = 0;
    for (int64_t p = wid; p < total; p += nwp) {
        const PnClass &c = cls[member_class[p]];
        const PnAnchor &A = v.anchors[c.anchor];
        const PnSeries &S = v.series[A.series];
        const int a = A.a;
        const int64_t u = p - c.moff;
        const int64_t vend = exhaustive ? (int64_t)c.size : min((int64_t)c.size, u + 1 + w);
        if (u + 1 >= vend) continue;
        const uint32_t xu = members[p];
        const auto mu_ = Z::load(v, A.win_off + xu);
        if (Z::degenerate(mu_)) continue;
        const void *Fa = pn_rows<HALF>(v, A.row_off);
        const uint32_t nch = (uint32_t)A.nchunk;
        sF[warp][lane] = pn_row_elem<HALF>(Fa, pn_row32(xu, v.cshift, nch), lane);
        {
            const auto *xs = Z::samples(v, S.x_off + xu);
            for (int r = lane; r < a; r += 32) zu[r] = Z::stage(Z::z(mu_, xs[r]));
        }
        __syncwarp();
        unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
        const float4 fq = reinterpret_cast<const float4 *>(sF[warp])[lane & 7];
        const float lbscale = 2.0f / (float)a;
        const ZT lbmargin = HALF ? (ZT)(shrink * pn_row_margin(v.lb_eps, a)) : (ZT)0;
        unsigned long long bestkey = PN_EMPTY_KEY;
        for (int64_t b0 = u + 1; b0 < vend; b0 += 32) {
            const int nblk = (int)min((int64_t)32, vend - b0);
            // lane l owns neighbour l of the block; rows read by 8-lane groups,
            // partial sums reduced by a transposed butterfly (as in the search)
            uint32_t xv = 0, roff = 0;
            if (lane < nblk) {
                xv = members[c.moff + b0 + lane];
                roff = pn_row32(xv, v.cshift, nch);
            }
            float4 fc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = 4 * j + (lane >> 3);
                const uint32_t ro = __shfl_sync(0xffffffffu, roff, k);
                fc[j] = k < nblk ? pn_row_quad<HALF>(Fa, ro, lane & 7) : fq;
            }
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float dx = fq.x - fc[j].x, dy = fq.y - fc[j].y, dz = fq.z - fc[j].z, dw = fq.w - fc[j].w;
                acc[j] = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, dw * dw)));
            }
            const bool b2 = (lane & 4) != 0, b1 = (lane & 2) != 0, b0l = (lane & 1) != 0;
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
            const float tot = (b0l ? r2[1] : r2[0]) + __shfl_xor_sync(0xffffffffu, b0l ? r2[0] : r2[1], 1);
            const float lbsq = __shfl_sync(0xffffffffu, tot, ((lane & 3) << 3) | (lane >> 2));
            bool surv = false;
            unsigned long long kc = 0;
            if (lane < nblk) {
                if (llabs((int64_t)xv - (int64_t)xu) >= S.excl) {
                    kc = __ldcg(&prow[xv]);
                    const float lbs = shrink * sqrtf(lbscale * lbsq);
                    const ZT tu = Z::fmn(Z::cell(bestkey), Z::cell(__ldcg(&prow[xu])));
                    ZT tt = Z::fmx(tu, Z::cell(kc));
                    if constexpr (HALF) tt += lbmargin;
                    surv = (ZT)lbs < tt;
                }
            }
            const uint32_t sm = __ballot_sync(0xffffffffu, surv);
            if (surv) {
                const int rank = __popc(sm & ((1u << lane) - 1u));
                scand[warp][rank] = xv;
                snap[warp][rank] = kc;
            }
            __syncwarp();
            const int ns = __popc(sm);
            for (int h = 0; h < ns; h += 4)
                eval_batch<Z>(v, zu, scand[warp] + h, snap[warp] + h, min(4, ns - h), S.x_off, A.win_off, a, xu,
                              prow, bestkey, lane);
            n_ex += ns;
            __syncwarp();
        }
        if (lane == 0 && bestkey != PN_EMPTY_KEY) atomicMin(&prow[xu], bestkey);
        __syncwarp();
    }
    if (lane == 0 && v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], n_ex);
}

// ---------------------------------------------------------------------------
// Sieve of the mixed form as a band (Sec. 3.6: pairs within w positions of
// the projected order).  The members of all hot classes lie in one flat
// array sorted by (class, projection); block b takes the 256 members
// b*256 .. b*256+255 as the first element u of its pairs, one per thread,
// and the w members after each as v, so its pairs live in a band of
// 256 + w consecutive members.  Those windows are staged 32 samples at a time
// in shared memory as float4 runs of four consecutive samples (each member
// z-normalised by its own anchor's moments); thread u reads its own run and
// the runs of its w partners, one 16-byte load per window and four samples,
// and keeps the w squared-difference sums in registers, in ascending sample
// order.  Pairs across a class boundary or inside the exclusion zone are
// skipped.  Every band pair is evaluated (no bound test): the cells are the
// minimum over the same pairs the bound-filtered form admits.
// ---------------------------------------------------------------------------
constexpr int SB_U = 256;         // first elements per block, one per thread
constexpr int SB_WMAX = 16;       // widest band of this kernel
constexpr int SB_K = 32;          // samples staged per step
constexpr int SB_ROWS = SB_U + SB_WMAX;

// WC: the band width as a compile-time constant (the default 8), so the
// partner loop unrolls without predicates; 0 takes w at run time.
template <class Z, int WC>
__global__ void __launch_bounds__(SB_U) k_sieve_band(PnView v, const PnClass *cls, int64_t nmem,
                                                     const uint32_t *member_class, const uint32_t *members, int w_rt) {
    constexpr int WMAXC = WC ? WC : SB_WMAX;
    const int w = WC ? WC : w_rt;
    // row stride of SB_ROWS + 1 float4 (4 mod 32 words): the staging stores of
    // 8 lanes (one row, 8 runs) fall in distinct banks
    __shared__ float4 zs[SB_K / 4][SB_ROWS + 1];
    __shared__ uint32_t s_x[SB_ROWS], s_cls[SB_ROWS];
    __shared__ int32_t s_a[SB_ROWS];
    __shared__ float2 s_m[SB_ROWS];
    __shared__ const typename Z::X *s_xp[SB_ROWS];   // first sample of each row's window
    __shared__ unsigned long long colmin[SB_ROWS];
    __shared__ int s_amax;
    __shared__ unsigned long long s_ex;
    const int tid = threadIdx.x;
    const int nrow = SB_U + w;
    if (tid == 0) s_ex = 0;
    for (int64_t b = blockIdx.x; b * SB_U < nmem; b += gridDim.x) {
        const int64_t p0 = b * SB_U;
        __syncthreads();
        if (tid == 0) s_amax = 0;
        __syncthreads();
        for (int row = tid; row < nrow; row += SB_U) {
            const int64_t p = p0 + row;
            uint32_t x = 0, ci = 0xFFFFFFFFu;
            int a = 0;
            float2 m = make_float2(0.0f, 0.0f);
            const typename Z::X *xp = nullptr;
            if (p < nmem) {
                ci = member_class[p];
                x = members[p];
                const PnAnchor &A = v.anchors[cls[ci].anchor];
                a = A.a;
                const auto mm = Z::load(v, A.win_off + x);
                m = make_float2(mm.x, mm.y);
                xp = Z::samples(v, v.series[A.series].x_off + x);
                atomicMax(&s_amax, a);
            }
            s_x[row] = x;
            s_cls[row] = ci;
            s_a[row] = a;
            s_m[row] = m;
            s_xp[row] = xp;
            colmin[row] = PN_EMPTY_KEY;
        }
        __syncthreads();
        const int amax = s_amax;
        float acc[WMAXC];
#pragma unroll
        for (int j = 0; j < WMAXC; ++j) acc[j] = 0.0f;
        for (int k0 = 0; k0 < amax; k0 += SB_K) {
            // run e: samples k0 + 4 (e & 7) .. + 3 of row e >> 3; zero past the window
            for (int e = tid; e < nrow * (SB_K / 4); e += SB_U) {
                const int row = e >> 3, q4 = e & 7;
                const int k = k0 + 4 * q4;
                const int a = s_a[row];
                float4 z = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (k < a) {
                    typename Z::M mm;
                    mm.x = s_m[row].x;
                    mm.y = s_m[row].y;
                    const typename Z::X *xp = s_xp[row] + k;
                    z.x = Z::z(mm, xp[0]);
                    if (k + 1 < a) z.y = Z::z(mm, xp[1]);
                    if (k + 2 < a) z.z = Z::z(mm, xp[2]);
                    if (k + 3 < a) z.w = Z::z(mm, xp[3]);
                }
                zs[q4][row] = z;
            }
            __syncthreads();
#pragma unroll 2
            for (int q4 = 0; q4 < SB_K / 4; ++q4) {
                const float4 zu = zs[q4][tid];
#pragma unroll
                for (int j = 0; j < WMAXC; ++j) {
                    if (WC || j < w) {
                        const float4 zv = zs[q4][tid + 1 + j];
                        float d = zu.x - zv.x;
                        acc[j] = fmaf(d, d, acc[j]);
                        d = zu.y - zv.y;
                        acc[j] = fmaf(d, d, acc[j]);
                        d = zu.z - zv.z;
                        acc[j] = fmaf(d, d, acc[j]);
                        d = zu.w - zv.w;
                        acc[j] = fmaf(d, d, acc[j]);
                    }
                }
            }
            __syncthreads();
        }
        // u's own cell: the minimum over its w pairs; each partner's through
        // shared memory, flushed once per row
        unsigned long long n_here = 0;
        if (p0 + tid < nmem && s_m[tid].x != 0.0f) {
            const uint32_t cu = s_cls[tid];
            const PnAnchor &A = v.anchors[cls[cu].anchor];
            const PnSeries &S = v.series[A.series];
            const uint32_t xu = s_x[tid];
            unsigned long long ku = PN_EMPTY_KEY;
#pragma unroll
            for (int j = 0; j < WMAXC; ++j) {
                const int vv = tid + 1 + j;
                if ((WC || j < w) && p0 + vv < nmem && s_cls[vv] == cu && s_m[vv].x != 0.0f &&
                    llabs((int64_t)xu - (int64_t)s_x[vv]) >= S.excl) {
                    const float d = sqrtf(acc[j]);
                    const unsigned long long kv = pn_pack_f(d, s_x[vv]);
                    ku = kv < ku ? kv : ku;
                    atomicMin(&colmin[vv], pn_pack_f(d, xu));
                    ++n_here;
                }
            }
            if (ku != PN_EMPTY_KEY) atomicMin(&v.prof[S.row_off + (int64_t)(A.a - S.m_min) * S.ld + xu], ku);
        }
        if (n_here) atomicAdd(&s_ex, n_here);
        __syncthreads();
        for (int row = tid; row < nrow; row += SB_U) {
            if (p0 + row < nmem && colmin[row] != PN_EMPTY_KEY) {
                const PnAnchor &A = v.anchors[cls[s_cls[row]].anchor];
                const PnSeries &S = v.series[A.series];
                atomicMin(&v.prof[S.row_off + (int64_t)(A.a - S.m_min) * S.ld + s_x[row]], colmin[row]);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && v.stats && s_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], s_ex);
}

// ---------------------------------------------------------------------------
// Exhaustive sieve, mixed form: every valid pair of every hot class (the
// wide variant of S_hot, Sec. 3.6), as a tiled all-pairs computation.  A
// class of s members is cut into 64-member blocks; block pair (bu, bv),
// bu <= bv, is one tile of 64 x 64 pairs.  The tile's z-normalised windows
// are staged 32 samples at a time in shared memory and each thread
// accumulates 4 x 4 squared differences in registers, so every staged
// sample feeds 64 pairs instead of one.  Both cells of every valid pair
// take the distance (row minima by shuffles, column minima through shared
// memory, then atomicMin).  No bound test is needed: every pair is
// evaluated, so the result is the minimum over all of them.
// ---------------------------------------------------------------------------
constexpr int ST_B = 64;          // members per tile side
constexpr int ST_K = 32;          // samples staged per step

// Tiles per class; a class above 2^31 tiles, or a total above 2^31, sets
// *overflow and the launcher refuses the request (no truncated table).
__global__ void k_tile_count(const PnClass *cls, int32_t ncls, uint32_t *cnt, unsigned long long *total,
                             int *overflow) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncls) return;
    const uint64_t nb = (cls[ci].size + ST_B - 1) / ST_B;
    const uint64_t t = nb * (nb + 1) / 2;
    if (t > 0x7FFFFFFFull) {
        atomicExch(overflow, 1);
        cnt[ci] = 0;
        return;
    }
    cnt[ci] = (uint32_t)t;
    atomicAdd(total, (unsigned long long)t);
}

// One warp per class writes its tiles (class, bu, bv) at the class's offset.
__global__ void k_tile_fill(const PnClass *cls, int32_t ncls, const uint32_t *off, uint32_t *tiles) {
    const int ci = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (ci >= ncls) return;
    const uint32_t nb = (cls[ci].size + ST_B - 1) / ST_B;
    const uint32_t total = (uint32_t)(((uint64_t)nb * (nb + 1)) / 2);
    for (uint32_t t = lane; t < total; t += 32) {
        // row bu holds nb - bu tiles; bu of the t-th tile by bisection
        const uint32_t bu = tri_row(t, nb);
        const uint32_t bv = bu + (t - (uint32_t)((uint64_t)bu * nb - ((uint64_t)bu * (bu - 1)) / 2));
        uint4 *dst = reinterpret_cast<uint4 *>(tiles) + (int64_t)off[ci] + t;
        *dst = make_uint4((uint32_t)ci, bu, bv, 0u);
    }
}

template <class Z>
__global__ void __launch_bounds__(256) k_sieve_tiles(PnView v, const PnClass *cls, const uint4 *tiles,
                                                     int64_t ntiles, const uint32_t *members) {
    __shared__ float zu[ST_K][ST_B + 1];
    __shared__ float zv[ST_K][ST_B + 1];
    __shared__ uint32_t su[ST_B], sv[ST_B];
    __shared__ float2 mu_u[ST_B], mu_v[ST_B];
    __shared__ unsigned long long colmin[ST_B];
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    unsigned long long n_ex = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint4 tl = tiles[t];
        const PnClass &c = cls[tl.x];
        const PnAnchor &A = v.anchors[c.anchor];
        const PnSeries &S = v.series[A.series];
        const int a = A.a;
        const int u0 = (int)tl.y * ST_B, v0 = (int)tl.z * ST_B;
        const int nu = min(ST_B, (int)c.size - u0), nv = min(ST_B, (int)c.size - v0);
        __syncthreads();                                    // the previous tile's staging is no longer read
        if (tid < ST_B) {
            const uint32_t xu = tid < nu ? members[c.moff + u0 + tid] : 0u;
            const uint32_t xv = tid < nv ? members[c.moff + v0 + tid] : 0u;
            su[tid] = xu;
            sv[tid] = xv;
            const auto mu = Z::load(v, A.win_off + xu), mv = Z::load(v, A.win_off + xv);
            mu_u[tid] = tid < nu ? make_float2(mu.x, mu.y) : make_float2(0.0f, 0.0f);
            mu_v[tid] = tid < nv ? make_float2(mv.x, mv.y) : make_float2(0.0f, 0.0f);
            colmin[tid] = PN_EMPTY_KEY;
        }
        __syncthreads();
        float acc[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
        const auto *xs = Z::samples(v, S.x_off);
        for (int k0 = 0; k0 < a; k0 += ST_K) {
            // stage: 64 windows x 32 samples per side, z = fma(x, 1/sigma, -mu/sigma)
            for (int e = tid; e < ST_B * ST_K; e += blockDim.x) {
                const int row = e / ST_K, r = e - row * ST_K;
                const int k = k0 + r;
                float a_ = 0.0f, b_ = 0.0f;
                if (k < a) {
                    const float2 m1 = mu_u[row], m2 = mu_v[row];
                    typename Z::M z1, z2;
                    z1.x = m1.x;
                    z1.y = m1.y;
                    z2.x = m2.x;
                    z2.y = m2.y;
                    if (row < nu) a_ = Z::z(z1, xs[su[row] + k]);
                    if (row < nv) b_ = Z::z(z2, xs[sv[row] + k]);
                }
                zu[r][row] = a_;
                zv[r][row] = b_;
            }
            __syncthreads();
#pragma unroll 8
            for (int r = 0; r < ST_K; ++r) {
                float pu[4], pv[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    pu[i] = zu[r][ty * 4 + i];
                    pv[i] = zv[r][tx * 4 + i];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const float d = pu[i] - pv[j];
                        acc[i][j] = fmaf(d, d, acc[i][j]);
                    }
            }
            __syncthreads();
        }
        // keys of the valid pairs: row minima by shuffles, column minima in shared memory
        const bool diag = tl.y == tl.z;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ur = ty * 4 + i;
            unsigned long long rowk = PN_EMPTY_KEY;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int vc = tx * 4 + j;
                bool ok = ur < nu && vc < nv && (!diag || ur < vc) && mu_u[ur].x != 0.0f && mu_v[vc].x != 0.0f;
                if (ok) ok = llabs((int64_t)su[ur] - (int64_t)sv[vc]) >= S.excl;
                if (ok) {
                    const float d = sqrtf(acc[i][j]);
                    const unsigned long long ku = pn_pack_f(d, sv[vc]), kv = pn_pack_f(d, su[ur]);
                    rowk = ku < rowk ? ku : rowk;
                    atomicMin(&colmin[vc], kv);
                    ++n_ex;
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, rowk, o);
                rowk = other < rowk ? other : rowk;
            }
            if (tx == 0 && rowk != PN_EMPTY_KEY) {
                unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
                atomicMin(&prow[su[ur]], rowk);
            }
        }
        __syncthreads();
        if (tid < nv && colmin[tid] != PN_EMPTY_KEY) {
            unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
            atomicMin(&prow[sv[tid]], colmin[tid]);
        }
    }
    // counts per block
    __shared__ unsigned long long s_ex;
    if (tid == 0) s_ex = 0;
    __syncthreads();
    if (n_ex) atomicAdd(&s_ex, n_ex);
    __syncthreads();
    if (tid == 0 && v.stats && s_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], s_ex);
}

// ---------------------------------------------------------------------------
// Local completion (Sec. 3.6): for each seed (m0, i0, j0) every admissible
// (m, i, j) with |m-m0| <= dm, |i-i0| <= dp, |j-j0| <= dp, |i-j| >= excl is
// evaluated exactly; both cells take the distance, and the partner written
// is the hint later rounds re-cut from.  One block (8 warps) per seed.  The
// box's (2dm+1)(2dp+1) windows on each side are normalised once into shared
// memory (FP64 moments), then every triple reads its two windows from there.
// ---------------------------------------------------------------------------
__global__ void k_complete(PnView v, const PnSeed *seeds, int32_t nseeds_max, const int32_t *nseeds_dev, int dm,
                           int dp, int *improved) {
    if (pn_gated(v)) return;
    const int32_t nseeds = nseeds_dev ? min(*nseeds_dev, nseeds_max) : nseeds_max;
    extern __shared__ __align__(16) unsigned char csm[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int side = 2 * dp + 1;
    const int nwin = (2 * dm + 1) * side;
    PnWin *win_i = reinterpret_cast<PnWin *>(csm);
    PnWin *win_j = win_i + nwin;
    unsigned long long n_ex = 0;
    int imp = 0;
    for (int sd = blockIdx.x; sd < nseeds; sd += gridDim.x) {
        const PnSeed sdv = seeds[sd];
        const int s = sdv.series;
        const PnSeries &S = v.series[s];
        const int ntrip = (2 * dm + 1) * side * side;
        __syncthreads();                                   // the previous seed's windows are no longer read
        for (int t = threadIdx.x; t < 2 * nwin; t += blockDim.x) {
            const int k = t < nwin ? t : t - nwin;
            const int m = sdv.m + k / side - dm;
            const int64_t p = (t < nwin ? sdv.i : sdv.j) + k % side - dp;
            PnWin w;
            w.mu = 0.0;
            w.inv = 0.0;
            w.mu_hi = w.mu_lo = w.invf = 0.0f;
            if (m >= S.m_min && m <= S.m_max && p >= 0 && p <= S.n - m) w = pn_window(v, s, p, m);
            (t < nwin ? win_i : win_j)[k] = w;
        }
        __syncthreads();
        for (int t = warp; t < ntrip; t += nwarps) {
            const int tm = t / (side * side);
            const int rem = t - tm * side * side;
            const int m = sdv.m + tm - dm;
            const int64_t i = sdv.i + rem / side - dp;
            const int64_t j = sdv.j + rem % side - dp;
            if (m < S.m_min || m > S.m_max) continue;
            if (i < 0 || j < 0 || i > S.n - m || j > S.n - m) continue;
            if (llabs(i - j) < S.excl) continue;
            if (v.runlen[S.x_off + i] >= m || v.runlen[S.x_off + j] >= m) continue;
            const PnWin wi = win_i[tm * side + rem / side];
            const PnWin wj = win_j[tm * side + rem % side];
            const double dd = pn_dist_warp(v, S.x_off, m, i, wi, j, wj, lane);
            n_ex += 1;
            if (lane == 0 && dd < __longlong_as_double(0x7ff0000000000000ll)) {
                unsigned long long *row = v.prof + S.row_off + (int64_t)(m - S.m_min) * S.ld;
                const unsigned long long ki = pn_pack(dd, (uint32_t)j), kj = pn_pack(dd, (uint32_t)i);
                if (atomicMin(&row[i], ki) > ki) imp = 1;
                if (atomicMin(&row[j], kj) > kj) imp = 1;
            }
        }
    }
    if (lane == 0) {
        if (imp) atomicExch(improved, 1);
        if (v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_COMPLETION], n_ex);
    }
}

// ---------------------------------------------------------------------------
// Top-k selection (Sec. 2, Algorithm 2 last step).
//
// A selection group is one series (global mode) or one length row of a
// series (per-length mode).  Each accepted cell suppresses at most m+1 cells
// of its length, so the first k accepted cells lie among the k(m_max+1)
// smallest cells: a two-level radix select on the key bits picks a
// threshold covering that many cells (plus one bin of slack for the
// in-stream rounding), the cells under it are pooled, their distances are
// recomputed in FP64 from two-pass moments, snapped to 0 below eps0, sorted
// by (d, m, i) and scanned greedily under the m/2 rule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sel_bits(unsigned long long key, double eps0, int level) {
    double d = pn_key_dist(key);
    unsigned long long b = d < eps0 ? 0ull : (key & ~PN_IDX_MASK);
    return level == 0 ? (uint32_t)(b >> 51) & 0xFFFu : (uint32_t)(b >> 39) & 0xFFFu;
}

__device__ __forceinline__ int group_of(const PnView &v, const PnSelGroup *grp, int32_t ngrp, int64_t cell) {
    return pn_find(grp, ngrp, cell, [](const PnSelGroup &g) { return g.cell_off; });
}

// Histogram of the level-0 (or, within the level-0 bin b1, level-1) key
// bits of every group.  Block b takes the contiguous cells
// [b per_block, (b+1) per_block); the groups tile the cell space, so the
// range splits into a few group segments, each counted in a shared-memory
// histogram (warp-aggregated atomics) and flushed once to the group's
// global histogram.
__global__ void __launch_bounds__(256) k_sel_hist(PnView v, const PnSelGroup *grp, int32_t ngrp, int64_t total,
                                                  double eps0, int level, const uint32_t *b1, uint32_t *hist,
                                                  int64_t per_block) {
    if (pn_gated(v)) return;
    __shared__ uint32_t sh[4096];
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int64_t hi = min(total, lo + per_block);
    int64_t t0 = lo;
    while (t0 < hi) {
        const int gi = group_of(v, grp, ngrp, t0);
        const int64_t gend = grp[gi].cell_off + grp[gi].ncell;
        const int64_t seg_end = gend > t0 ? min(hi, gend) : min(hi, gi + 1 < ngrp ? grp[gi + 1].cell_off : hi);
        const bool in_group = gend > t0;
        for (int b = threadIdx.x; b < 4096; b += blockDim.x) sh[b] = 0u;
        __syncthreads();
        const uint32_t want = (in_group && level == 1) ? b1[gi] : 0u;
        // four independent coalesced key loads in flight per thread
        for (int64_t base = t0; base < seg_end; base += 4 * (int64_t)blockDim.x) {
            unsigned long long key[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t t = base + threadIdx.x + (int64_t)u * blockDim.x;
                key[u] = (in_group && t < seg_end) ? __ldcs(&v.prof[t]) : PN_EMPTY_KEY;
            }
            // warp-aggregated counts, one distinct bin per step: the keys of a
            // warp fall in few bins (level 0 is mostly the distance's
            // exponent; level 1 counts only the keys inside bin b1)
            const int lane = threadIdx.x & 31;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                bool ok = key[u] != PN_EMPTY_KEY;
                if (ok && level == 1) ok = sel_bits(key[u], eps0, 0) == want;
                const uint32_t bin = ok ? sel_bits(key[u], eps0, level) : 0u;
                unsigned pending = __ballot_sync(0xffffffffu, ok);
                while (pending) {
                    const int leader = __ffs(pending) - 1;
                    const uint32_t b = __shfl_sync(0xffffffffu, bin, leader);
                    const unsigned same = __ballot_sync(0xffffffffu, ok && bin == b);
                    if (lane == leader) atomicAdd(&sh[b], (uint32_t)__popc(same));
                    pending &= ~same;
                }
            }
        }
        __syncthreads();
        if (in_group)
            for (int b = threadIdx.x; b < 4096; b += blockDim.x)
                if (sh[b]) atomicAdd(&hist[(int64_t)gi * 4096 + b], sh[b]);
        __syncthreads();
        t0 = seg_end > t0 ? seg_end : hi;
    }
}

// One warp per group: the first bin whose cumulative count (after carry_in)
// reaches `need`, and the count below it; bin 4095 and the full count when
// no bin does.  Lane l sums bins [128 l, 128 l + 128) with 16-byte loads, a
// warp scan of the lane sums finds the lane whose range crosses `need`, and
// that lane's bins are scanned 32 at a time.
__global__ void k_sel_pick(const PnSelGroup *grp, int32_t ngrp, const uint32_t *hist, const uint32_t *carry_in,
                           uint32_t *bin_out, uint32_t *carry_out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int gi = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (gi >= ngrp) return;                                // warp-uniform
    const uint32_t need = grp[gi].need;
    const uint32_t run0 = carry_in ? carry_in[gi] : 0u;
    const uint32_t *hg = hist + (int64_t)gi * 4096;
    const uint4 *h4 = reinterpret_cast<const uint4 *>(hg) + lane * 32;
    uint32_t s = 0;
#pragma unroll 8
    for (int q = 0; q < 32; ++q) {
        const uint4 u = h4[q];
        s += u.x + u.y + u.z + u.w;
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
    }
    const unsigned hit = __ballot_sync(full, run0 + incl >= need);
    uint32_t b = 4095, carry = run0 + __shfl_sync(full, incl, 31);
    if (hit) {
        const int L = __ffs(hit) - 1;
        uint32_t base = run0 + __shfl_sync(full, incl - s, L);
        for (int c = 0; c < 4; ++c) {
            const uint32_t val = hg[128 * L + 32 * c + lane];
            uint32_t in2 = val;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(full, in2, o);
                if (lane >= o) in2 += y;
            }
            const unsigned h2 = __ballot_sync(full, base + in2 >= need);
            if (h2) {
                const int L2 = __ffs(h2) - 1;
                b = (uint32_t)(128 * L + 32 * c + L2);
                carry = base + __shfl_sync(full, in2 - val, L2);
                break;
            }
            base += __shfl_sync(full, in2, 31);
        }
    }
    if (lane == 0) {
        bin_out[gi] = b;
        if (carry_out) carry_out[gi] = carry;
    }
}

__global__ void k_sel_pool(PnView v, const PnSelGroup *grp, int32_t ngrp, int64_t total, double eps0,
                           const uint32_t *b1, const uint32_t *b2, PnPoolEntry *pool, uint32_t *pool_cnt,
                           int32_t cap, int *overflow) {
    if (pn_gated(v)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const unsigned long long key = v.prof[t];
        if (key == PN_EMPTY_KEY) continue;
        const int gi = group_of(v, grp, ngrp, t);
        if (t >= grp[gi].cell_off + grp[gi].ncell) continue;
        const uint32_t h = (sel_bits(key, eps0, 0) << 12) | sel_bits(key, eps0, 1);
        const uint32_t thr = (b1[gi] << 12) | b2[gi];
        if (h > thr + 1u) continue;
        const uint32_t slot = atomicAdd(&pool_cnt[gi], 1u);
        if ((int32_t)slot >= cap) {
            atomicExch(overflow, 1);
            continue;
        }
        PnPoolEntry e;
        e.cell = (uint32_t)(t - grp[gi].cell_off);
        e.j = pn_key_idx(key);
        e.d = pn_key_dist(key);
        pool[(int64_t)gi * cap + slot] = e;
    }
}

// FP64 two-pass distance of every pooled cell (one warp per entry).
__global__ void k_sel_verify(PnView v, const PnSelGroup *grp, int32_t ngrp, PnPoolEntry *pool,
                             const uint32_t *pool_cnt, int32_t cap, double eps0) {
    if (pn_gated(v)) return;
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t total = (int64_t)ngrp * cap;
    for (int64_t e = wid; e < total; e += nwp) {
        const int gi = (int)(e / cap);
        const int slot = (int)(e - (int64_t)gi * cap);
        if (slot >= (int)min(pool_cnt[gi], (uint32_t)cap)) continue;
        const PnSelGroup &G = grp[gi];
        const PnSeries &S = v.series[G.series];
        PnPoolEntry &pe = pool[e];
        const int64_t cell = (int64_t)pe.cell + (G.cell_off - S.row_off);
        const int m = S.m_min + (int)(cell / S.ld);
        // both cells of a pair get bit-identical values: evaluate in (min, max) order
        const int64_t c0 = cell % S.ld, c1 = pe.j;
        const int64_t i = c0 < c1 ? c0 : c1, j = c0 < c1 ? c1 : c0;
        const double *xi = v.x + S.x_off + i, *xj = v.x + S.x_off + j;
        double si = 0, sj = 0;
        for (int r = lane; r < m; r += 32) {
            si += xi[r];
            sj += xj[r];
        }
        const double mi = pn_warp_sumd(si) / m, mj = pn_warp_sumd(sj) / m;
        double qi = 0, qj = 0;
        for (int r = lane; r < m; r += 32) {
            qi += (xi[r] - mi) * (xi[r] - mi);
            qj += (xj[r] - mj) * (xj[r] - mj);
        }
        const double ii = 1.0 / sqrt(pn_warp_sumd(qi) / m), ij = 1.0 / sqrt(pn_warp_sumd(qj) / m);
        double acc = 0;
        for (int r = lane; r < m; r += 32) {
            const double dz = (xi[r] - mi) * ii - (xj[r] - mj) * ij;
            acc += dz * dz;
        }
        const double d = sqrt(pn_warp_sumd(acc));
        if (lane == 0) pe.d = d < eps0 ? 0.0 : d;
    }
}

__device__ __forceinline__ bool pool_less(const PnPoolEntry &a, const PnPoolEntry &b) {
    return a.d < b.d || (a.d == b.d && a.cell < b.cell);
}

// One block per group: bitonic sort of the pool in shared memory, then a
// greedy scan by warp 0 under the m/2 rule.
__global__ void k_sel_greedy(PnView v, const PnSelGroup *grp, const PnPoolEntry *pool, const uint32_t *pool_cnt,
                             int32_t cap, int32_t npow2, PnPick *out, int32_t *out_cnt, int32_t kmax) {
    if (pn_gated(v)) return;
    extern __shared__ __align__(16) unsigned char smem[];
    PnPoolEntry *e = reinterpret_cast<PnPoolEntry *>(smem);
    int32_t *acc_m = reinterpret_cast<int32_t *>(e + npow2);
    int64_t *acc_i = reinterpret_cast<int64_t *>(acc_m + kmax + (kmax & 1));
    const int gi = blockIdx.x;
    const PnSelGroup G = grp[gi];
    const PnSeries &S = v.series[G.series];
    const int cnt = (int)min(pool_cnt[gi], (uint32_t)cap);
    for (int t = threadIdx.x; t < npow2; t += blockDim.x) {
        if (t < cnt) {
            e[t] = pool[(int64_t)gi * cap + t];
        } else {
            e[t].d = __longlong_as_double(0x7ff0000000000000ll);
            e[t].cell = 0xFFFFFFFFu;
            e[t].j = 0;
        }
    }
    __syncthreads();
    // bitonic network: each stage's npow2/2 compare-exchanges enumerated
    // directly (the lower index t of pair i has bit jj clear), no idle half
    for (int kk = 2; kk <= npow2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < (npow2 >> 1); i += blockDim.x) {
                const int t = ((i & ~(jj - 1)) << 1) | (i & (jj - 1));
                const int p = t | jj;
                const bool up = (t & kk) == 0;
                PnPoolEntry A = e[t], Bv = e[p];
                if (pool_less(Bv, A) == up) {
                    e[t] = Bv;
                    e[p] = A;
                }
            }
            __syncthreads();
        }
    }
    // Greedy suppression in pool order, 32 entries at a time: each lane
    // decodes one entry and tests it against the cells accepted before the
    // chunk; then the chunk is resolved in order, an accepted entry marking
    // the later lanes it suppresses.  An entry is accepted exactly when the
    // one-at-a-time scan would accept it.
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int nacc = 0;
        const int k = min(G.k, kmax);
        const int64_t base = G.cell_off - S.row_off;
        for (int t0 = 0; t0 < cnt && nacc < k; t0 += 32) {
            const int t = t0 + lane;
            int m = 0;
            int64_t i = 0;
            bool clash = t >= cnt;
            if (!clash) {
                const int64_t cell = base + e[t].cell;
                m = S.m_min + (int)(cell / S.ld);
                i = cell % S.ld;
                for (int u = 0; u < nacc; ++u)
                    if (acc_m[u] == m && 2 * llabs(i - acc_i[u]) <= m) clash = true;
            }
            for (int l = 0; l < 32 && nacc < k; ++l) {
                if (__shfl_sync(0xffffffffu, clash ? 1 : 0, l)) continue;
                const int ml = __shfl_sync(0xffffffffu, m, l);
                const int64_t il = __shfl_sync(0xffffffffu, i, l);
                if (lane == 0) {
                    acc_m[nacc] = ml;
                    acc_i[nacc] = il;
                    PnPick pk;
                    pk.series = G.series;
                    pk.m = ml;
                    pk.i = il;
                    pk.j = e[t0 + l].j;
                    pk.d = e[t0 + l].d;
                    out[(int64_t)gi * kmax + nacc] = pk;
                }
                ++nacc;
                if (lane > l && m == ml && 2 * llabs(i - il) <= m) clash = true;
            }
            __syncwarp();
        }
        if (lane == 0) out_cnt[gi] = nacc;
    }
}

template <class Z>
cudaError_t sieve_band_t(const PnView &v, const PnClass *cls, int64_t nmem, const uint32_t *keys,
                         const uint32_t *vals, int w, int grid_blocks, cudaStream_t st) {
    const int64_t need = (nmem + SB_U - 1) / SB_U;
    const int64_t g = std::min<int64_t>(need, (int64_t)grid_blocks * 2);
    if (w == 8) k_sieve_band<Z, 8><<<(unsigned)g, SB_U, 0, st>>>(v, cls, nmem, keys, vals, w);
    else k_sieve_band<Z, 0><<<(unsigned)g, SB_U, 0, st>>>(v, cls, nmem, keys, vals, w);
    return cudaGetLastError();
}

// Exhaustive sieve of the mixed form: tile table, then the tiled all-pairs kernel.
template <class Z>
cudaError_t sieve_tiles_t(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int grid_blocks,
                          cudaStream_t st) {
    uint32_t *cnt = nullptr, *off = nullptr, *tot = nullptr, *tiles = nullptr;
    unsigned long long *tot64 = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&cnt, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&off, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot, 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot64, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tot64, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_tile_count<<<grid_for(ncls, 256), 256, 0, st>>>(cls, ncls, cnt, tot64, reinterpret_cast<int *>(tot64 + 1));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(cnt, off, ncls, tot, st);
    unsigned long long h64[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h64, tot64, sizeof(h64), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && (h64[1] != 0ull || h64[0] > 0x7FFFFFFFull)) e = cudaErrorMemoryAllocation;
    const uint32_t ntiles = e == cudaSuccess ? (uint32_t)h64[0] : 0u;
    if (e == cudaSuccess && ntiles > 0) e = cudaMallocAsync((void **)&tiles, sizeof(uint4) * (size_t)ntiles, st);
    if (e == cudaSuccess && ntiles > 0) {
        k_tile_fill<<<grid_for((int64_t)ncls * 32, 256), 256, 0, st>>>(cls, ncls, off, tiles);
        const int64_t g = std::min<int64_t>((int64_t)ntiles, (int64_t)grid_blocks);
        k_sieve_tiles<Z><<<(unsigned)g, 256, 0, st>>>(v, cls, reinterpret_cast<const uint4 *>(tiles), ntiles, vals);
        e = cudaGetLastError();
    }
    for (void *p : {(void *)cnt, (void *)off, (void *)tot, (void *)tot64, (void *)tiles})
        if (p) cudaFreeAsync(p, st);
    return e;
}

template <class Z, bool HALF>
cudaError_t sieve_pairs_t(const PnView &v, const PnClass *cls, int64_t nmem, const uint32_t *keys,
                          const uint32_t *vals, int w, int exhaustive, int zcap, int64_t blocks, cudaStream_t st) {
    const size_t sm = sizeof(typename Z::Q) * zcap * 8;
    cudaError_t e = pn_allow_smem(k_sieve_pairs<Z, HALF>, sm);
    if (e != cudaSuccess) return e;
    k_sieve_pairs<Z, HALF><<<(unsigned)blocks, 256, sm, st>>>(v, cls, nmem, keys, vals, w, exhaustive, zcap);
    return cudaGetLastError();
}

// Per-member sieve: the plain form always, the mixed form for bands wider
// than the band kernel's; half rows only occur in the mixed form.
template <class Z>
cudaError_t sieve_t(const PnView &v, const PnClass *cls, int64_t nmem, const uint32_t *keys, const uint32_t *vals,
                    int w, int exhaustive, int zcap, int64_t blocks, cudaStream_t st) {
    if constexpr (!std::is_same<Z, ZPlain>::value)
        if (v.Fh) return sieve_pairs_t<Z, true>(v, cls, nmem, keys, vals, w, exhaustive, zcap, blocks, st);
    return sieve_pairs_t<Z, false>(v, cls, nmem, keys, vals, w, exhaustive, zcap, blocks, st);
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t launch_sieve(const PnView &v, const int64_t *slot_off_dev, int64_t total_slots, int w, int exhaustive,
                         int grid_blocks, int a_max, cudaStream_t st, int32_t *n_classes_out, const float *topk_thr,
                         const uint32_t *focus_anchors, int *improved) {
    *n_classes_out = 0;
    if (total_slots <= 0) return cudaSuccess;
    uint32_t *flag = nullptr, *size = nullptr, *cid = nullptr, *moff = nullptr, *tot = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&flag, 4 * total_slots, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&size, 4 * total_slots, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&cid, 4 * total_slots, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&moff, 4 * total_slots, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot, 8, st);
    if (e == cudaSuccess) {
        k_hot_flags<<<grid_for(total_slots, 256), 256, 0, st>>>(v, slot_off_dev, total_slots, flag, size,
                                                                topk_thr ? focus_anchors : nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(flag, cid, total_slots, tot, st);
    if (e == cudaSuccess) e = excl_scan_u32(size, moff, total_slots, tot + 1, st);
    uint32_t h_tot[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_tot, tot, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int32_t ncls = (int32_t)h_tot[0];
    const int64_t nmem = (int64_t)h_tot[1];
    bool topk_done = false;
    PnClass *cls = nullptr;
    uint32_t *keys = nullptr, *vals = nullptr;
    if (e == cudaSuccess && ncls > 0) {
        e = cudaMallocAsync((void **)&cls, sizeof(PnClass) * ncls, st);
        if (e == cudaSuccess && !topk_thr) e = cudaMallocAsync((void **)&keys, 4 * nmem, st);
        if (e == cudaSuccess) e = cudaMallocAsync((void **)&vals, 4 * nmem, st);
        if (e == cudaSuccess) {
            k_hot_compact<<<grid_for(total_slots, 256), 256, 0, st>>>(v, slot_off_dev, total_slots, flag, cid, moff,
                                                                      cls);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && topk_thr) {
            // the top-k sieves: members in directory order, no sort-key order
            k_class_members<<<(unsigned)ncls, 256, 0, st>>>(v, cls, vals);
            e = cudaGetLastError();
            pn_kt_begin(v.kt, PN_KT_TOPK, st);
            if (e == cudaSuccess)
                e = launch_sieve_gram(v, cls, ncls, vals, nmem, a_max, grid_blocks, st, topk_thr, improved);
            pn_kt_end(v.kt, PN_KT_TOPK, st);
            topk_done = true;
        }
        if (e == cudaSuccess && !topk_done) {
            k_sieve_keys<<<grid_for(nmem, 256), 256, 0, st>>>(v, cls, ncls, nmem, keys, vals);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess && !topk_done) e = radix_sort_pairs(keys, vals, nmem, 32, st);
        if (e == cudaSuccess && !topk_done) {
            k_sieve_rekey<<<grid_for(nmem, 256), 256, 0, st>>>(v, cls, ncls, nmem, keys, vals);
            e = cudaGetLastError();
        }
        int cbits = 1;
        while (cbits < 32 && ((int64_t)1 << cbits) <= ncls) ++cbits;
        if (e == cudaSuccess && !topk_done) e = radix_sort_pairs(keys, vals, nmem, cbits, st);
        if (e == cudaSuccess && !topk_done) {
            int64_t warps_needed = nmem;
            int64_t blocks = (warps_needed + 7) / 8;
            if (blocks > grid_blocks) blocks = grid_blocks;
            const int zcap = (a_max + 3) & ~3;
            pn_kt_begin(v.kt, PN_KT_SIEVE, st);
            // after the class sort, keys[p] is the class of member p
            if (v.precision == 0) e = sieve_t<ZPlain>(v, cls, nmem, keys, vals, w, exhaustive, zcap, blocks, st);
            else if (exhaustive == 1 && sieve_gram_supported(a_max))
                e = launch_sieve_gram(v, cls, ncls, vals, nmem, a_max, grid_blocks, st);
            else if (exhaustive && v.x1) e = sieve_tiles_t<ZMix1>(v, cls, ncls, vals, grid_blocks, st);
            else if (exhaustive) e = sieve_tiles_t<ZMix2>(v, cls, ncls, vals, grid_blocks, st);
            else if (w <= SB_WMAX && v.x1) e = sieve_band_t<ZMix1>(v, cls, nmem, keys, vals, w, grid_blocks, st);
            else if (w <= SB_WMAX) e = sieve_band_t<ZMix2>(v, cls, nmem, keys, vals, w, grid_blocks, st);
            else if (v.x1) e = sieve_t<ZMix1>(v, cls, nmem, keys, vals, w, exhaustive, zcap, blocks, st);
            else e = sieve_t<ZMix2>(v, cls, nmem, keys, vals, w, exhaustive, zcap, blocks, st);
            pn_kt_end(v.kt, PN_KT_SIEVE, st);
            if (e == cudaSuccess) e = cudaGetLastError();
        }
    }
    *n_classes_out = ncls;
    if (cls) cudaFreeAsync(cls, st);
    if (keys) cudaFreeAsync(keys, st);
    if (vals) cudaFreeAsync(vals, st);
    cudaFreeAsync(flag, st);
    cudaFreeAsync(size, st);
    cudaFreeAsync(cid, st);
    cudaFreeAsync(moff, st);
    cudaFreeAsync(tot, st);
    return e;
}

cudaError_t launch_complete(const PnView &v, const PnSeed *seeds, int32_t nseeds, const int32_t *nseeds_dev, int dm,
                            int dp, int *improved, int grid_blocks, cudaStream_t st) {
    if (nseeds <= 0) return cudaSuccess;
    int g = nseeds < grid_blocks ? nseeds : grid_blocks;
    const size_t sm = sizeof(PnWin) * 2 * (size_t)(2 * dm + 1) * (2 * dp + 1);
    cudaError_t e = pn_allow_smem(k_complete, sm);
    if (e != cudaSuccess) return e;
    k_complete<<<g, 256, sm, st>>>(v, seeds, nseeds, nseeds_dev, dm, dp, improved);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Device-driven rounds of the emit stage.  A round (completion) or pass
// (refinement) is enqueued in full; a gate word decides on the device
// whether its kernels run, so the host enqueues the maximum number of
// rounds without waiting for any of them.
// ---------------------------------------------------------------------------
namespace {

// Ends a round: an empty round closes the gate, a round that ran is
// counted and closes the gate when nothing improved; the flag and the
// count start again at 0 for the next round.
__global__ void k_round_end(int *gate, int *flag, int32_t *count, int32_t *rounds, int32_t *count2) {
    if (count2) *count2 = 0;
    if (*gate) {
        if (*count == 0) {
            *gate = 0;
        } else {
            ++*rounds;
            if (!*flag) *gate = 0;
        }
        *flag = 0;
        *count = 0;
    }
}

// Refreshed completion seeds: each target's partner j read back from its
// cell (m, i), so a box is re-cut around the pair the cell now holds.
__global__ void k_seeds_refresh(PnView v, PnSeed *seeds, int32_t nmax, const int32_t *n_dev) {
    if (pn_gated(v)) return;
    const int32_t n = min(*n_dev, nmax);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    PnSeed sd = seeds[t];
    const PnSeries &S = v.series[sd.series];
    const unsigned long long key = v.prof[S.row_off + (int64_t)(sd.m - S.m_min) * S.ld + sd.i];
    if (key != PN_EMPTY_KEY) {
        sd.j = (int64_t)pn_key_idx(key);
        seeds[t] = sd;
    }
}

// Completion seeds from a selection's picks (group g's at picks[g kmax ...]).
__global__ void k_picks_to_seeds(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *seeds,
                                 int32_t *nseeds, const int *gate) {
    if (!*gate) return;
    const int gi = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gi >= ng) return;
    const int c = cnt[gi];
    int base = 0;
    if (lane == 0 && c > 0) base = atomicAdd(nseeds, c);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int t = lane; t < c; t += 32) {
        const PnPick p = picks[(int64_t)gi * kmax + t];
        seeds[base + t] = PnSeed{p.series, p.m, p.i, p.j};
    }
}

// Refinement targets: the picks of group g not refined in an earlier pass
// (done[g][0 .. ndone[g])), appended to the group's done list and to the
// targets; those among the group's first knear picks also to `near` (the
// cells whose boxes the pass completes).  One warp per group, so a group's
// list has one writer.
__global__ void k_new_targets(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *done,
                              int32_t *ndone, int32_t done_cap, PnSeed *targets, int32_t *ntargets, const int *gate,
                              PnSeed *near, int32_t *nnear, int32_t knear) {
    if (!*gate) return;
    const int gi = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (gi >= ng) return;
    const int c = cnt[gi];
    PnSeed *dl = done + (int64_t)gi * done_cap;
    int nd = ndone[gi];
    for (int t0 = 0; t0 < c; t0 += 32) {
        const int t = t0 + lane;
        PnSeed sd{0, 0, 0, 0};
        bool fresh = false;
        if (t < c) {
            const PnPick p = picks[(int64_t)gi * kmax + t];
            sd = PnSeed{p.series, p.m, p.i, p.j};
            fresh = true;
            for (int e = 0; e < nd && fresh; ++e)
                if (dl[e].m == p.m && dl[e].i == p.i) fresh = false;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, fresh);
        const int nf = __popc(bal);
        if (nf == 0) continue;
        const int rank = __popc(bal & ((1u << lane) - 1u));
        int base = 0;
        if (lane == 0) base = atomicAdd(ntargets, nf);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (fresh) {
            targets[base + rank] = sd;
            if (nd + rank < done_cap) dl[nd + rank] = sd;
        }
        // the fresh targets among the group's first knear picks also seed
        // the pass's completion
        const bool is_near = fresh && t < knear;
        const uint32_t nb = __ballot_sync(0xffffffffu, is_near);
        if (near && nb) {
            int nbase = 0;
            if (lane == 0) nbase = atomicAdd(nnear, __popc(nb));
            nbase = __shfl_sync(0xffffffffu, nbase, 0);
            if (is_near) near[nbase + __popc(nb & ((1u << lane) - 1u))] = sd;
        }
        nd = min(done_cap, nd + nf);
        __syncwarp();
    }
    if (lane == 0) ndone[gi] = nd;
}

}  // namespace

cudaError_t launch_round_end(int *gate, int *flag, int32_t *count, int32_t *rounds, cudaStream_t st,
                             int32_t *count2) {
    k_round_end<<<1, 1, 0, st>>>(gate, flag, count, rounds, count2);
    return cudaGetLastError();
}
cudaError_t launch_seeds_refresh(const PnView &v, PnSeed *seeds, int32_t nmax, const int32_t *n_dev, cudaStream_t st) {
    if (nmax <= 0) return cudaSuccess;
    k_seeds_refresh<<<grid_for(nmax, 256), 256, 0, st>>>(v, seeds, nmax, n_dev);
    return cudaGetLastError();
}
cudaError_t launch_picks_to_seeds(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *seeds,
                                  int32_t *nseeds, const int *gate, cudaStream_t st) {
    if (ng <= 0) return cudaSuccess;
    k_picks_to_seeds<<<grid_for((int64_t)ng * 32, 256), 256, 0, st>>>(picks, cnt, ng, kmax, seeds, nseeds, gate);
    return cudaGetLastError();
}
cudaError_t launch_new_targets(const PnPick *picks, const int32_t *cnt, int32_t ng, int32_t kmax, PnSeed *done,
                               int32_t *ndone, int32_t done_cap, PnSeed *targets, int32_t *ntargets, const int *gate,
                               cudaStream_t st, PnSeed *near, int32_t *nnear, int32_t knear) {
    if (ng <= 0) return cudaSuccess;
    k_new_targets<<<grid_for((int64_t)ng * 32, 256), 256, 0, st>>>(picks, cnt, ng, kmax, done, ndone, done_cap,
                                                                     targets, ntargets, gate, near, nnear, knear);
    return cudaGetLastError();
}

cudaError_t launch_select(const PnView &v, const PnSelGroup *grp_dev, int32_t ngrp, int64_t cell_begin,
                          int64_t cell_end, int32_t cap, double eps0, int32_t kmax, PnPick *out, int32_t *out_cnt,
                          int *overflow, int grid_blocks, cudaStream_t st) {
    if (ngrp <= 0) return cudaSuccess;
    (void)cell_begin;
    const int64_t total = cell_end;
    uint32_t *hist = nullptr, *b1 = nullptr, *b2 = nullptr, *carry = nullptr, *pcnt = nullptr;
    PnPoolEntry *pool = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&hist, sizeof(uint32_t) * 4096 * ngrp, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&b1, 4 * ngrp, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&b2, 4 * ngrp, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&carry, 4 * ngrp, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&pcnt, 4 * ngrp, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&pool, sizeof(PnPoolEntry) * (int64_t)cap * ngrp, st);
    // histogram blocks: contiguous ranges of at least 16 cells per thread
    const int64_t hist_blocks = std::max<int64_t>(1, std::min<int64_t>((total + 4095) / 4096, (int64_t)grid_blocks));
    const int64_t per_block = ((total + hist_blocks - 1) / hist_blocks + 255) / 256 * 256;
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 4096 * ngrp, st);
    if (e == cudaSuccess) {
        k_sel_hist<<<(unsigned)hist_blocks, 256, 0, st>>>(v, grp_dev, ngrp, total, eps0, 0, nullptr, hist, per_block);
        k_sel_pick<<<grid_for((int64_t)ngrp * 32, 128), 128, 0, st>>>(grp_dev, ngrp, hist, nullptr, b1, carry);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * 4096 * ngrp, st);
    if (e == cudaSuccess) {
        k_sel_hist<<<(unsigned)hist_blocks, 256, 0, st>>>(v, grp_dev, ngrp, total, eps0, 1, b1, hist, per_block);
        k_sel_pick<<<grid_for((int64_t)ngrp * 32, 128), 128, 0, st>>>(grp_dev, ngrp, hist, carry, b2, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(pcnt, 0, 4 * ngrp, st);
    if (e == cudaSuccess) {
        const int64_t pool_blocks = std::min<int64_t>(grid_for(total, 256), (int64_t)grid_blocks * 4);
        k_sel_pool<<<(unsigned)pool_blocks, 256, 0, st>>>(v, grp_dev, ngrp, total, eps0, b1, b2, pool, pcnt, cap,
                                                           overflow);
        int64_t vw = (int64_t)ngrp * cap;
        int64_t vb = (vw + 7) / 8;
        if (vb > grid_blocks) vb = grid_blocks;
        k_sel_verify<<<(unsigned)vb, 256, 0, st>>>(v, grp_dev, ngrp, pool, pcnt, cap, eps0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        int npow2 = 1;
        while (npow2 < cap) npow2 <<= 1;
        size_t sm = sizeof(PnPoolEntry) * npow2 + sizeof(int32_t) * (kmax + 1) + sizeof(int64_t) * kmax + 16;
        e = pn_allow_smem(k_sel_greedy, sm);
        if (e == cudaSuccess) {
            k_sel_greedy<<<ngrp, 1024, sm, st>>>(v, grp_dev, pool, pcnt, cap, npow2, out, out_cnt, kmax);
            e = cudaGetLastError();
        }
    }
    cudaFreeAsync(hist, st);
    cudaFreeAsync(b1, st);
    cudaFreeAsync(b2, st);
    cudaFreeAsync(carry, st);
    cudaFreeAsync(pcnt, st);
    cudaFreeAsync(pool, st);
    return e;
}

}  // namespace pn
