// Exhaustive hot-class sieve on the tensor cores (Sec. 3.6's hot-class
// sieve, every valid pair of each class), mixed form.
//
// A class's members are windows of one anchor length a.  For a tile of
// 128 x 128 members (u, v) the squared distances are a dense contraction:
// with y = z - z_r for one reference window r of the row block (the
// z-normalised windows shifted by a common vector, which leaves every
// difference unchanged), d^2(u, v) = |y_u|^2 + |y_v|^2 - 2 <y_u, y_v>.  The
// shift keeps the cancellation small where it matters: a hot class of
// near-copies of one pattern has |y|^2 of the order of the distances
// themselves instead of a.  Both blocks are staged in shared memory as FP16
// y-values (K-major, 128-byte swizzle, zero past a), one thread issues a/16
// tcgen05.mma kind::f16 (M = N = 128, K = 16 each) into a 128 x 128 FP32
// accumulator in tensor memory, and each warp reads its 32 rows back with
// tcgen05.ld.  The estimate decides which pairs are evaluated exactly (FP32
// differences, the search's arithmetic); the survivors lower both cells.
//
// Error of the estimate.  y is the FP32 difference of FP32 z-values (|y| <=
// 2 sqrt(a) < 28), y~ its FP16 rounding, |y~ - y| <= 2^-11 |y| + 2^-25, so
// each product is off by at most (2^-10 + 2^-22) |y_u y_v| plus a subnormal
// term below a 2^-19 in total; FP16 products are exact in FP32 and the
// accumulation of a <= 192 of them adds at most a 2^-23 of their
// magnitudes; Cauchy-Schwarz gives sum |y_u y_v| <= (|y_u|^2 + |y_v|^2) / 2;
// the norms are FP32 sums; y_u - y_v differs from z_u - z_v by the rounding
// of the two subtractions (<= 2^-23 |z| each), which moves the squared
// distance by less than a 2^-16; and the exact pass's FP32 sum of squares is
// within a 2^-24 of <= 2 (|y_u|^2 + |y_v|^2).  Together |d~^2 - d_f^2| <=
// 2^-9.9 (|y_u|^2 + |y_v|^2) + a 2^-16, with d_f the distance the exact pass
// would store; the tests use M = 2^-9 (|y_u|^2 + |y_v|^2) + a 2^-14.
//
// Which pairs are evaluated.  Pair (u, v) is evaluated iff
//   [d~^2 - M < P[u]^2 and d~^2 <= rowmin(u) + 2 M_row]  or
//   [d~^2 - M < P[v]^2 and d~^2 <= colmin(v) + 2 M_col],
// P the cells' current values (read when the block is staged: a stale,
// larger value keeps more pairs), rowmin / colmin the smallest estimate of
// the row / column in this tile, M_row (M_col) the margin with the row's
// (column's) own norm and the largest norm of the other block.  A pair
// failing the first part of a clause has d_f > P, so it cannot lower that
// cell; a pair failing the second has d_f above the best pair of its row
// (column) in the tile, which wins that cell against it.  So every pair
// whose key could end in a cell is evaluated, and the rows equal those of
// evaluating every pair, up to the FP32 rounding order of the distances.
//
// Column minima: each warp reduces a 32 x 32 block of estimates to its 32
// column minima with a transposing butterfly (31 shuffles), then one shared
// atomicMin per column and warp.
//
// Tiles are handed out by a work counter in runs of consecutive tiles of a
// class row, so a block restages only the column block when the row block
// is unchanged.  Waits on the MMA are bounded: on timeout the kernel records
// the error word, waits once more (bounded), frees its tensor memory and
// returns; the request reports ETIMEOUT.
#include <cuda_fp16.h>

#include <type_traits>

#include "emit.cuh"
#include "prims.cuh"
#include "tcgen05.cuh"
#include "zops.cuh"

namespace pn {
namespace {

constexpr int ZG_B = 128;           // members per tile side (MMA M and N)
constexpr int ZG_THREADS = 128;     // 4 warps: warp w owns tile rows / TMEM lanes 32w..32w+31
constexpr int ZG_Q = 256;           // survivor queue per warp
constexpr int ZG_RUN = 4;           // tiles a block draws at a time
constexpr int ZG_SPIN = 1 << 22;    // try_wait iterations before giving up
constexpr int ZG_AMAX = 192;        // longest anchor served (three K atoms)
constexpr int ZG_TMEM_COLS = 128;

// Tiles per class (upper triangle of 128-member blocks).  A class with more
// than 2^31 tiles, or a total above 2^31, sets *overflow: the launcher
// refuses such a request instead of enumerating a truncated table.
__global__ void k_zg_tile_count(const PnClass *cls, int32_t ncls, uint32_t *cnt, unsigned long long *total,
                                int *overflow) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncls) return;
    const uint64_t nb = (cls[ci].size + ZG_B - 1) / ZG_B;
    const uint64_t t = nb * (nb + 1) / 2;
    if (t > 0x7FFFFFFFull) {
        atomicExch(overflow, 1);
        cnt[ci] = 0;
        return;
    }
    cnt[ci] = (uint32_t)t;
    atomicAdd(total, (unsigned long long)t);
}

// One warp per class writes its tiles (class, bu, bv), bu-major.
__global__ void k_zg_tile_fill(const PnClass *cls, int32_t ncls, const uint32_t *off, uint4 *tiles) {
    const int ci = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (ci >= ncls) return;
    const uint32_t nb = (cls[ci].size + ZG_B - 1) / ZG_B;
    const uint32_t total = (uint32_t)(((uint64_t)nb * (nb + 1)) / 2);
    for (uint32_t t = lane; t < total; t += 32) {
        const uint32_t bu = tri_row(t, nb);
        const uint32_t before = (uint32_t)((uint64_t)bu * nb - ((uint64_t)bu * (bu - 1)) / 2);
        tiles[(int64_t)off[ci] + t] = make_uint4((uint32_t)ci, bu, bu + (t - before), 0u);
    }
}

// ---------------------------------------------------------------------------
// Pivot order of the top-k sieve.  Each member p of a class gets
// r_p = |z_p - z_c|, its distance to the class's first member c in the exact
// pass's FP32 z-values, and every class is re-sorted by r.  A pair (u, v) is
// at least |r_u - r_v| apart (triangle inequality), so in r order a column
// block bv whose smallest r exceeds row block bu's largest by more than T
// holds no pair of bu closer than T, and neither does any later column
// block: the tile table lists, per row block, only the column blocks before
// the first such one.
//
// Rounding: r~ is an FP32 norm of FP32 differences (a warp tree over at
// most 192 squares), |r~ - r| <= 2^-19 r for the z-values the exact pass
// uses, and the exact pass's distance d_f is within 2^-19 d of their true
// distance d.  A block pair is skipped only when
//   lo (1 - 2^-12) - hi (1 + 2^-12) > T (1 + 2^-12) + 2^-12,
// which leaves every skipped pair with d_f above the list threshold's FP32
// square root (T (1 + 5e-7) + 1e-6) by a wide margin.
// ---------------------------------------------------------------------------
constexpr float ZT_PIV_SLACK = 2.44140625e-4f;     // 2^-12

__device__ __forceinline__ bool zt_far(float lo, float hi, float T) {
    return lo * (1.0f - ZT_PIV_SLACK) - hi * (1.0f + ZT_PIV_SLACK) > T * (1.0f + ZT_PIV_SLACK) + ZT_PIV_SLACK;
}

// One warp per member: r (by position in the class-sorted member list), the
// sort key (the bits of r >= 0 order like r) and the position itself.
template <class Z>
__global__ void k_zt_pivot(PnView v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int64_t nmem, float *r,
                           uint32_t *keys, uint32_t *idx) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= nmem) return;
    const int ci = pn_find(cls, ncls, p, [](const PnClass &c) { return (int64_t)c.moff; });
    const PnClass c = cls[ci];
    const PnAnchor &A = v.anchors[c.anchor];
    const PnSeries &S = v.series[A.series];
    const uint32_t su = vals[p], sc = vals[c.moff];
    const auto mu = Z::load(v, A.win_off + su), mc = Z::load(v, A.win_off + sc);
    const auto *xu = Z::samples(v, S.x_off + su);
    const auto *xc = Z::samples(v, S.x_off + sc);
    float acc = 0.0f;
    for (int k = lane; k < A.a; k += 32) {
        const float d = Z::z(mu, xu[k]) - Z::z(mc, xc[k]);
        acc = fmaf(d, d, acc);
    }
    const float rr = sqrtf(pn_warp_sum(acc));
    if (lane == 0) {
        r[p] = rr;
        keys[p] = __float_as_uint(rr);
        idx[p] = (uint32_t)p;
    }
}

// After the sort by r: the class of each position, for the stable class sort.
__global__ void k_zt_rekey(const PnClass *cls, int32_t ncls, int64_t nmem, uint32_t *keys, const uint32_t *idx) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmem) return;
    keys[q] = (uint32_t)pn_find(cls, ncls, (int64_t)idx[q], [](const PnClass &c) { return (int64_t)c.moff; });
}

// After the class sort: position q's record (start, 1/sigma, -mu/sigma, r),
// the one 16-byte load a staging lane needs per row.
template <class Z>
__global__ void k_zt_records(PnView v, const PnClass *cls, const uint32_t *vals, const float *r, const uint32_t *idx,
                             const uint32_t *cid, int64_t nmem, uint4 *rec) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nmem) return;
    const uint32_t p = idx[q];
    const uint32_t s = vals[p];
    const auto m = Z::load(v, v.anchors[cls[cid[q]].anchor].win_off + s);
    rec[q] = make_uint4(s, __float_as_uint(m.x), __float_as_uint(m.y), __float_as_uint(r[p]));
}

__global__ void k_zt_blocks(const PnClass *cls, int32_t ncls, uint32_t *nb) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci < ncls) nb[ci] = (cls[ci].size + ZG_B - 1) / ZG_B;
}

// Row g = (class, bu): its tiles are bv = bu .. e, e the last column block
// not far from bu (far is monotone in bv: the blocks' smallest r ascend).
__device__ __forceinline__ float zt_r(const uint4 *rec, int64_t q) { return __uint_as_float(rec[q].w); }

__device__ __forceinline__ void zt_row(const PnClass *cls, int32_t ncls, const uint32_t *roff, const uint4 *rec,
                                       const float *thr_a, int64_t g, int &ci, uint32_t &bu, uint32_t &e) {
    ci = pn_find(roff, ncls, g, [](uint32_t o) { return (int64_t)o; });
    const PnClass c = cls[ci];
    const float T = thr_a[c.anchor];
    const uint32_t nb = (c.size + ZG_B - 1) / ZG_B;
    bu = (uint32_t)(g - roff[ci]);
    const float hi = zt_r(rec, (int64_t)c.moff + min((int64_t)c.size, ((int64_t)bu + 1) * ZG_B) - 1);
    uint32_t lo_b = bu, hi_b = nb - 1;                  // zt_far(lo(bu), hi) is false
    while (lo_b < hi_b) {
        const uint32_t mid = (lo_b + hi_b + 1) >> 1;
        if (zt_far(zt_r(rec, (int64_t)c.moff + (int64_t)mid * ZG_B), hi, T)) hi_b = mid - 1; else lo_b = mid;
    }
    e = lo_b;
}

__global__ void k_zt_row_count(const PnClass *cls, int32_t ncls, const uint32_t *roff, const uint32_t *nrows,
                               int64_t nrows_max, const uint4 *rec, const float *thr_a, uint32_t *tcnt,
                               unsigned long long *total) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nrows_max) return;
    if (g >= (int64_t)*nrows) {
        tcnt[g] = 0;
        return;
    }
    int ci;
    uint32_t bu, e;
    zt_row(cls, ncls, roff, rec, thr_a, g, ci, bu, e);
    tcnt[g] = e - bu + 1;
    atomicAdd(total, (unsigned long long)(e - bu + 1));
}

// One warp per row writes its tiles: class, first record of the row and of
// the column block, rows | columns << 8 | diagonal << 16.
__global__ void k_zt_row_fill(const PnClass *cls, int32_t ncls, const uint32_t *roff, const uint32_t *nrows,
                              const uint4 *rec, const float *thr_a, const uint32_t *toff, uint4 *tiles) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (g >= (int64_t)*nrows) return;
    int ci;
    uint32_t bu, e;
    zt_row(cls, ncls, roff, rec, thr_a, g, ci, bu, e);
    const PnClass c = cls[ci];
    const uint32_t nu = min((uint32_t)ZG_B, c.size - bu * ZG_B);
    for (uint32_t t = lane; t <= e - bu; t += 32) {
        const uint32_t bv = bu + t;
        const uint32_t nv = min((uint32_t)ZG_B, c.size - bv * ZG_B);
        tiles[(int64_t)toff[g] + t] =
            make_uint4((uint32_t)ci, c.moff + bu * ZG_B, c.moff + bv * ZG_B, nu | (nv << 8) | ((t == 0 ? 1u : 0u) << 16));
    }
}

struct ZgSide {
    uint32_t s[ZG_B];        // member window start (0 past the block)
    float2 m[ZG_B];          // (1/sigma, -mu/sigma); x = 0 for a degenerate window or past the block
    float n[ZG_B];           // |y|^2, y = z - z_ref
    float t[ZG_B];           // the cell's distance when staged
};

struct ZgShared {
    ZgSide A, B;
    float zref[ZG_AMAX];                       // z-values of the row block's reference window
    int colmin[ZG_B];                          // float bits
    unsigned long long rkey[ZG_B], ckey[ZG_B]; // exact keys of this tile, flushed to the cells once
    uint32_t queue[ZG_THREADS / 32][ZG_Q];
    int nmax_a, nmax_b;                        // float bits
    int fail;
    uint32_t taddr;
    __align__(8) uint64_t mbar;
    unsigned long long run;
};

// Stages block `first .. first + n` of class members into a swizzled FP16
// tile, as y = z - z_ref (the row block's reference window), and its side
// tables (n = |y|^2).  NW warps take RPG rows at a time each (rows
// warp RPG + RPG NW g + r), so every lane has 2 RPG sample loads in flight;
// each warp's rows have their member, moments and cell loaded up front, one
// per lane, so that only the sample loads wait inside the row loop.
template <class Z, int NW = ZG_THREADS / 32, int RPG = 4>
__device__ __forceinline__ void zg_stage(const PnView &v, const PnAnchor &A, const PnSeries &S, const uint32_t *members,
                                         int64_t first, int n, int a, int kp, unsigned char *tile, ZgSide &side,
                                         int *nmax, const unsigned long long *prow, const float *zref, int warp,
                                         int lane) {
    constexpr int RPW = ZG_B / NW;                 // rows per warp
    static_assert(RPW <= 32 && RPW % RPG == 0, "one lane per row of the warp");
    uint32_t c_l = 0;
    float2 m_l = make_float2(0.0f, 0.0f);
    unsigned long long k_l = PN_EMPTY_KEY;
    {
        const int g = lane / RPG, r = lane % RPG;
        const int row = warp * RPG + RPG * NW * g + r;
        if (lane < RPW && row < n) {
            c_l = members[first + row];
            const auto m = Z::load(v, A.win_off + c_l);
            m_l = make_float2(m.x, m.y);
            k_l = __ldcg(&prow[c_l]);
        }
    }
    for (int r0 = warp * RPG, gi = 0; r0 < ZG_B; r0 += RPG * NW, ++gi) {
        uint32_t cr[RPG];
        typename Z::M mr[RPG];
        const typename Z::X *xr[RPG];
#pragma unroll
        for (int r = 0; r < RPG; ++r) {
            cr[r] = __shfl_sync(0xffffffffu, c_l, gi * RPG + r);
            mr[r].x = __shfl_sync(0xffffffffu, m_l.x, gi * RPG + r);
            mr[r].y = __shfl_sync(0xffffffffu, m_l.y, gi * RPG + r);
            xr[r] = Z::samples(v, S.x_off + cr[r]);
        }
        const unsigned long long kr = __shfl_sync(0xffffffffu, k_l, gi * RPG + (lane % RPG));
        float acc[RPG];
#pragma unroll
        for (int r = 0; r < RPG; ++r) acc[r] = 0.0f;
        for (int k = 2 * lane; k < kp; k += 64) {
            float z0[RPG], z1[RPG];
#pragma unroll
            for (int r = 0; r < RPG; ++r) {
                const bool ok = r0 + r < n;
                z0[r] = (ok && k < a) ? Z::z(mr[r], xr[r][k]) - zref[k] : 0.0f;
                z1[r] = (ok && k + 1 < a) ? Z::z(mr[r], xr[r][k + 1]) - zref[k + 1] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < RPG; ++r) {
                acc[r] = fmaf(z0[r], z0[r], fmaf(z1[r], z1[r], acc[r]));
                *reinterpret_cast<__half2 *>(tile + sw128_off(r0 + r, k, ZG_B)) = __floats2half2_rn(z0[r], z1[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < RPG; ++r) {
            const float nr = pn_warp_sum(acc[r]);
            if (lane == r) {
                const int row = r0 + r;
                const bool ok = row < n;
                side.s[row] = ok ? cr[r] : 0u;
                side.m[row] = ok ? make_float2(mr[r].x, mr[r].y) : make_float2(0.0f, 0.0f);
                side.n[row] = nr;
                side.t[row] = ok ? pn_key_distf(kr) : 0.0f;
                if (nmax && ok && mr[r].x != 0.0f) atomicMax(nmax, __float_as_int(nr));
            }
        }
    }
}

// Exact distances of up to four queued pairs at once, by the whole warp
// (lanes over samples, four independent sums); each key lowers the tile's
// shared row and column minima, written to the cells once per tile.
template <class Z>
__device__ __forceinline__ void zg_eval4(const typename Z::X *xs, int a, const uint32_t *q, int nq,
                                         const ZgSide &SA, const ZgSide &SB, unsigned long long *rkey,
                                         unsigned long long *ckey, int lane) {
    typename Z::M zu[4], zv[4];
    uint32_t uu[4], vv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t e = q[p < nq ? p : 0];
        uu[p] = e >> 16;
        vv[p] = e & 0xFFFFu;
        zu[p].x = SA.m[uu[p]].x;
        zu[p].y = SA.m[uu[p]].y;
        zv[p].x = SB.m[vv[p]].x;
        zv[p].y = SB.m[vv[p]].y;
    }
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = lane; r < a; r += 32) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float d = Z::z(zu[p], xs[SA.s[uu[p]] + r]) - Z::z(zv[p], xs[SB.s[vv[p]] + r]);
            acc[p] = fmaf(d, d, acc[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float d = sqrtf(pn_warp_sum(acc[p]));
        if (lane == p && p < nq) {
            atomicMin(&rkey[uu[p]], pn_pack_f(d, SB.s[vv[p]]));
            atomicMin(&ckey[vv[p]], pn_pack_f(d, SA.s[uu[p]]));
        }
    }
}

// Column minima of a warp's 32 x 32 block: lane L ends with the minimum of
// column L over the warp's 32 rows (five butterfly stages, each lane keeping
// the half of its remaining columns selected by its own lane bit).
__device__ __forceinline__ float zg_colmin32(float (&dd)[32], int lane) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int j = 0; j < h; ++j) {
            const float send = up ? dd[j] : dd[j + h];
            const float keep = up ? dd[j + h] : dd[j];
            dd[j] = fminf(keep, __shfl_xor_sync(0xffffffffu, send, h));
        }
    }
    return dd[0];
}

template <class Z>
__global__ void __launch_bounds__(ZG_THREADS) k_sieve_zgram(PnView v, const PnClass *cls, const uint4 *tiles,
                                                            int64_t ntiles, const uint32_t *members, int kpad_max,
                                                            unsigned long long *work) {
    extern __shared__ __align__(1024) unsigned char zsm_raw[];
    __shared__ ZgShared sh;
    unsigned char *zsm = zsm_raw + ((1024 - (smem_u32(zsm_raw) & 1023)) & 1023);
    const int atoms = (kpad_max + 63) >> 6;
    unsigned char *tA = zsm;
    unsigned char *tB = tA + atoms * ZG_B * 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        sh.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.taddr)),
                     "r"(ZG_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = sh.taddr;
    const uint32_t idesc = umma_idesc_f16(ZG_B, ZG_B);
    const float inf = __int_as_float(0x7f800000);
    uint32_t phase = 0;
    unsigned long long n_ex = 0;
    uint32_t staged_cls = 0xFFFFFFFFu, staged_bu = 0xFFFFFFFFu;

    for (;;) {
        __syncthreads();
        if (tid == 0) sh.run = atomicAdd(work, (unsigned long long)ZG_RUN);
        __syncthreads();
        const int64_t run0 = (int64_t)sh.run;
        if (run0 >= ntiles || sh.fail) break;
        const int64_t run1 = min(ntiles, run0 + ZG_RUN);
        for (int64_t t = run0; t < run1; ++t) {
            const uint4 tl = tiles[t];
            const PnClass c = cls[tl.x];
            const PnAnchor &A = v.anchors[c.anchor];
            const PnSeries &S = v.series[A.series];
            const int a = A.a;
            const int kp = (a + 15) & ~15;
            const int u0 = (int)tl.y * ZG_B, v0 = (int)tl.z * ZG_B;
            const int nu = min(ZG_B, (int)c.size - u0), nv = min(ZG_B, (int)c.size - v0);
            const bool diag = tl.y == tl.z;
            unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
            __syncthreads();                            // the previous tile's reads of both blocks are done
            const bool new_row = tl.x != staged_cls || tl.y != staged_bu;
            if (tid == 0) {
                if (new_row) sh.nmax_a = 0;
                sh.nmax_b = 0;
            }
            sh.rkey[tid] = PN_EMPTY_KEY;
            sh.ckey[tid] = PN_EMPTY_KEY;
            sh.colmin[tid] = 0x7f800000;
            __syncthreads();
            if (new_row) {
                // reference: the row block's first member (both blocks of a tile share it)
                const uint32_t cr = members[(int64_t)c.moff + u0];
                const auto mref = Z::load(v, A.win_off + cr);
                const auto *xref = Z::samples(v, S.x_off + cr);
                for (int k = tid; k < kp; k += ZG_THREADS) sh.zref[k] = k < a ? Z::z(mref, xref[k]) : 0.0f;
                __syncthreads();
                zg_stage<Z>(v, A, S, members, (int64_t)c.moff + u0, nu, a, kp, tA, sh.A, &sh.nmax_a, prow, sh.zref,
                            warp, lane);
            }
            zg_stage<Z>(v, A, S, members, (int64_t)c.moff + v0, nv, a, kp, tB, sh.B, &sh.nmax_b, prow, sh.zref, warp,
                        lane);
            staged_cls = tl.x;
            staged_bu = tl.y;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid == 0) {
                const uint32_t a0 = smem_u32(tA), b0 = smem_u32(tB);
                for (int s = 0; s < kp / 16; ++s) {
                    const uint32_t off = (uint32_t)((s >> 2) * ZG_B * 128 + (s & 3) * 32);
                    const uint64_t ad = sw128_desc(a0 + off), bd = sw128_desc(b0 + off);
                    const uint32_t acc = s > 0 ? 1u : 0u;
                    asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                                 ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&sh.mbar))
                             : "memory");
            }
            if (!mbar_wait(smem_u32(&sh.mbar), phase, ZG_SPIN)) {
                if (lane == 0) atomicExch(&sh.fail, 1);
            }
            phase ^= 1u;
            __syncthreads();
            if (sh.fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

            // ---- pass 1: row minima (per thread) and column minima (butterfly + shared atomics)
            const int u = warp * 32 + lane;
            const bool urow = u < nu && sh.A.m[u].x != 0.0f;
            const float nu_ = sh.A.n[u];
            const int64_t pu = (int64_t)sh.A.s[u];
            const uint32_t tbase = taddr + ((uint32_t)(warp * 32) << 16);
            float rmin = inf;
            for (int c0 = 0; c0 < ZG_B; c0 += 32) {
                uint32_t r[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                    "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(tbase + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float dd[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int vc = c0 + j;
                    bool ok = urow && vc < nv && (!diag || u < vc) && sh.B.m[vc].x != 0.0f;
                    if (ok) ok = llabs(pu - (int64_t)sh.B.s[vc]) >= S.excl;
                    dd[j] = ok ? fmaxf(0.0f, nu_ + sh.B.n[vc] - 2.0f * __uint_as_float(r[j])) : inf;
                    rmin = fminf(rmin, dd[j]);
                }
                const float cm = zg_colmin32(dd, lane);
                if (cm < inf) atomicMin(&sh.colmin[c0 + lane], __float_as_int(cm));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

            // ---- pass 2: the pairs that can still lower a cell, evaluated exactly
            const float nmax_a = __int_as_float(sh.nmax_a), nmax_b = __int_as_float(sh.nmax_b);
            const float tu2 = sh.A.t[u] * sh.A.t[u];
            const float mabs = (float)a * 6.1035156e-05f;           // a 2^-14
            const float tol_row = 0.00390625f * (nu_ + nmax_b) + 2.0f * mabs;   // 2 M_row
            const auto *xs = Z::samples(v, S.x_off);
            int qn = 0;
            for (int c0 = 0; c0 < ZG_B; c0 += 32) {
                uint32_t r[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                    "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(tbase + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int vc = c0 + j;
                    bool s = urow && vc < nv && (!diag || u < vc) && sh.B.m[vc].x != 0.0f;
                    if (s) s = llabs(pu - (int64_t)sh.B.s[vc]) >= S.excl;
                    if (s) {
                        const float nv_ = sh.B.n[vc];
                        const float dd = fmaxf(0.0f, nu_ + nv_ - 2.0f * __uint_as_float(r[j]));
                        const float M = 0.001953125f * (nu_ + nv_) + mabs;     // 2^-9 (|y_u|^2 + |y_v|^2) + a 2^-14
                        const float tv = sh.B.t[vc];
                        const bool keep_u = dd - M < tu2 && dd <= rmin + tol_row;
                        const bool keep_v = dd - M < tv * tv && dd <= __int_as_float(sh.colmin[vc]) +
                                                                          0.00390625f * (nv_ + nmax_a) + 2.0f * mabs;
                        s = keep_u || keep_v;
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, s);
                    if (s) sh.queue[warp][qn + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)u << 16) | (uint32_t)vc;
                    qn += __popc(bal);
                    if (qn > ZG_Q - 32) {                     // warp-uniform: evaluate the queued pairs
                        __syncwarp();
                        for (int e = 0; e < qn; e += 4)
                            zg_eval4<Z>(xs, a, &sh.queue[warp][e], min(4, qn - e), sh.A, sh.B, sh.rkey, sh.ckey, lane);
                        n_ex += (unsigned long long)qn;
                        qn = 0;
                        __syncwarp();
                    }
                }
            }
            __syncwarp();
            for (int e = 0; e < qn; e += 4)
                zg_eval4<Z>(xs, a, &sh.queue[warp][e], min(4, qn - e), sh.A, sh.B, sh.rkey, sh.ckey, lane);
            n_ex += (unsigned long long)qn;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();                               // every warp's keys are in the tile minima
            if (sh.rkey[tid] != PN_EMPTY_KEY) atomicMin(&prow[sh.A.s[tid]], sh.rkey[tid]);
            if (sh.ckey[tid] != PN_EMPTY_KEY) atomicMin(&prow[sh.B.s[tid]], sh.ckey[tid]);
        }
        if (sh.fail) break;
    }
    __syncthreads();
    if (sh.fail && tid == 0) {
        atomicExch(v.err, PN_ERR_TC_TIMEOUT);
        mbar_wait(smem_u32(&sh.mbar), phase ^ 1u, ZG_SPIN);   // an MMA still in flight finishes (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ZG_TMEM_COLS));
    if (lane == 0 && v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], n_ex);
}

// The top-k sieve.  Instead of the row and column rules, a pair is evaluated
// exactly only when its estimate minus the margin is below thr2 (the square
// of a distance the top list already holds) and below one of its two cells:
// the pass looks only for pairs that can enter the list.  Eight warps (warps
// w and w + 4 read the same accumulator lanes, columns 0-63 and 64-127), and a fast test per pair
// -- one multiply-add against a per-row constant -- whose rare hits take the
// full test.  The fast test is the exact one rearranged:
// d~^2 - M < thr2  <=>  (1 - 2^-9) |y_v|^2 - 2 G < thr2 + a 2^-14 - (1 - 2^-9) |y_u|^2,
// with a relative slack of 2^-20 on the right for the rearranged rounding.
constexpr int ZT_THREADS = 256;
constexpr int ZT_WARPS = ZT_THREADS / 32;
constexpr int ZT_Q = 128;
constexpr int ZT_RUN = 16;          // tiles a block draws at a time (one row block mostly: A staged once)

struct ZtShared {
    ZgSide A, B;
    __align__(16) float zref[ZG_AMAX];
    __align__(16) float nbx[ZG_B];             // (1 - 2^-9) |y_v|^2 of the column block
    float2 nbt[ZG_B];                          // ((1 - 2^-9) |y_v|^2, P[v]^2) of the column block
    unsigned long long rkey[ZG_B], ckey[ZG_B];
    uint32_t queue[ZT_WARPS][ZT_Q];
    int fail;
    uint32_t taddr;
    __align__(8) uint64_t mbar;
    unsigned long long run;
};

// Stages a block of class members for the top-k sieve as y = z - z_ref in
// FP16 (the layout and side tables of zg_stage).  Warp w owns rows
// 16 w .. 16 w + 15 and takes U of them at a time, the whole warp on each
// row: lane l holds the sample pairs k = 2 l + 64 j, so a load instruction
// reads 256 consecutive bytes of a row, every lane stores one FP16 pair per
// step at an offset fixed per row (the 128-byte swizzle of row r puts the
// pair of lane l at r 128 + ((l / 4) xor (r mod 8)) 16 + (l mod 4) 4 in each
// 64-column atom), and all loads of a group are issued before the first is
// used.  The loads take whole steps without bounds (a window's last step
// reads at most 192 samples past its start, inside the sample buffer's
// zero padding past the last series) and the samples past the window's end
// are masked.  Lane l < 16 brings row 16 w + l's record (start, 1/sigma,
// -mu/sigma), loaded one tile ahead; the cells are read here, early, and
// used last, when each of these lanes writes its row's side entries.
// |y|^2 is the FP32 warp sum of the row's squares.
template <class Z, int U>
__device__ __forceinline__ void zt_stage(const typename Z::X *xs, uint4 rl, int n, int a, int kp,
                                         unsigned char *tile, ZgSide &side, const unsigned long long *prow,
                                         const float *zref, int warp, int lane) {
    constexpr int RPW = ZG_B / ZT_WARPS;        // 16 rows per warp
    constexpr int JP = (ZG_AMAX + 63) / 64;     // pair steps per row
    static_assert(RPW % U == 0, "row groups");
    static_assert(64 * JP <= PN_SAMPLE_PAD, "unbounded steps stay inside the padding");
    const bool mine = lane < RPW && warp * RPW + lane < n;
    const unsigned long long k_l = mine ? __ldcg(&prow[rl.x]) : PN_EMPTY_KEY;
    float2 zr[JP];
    bool in0[JP], in1[JP];
#pragma unroll
    for (int j = 0; j < JP; ++j) {
        const int k = 2 * lane + 64 * j;
        zr[j] = k < kp ? *reinterpret_cast<const float2 *>(zref + k) : make_float2(0.0f, 0.0f);
        in0[j] = k < a;
        in1[j] = k + 1 < a;
    }
    const uint32_t lane_off = (uint32_t)(lane & 3) * 4u;
    float n_own = 0.0f;                         // |y|^2 of row 16 w + l (lanes l < 16)
    for (int g = 0; g < RPW; g += U) {
        int row[U];
        bool ok[U];
        uint32_t cr[U];
        typename Z::M mr[U];
        typename Z::X xv[U][JP][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            row[u] = warp * RPW + g + u;
            ok[u] = row[u] < n;
            cr[u] = __shfl_sync(0xffffffffu, rl.x, g + u);
            mr[u].x = __uint_as_float(__shfl_sync(0xffffffffu, rl.y, g + u));
            mr[u].y = __uint_as_float(__shfl_sync(0xffffffffu, rl.z, g + u));
            const typename Z::X *xr = xs + cr[u] + 2 * lane;
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                if (64 * j < kp) {
                    xv[u][j][0] = __ldg(xr + 64 * j);
                    xv[u][j][1] = __ldg(xr + 64 * j + 1);
                } else {
                    xv[u][j][0] = typename Z::X{};
                    xv[u][j][1] = typename Z::X{};
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t roff = (uint32_t)row[u] * 128u + ((((uint32_t)lane >> 2) ^ ((uint32_t)row[u] & 7u)) << 4) +
                                  lane_off;
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < JP; ++j) {
                const float z0 = Z::z(mr[u], xv[u][j][0]) - zr[j].x;
                const float z1 = Z::z(mr[u], xv[u][j][1]) - zr[j].y;
                const float y0 = ok[u] && in0[j] ? z0 : 0.0f;
                const float y1 = ok[u] && in1[j] ? z1 : 0.0f;
                acc = fmaf(y0, y0, fmaf(y1, y1, acc));
                if (64 * j < kp)
                    *reinterpret_cast<__half2 *>(tile + roff + (uint32_t)j * (ZG_B * 128)) = __floats2half2_rn(y0, y1);
            }
            const float nr = pn_warp_sum(acc);
            if (lane == g + u) n_own = nr;
        }
    }
    // side tables: lane l < 16 writes its own row's entries
    const int row = warp * RPW + lane;
    if (lane < RPW) {
        side.s[row] = mine ? rl.x : 0u;
        side.m[row] = mine ? make_float2(__uint_as_float(rl.y), __uint_as_float(rl.z)) : make_float2(0.0f, 0.0f);
        side.n[row] = n_own;
        side.t[row] = mine ? pn_key_distf(k_l) : 0.0f;
    }
}

constexpr int ZT_U = 4;              // rows per half-warp in flight while staging

// The queued pairs of a warp evaluated exactly, four at a time (one copy of
// the evaluation code for both call sites of the top-k kernel).
template <class Z>
__device__ __noinline__ void zt_flush(const typename Z::X *xs, int a, const uint32_t *q, int qn, const ZgSide &SA,
                                      const ZgSide &SB, unsigned long long *rkey, unsigned long long *ckey, int lane) {
    __syncwarp();
    for (int e = 0; e < qn; e += 4) zg_eval4<Z>(xs, a, q + e, min(4, qn - e), SA, SB, rkey, ckey, lane);
    __syncwarp();
}

// Row-lane record of a block: lane l < 16 of warp w holds row 16 w + l's.
__device__ __forceinline__ uint4 zt_record(const uint4 *rec, uint32_t first, int n, int warp, int lane) {
    const int row = warp * (ZG_B / ZT_WARPS) + lane;
    return (lane < ZG_B / ZT_WARPS && row < n) ? __ldg(&rec[(int64_t)first + row]) : make_uint4(0u, 0u, 0u, 0u);
}

// Tiles: x = class, y / z = first record of the row / column block,
// w = rows | columns << 8 | diagonal << 16.
template <class Z>
__global__ void __launch_bounds__(ZT_THREADS, 2) k_sieve_topk(PnView v, const PnClass *cls, const uint4 *tiles,
                                                           int64_t ntiles, const uint4 *rec, int kpad_max,
                                                           unsigned long long *work, const float *thr_a,
                                                           unsigned long long *improved) {
    extern __shared__ __align__(1024) unsigned char ztm_raw[];
    __shared__ ZtShared sh;
    unsigned char *ztm = ztm_raw + ((1024 - (smem_u32(ztm_raw) & 1023)) & 1023);
    const int atoms = (kpad_max + 63) >> 6;
    unsigned char *tA = ztm;
    unsigned char *tB = tA + atoms * ZG_B * 128;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        sh.fail = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&sh.mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.taddr)),
                     "r"(ZG_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = sh.taddr;
    const uint32_t idesc = umma_idesc_f16(ZG_B, ZG_B);
    uint32_t phase = 0;
    unsigned long long n_ex = 0;
    uint32_t staged_a = 0xFFFFFFFFu;                 // first record of the staged row block
    const int quarter = warp & 3, half = warp >> 2;
    const int u = quarter * 32 + lane;

    for (;;) {
        __syncthreads();
        if (tid == 0) sh.run = atomicAdd(work, (unsigned long long)ZT_RUN);
        __syncthreads();
        const int64_t run0 = (int64_t)sh.run;
        if (run0 >= ntiles || sh.fail) break;
        const int64_t run1 = min(ntiles, run0 + ZT_RUN);
        uint4 tl = tiles[run0];
        uint4 ra = zt_record(rec, tl.y, (int)(tl.w & 0xFFu), warp, lane);
        uint4 rb = zt_record(rec, tl.z, (int)((tl.w >> 8) & 0xFFu), warp, lane);
        for (int64_t t = run0; t < run1; ++t) {
            // the next tile's coordinates, loaded now and used after this tile's staging
            const uint4 tn = t + 1 < run1 ? tiles[t + 1] : make_uint4(0u, 0u, 0u, 0u);
            const PnClass c = cls[tl.x];
            const PnAnchor &A = v.anchors[c.anchor];
            const PnSeries &S = v.series[A.series];
            const int a = A.a;
            const int kp = (a + 15) & ~15;
            const int excl = S.excl;
            const int nu = (int)(tl.w & 0xFFu), nv = (int)((tl.w >> 8) & 0xFFu);
            const bool diag = (tl.w >> 16) & 1u;
            unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
            const auto *xs = Z::samples(v, S.x_off);
            __syncthreads();
            const bool new_row = tl.y != staged_a;
            if (tid < ZG_B) {
                sh.rkey[tid] = PN_EMPTY_KEY;
                sh.ckey[tid] = PN_EMPTY_KEY;
            }
            if (new_row) {
                // reference: the row block's first member (both blocks of a tile share it)
                const uint4 r0 = __ldg(&rec[tl.y]);
                typename Z::M mref;
                mref.x = __uint_as_float(r0.y);
                mref.y = __uint_as_float(r0.z);
                const auto *xref = Z::samples(v, S.x_off + r0.x);
                for (int k = tid; k < kp; k += ZT_THREADS) sh.zref[k] = k < a ? Z::z(mref, xref[k]) : 0.0f;
            }
            __syncthreads();
            // the row block (when it changed) and the column block, through one copy of the staging code
#pragma unroll 1
            for (int sd = new_row ? 0 : 1; sd < 2; ++sd)
                zt_stage<Z, ZT_U>(xs, sd ? rb : ra, sd ? nv : nu, a, kp, sd ? tB : tA, sd ? sh.B : sh.A, prow, sh.zref,
                                  warp, lane);
            staged_a = tl.y;
            // the next tile's records, in flight during this tile's product and epilogue
            if (t + 1 < run1) {
                ra = tn.y != tl.y ? zt_record(rec, tn.y, (int)(tn.w & 0xFFu), warp, lane) : ra;
                rb = zt_record(rec, tn.z, (int)((tn.w >> 8) & 0xFFu), warp, lane);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid < ZG_B) {
                // columns past the block and degenerate windows never pass the fast test
                const bool colok = tid < nv && sh.B.m[tid].x != 0.0f;
                const float nb_ = colok ? 0.998046875f * sh.B.n[tid] : __int_as_float(0x7f800000);
                sh.nbx[tid] = nb_;
                sh.nbt[tid] = make_float2(nb_, sh.B.t[tid] * sh.B.t[tid]);
            }
            if (tid == 0) {
                const uint32_t a0 = smem_u32(tA), b0 = smem_u32(tB);
                for (int s2 = 0; s2 < kp / 16; ++s2) {
                    const uint32_t off = (uint32_t)((s2 >> 2) * ZG_B * 128 + (s2 & 3) * 32);
                    const uint64_t ad = sw128_desc(a0 + off), bd = sw128_desc(b0 + off);
                    const uint32_t acc = s2 > 0 ? 1u : 0u;
                    asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }"
                                 ::"r"(taddr), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&sh.mbar))
                             : "memory");
            }
            if (!mbar_wait(smem_u32(&sh.mbar), phase, ZG_SPIN)) {
                if (lane == 0) atomicExch(&sh.fail, 1);
            }
            phase ^= 1u;
            __syncthreads();
            if (sh.fail) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

            const bool urow = u < nu && sh.A.m[u].x != 0.0f;
            const float nu_ = sh.A.n[u];
            const float mabs = (float)a * 6.1035156e-05f;                    // a 2^-14
            const float tu2 = sh.A.t[u] * sh.A.t[u];
            const float ts = thr_a[c.anchor];
            const float thr2 = ts * ts * (1.0f + 1e-6f) + 1e-12f;              // FP32 rounding of the square
            // fast bound: (1 - 2^-9) |y_v|^2 - 2 G < min(thr2, max(P[u]^2, P[v]^2)) + cu, with
            // cu = a 2^-14 - (1 - 2^-9) |y_u|^2 and a slack of 2^-20 of the magnitudes involved
            const float slack = 9.5367432e-07f * (thr2 + mabs + nu_ + 1.0f);
            const float cu = urow ? mabs - 0.998046875f * nu_ + slack : -__int_as_float(0x7f800000);
            const float kt = thr2 + cu, ku = tu2 + cu;
            // no row of the warp holds a cell below the list threshold: the
            // fast test is e < kt alone, and a column group without any
            // e = (1 - 2^-9) |y_v|^2 - 2 G below kt is passed by a running minimum
            const bool rows_above = __all_sync(0xffffffffu, !urow || ku >= kt);
            const int64_t pu = (int64_t)sh.A.s[u];
            const uint32_t tbase = taddr + ((uint32_t)(quarter * 32) << 16);
            int qn = 0;
            for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 32) {
                uint32_t r[32];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                    "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(tbase + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (rows_above) {
                    float e4[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) e4[j] = fmaf(-2.0f, __uint_as_float(r[j]), sh.nbx[c0 + j]);
#pragma unroll
                    for (int j = 4; j < 32; ++j)
                        e4[j & 3] = fminf(e4[j & 3], fmaf(-2.0f, __uint_as_float(r[j]), sh.nbx[c0 + j]));
                    if (!__any_sync(0xffffffffu, fminf(fminf(e4[0], e4[1]), fminf(e4[2], e4[3])) < kt)) continue;
                }
                // the full test, one column at a time (rare: a group with a pair near
                // the list), each estimate read again from tensor memory
#pragma unroll 1
                for (int j = 0; j < 32; ++j) {
                    uint32_t gj;
                    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];"
                                 : "=r"(gj)
                                 : "r"(tbase + (uint32_t)(c0 + j)));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const float G = __uint_as_float(gj);
                    const int vc = c0 + j;
                    const float2 nt = sh.nbt[vc];
                    bool keep = fmaf(-2.0f, G, nt.x) < fminf(kt, fmaxf(ku, nt.y + cu)) && vc < nv && (!diag || u < vc) &&
                                sh.B.m[vc].x != 0.0f;
                    if (keep) keep = llabs(pu - (int64_t)sh.B.s[vc]) >= excl;
                    if (keep) {
                        const float nv_ = sh.B.n[vc];
                        const float dd = fmaxf(0.0f, nu_ + nv_ - 2.0f * G);
                        const float M = 0.001953125f * (nu_ + nv_) + mabs;
                        const float tv = sh.B.t[vc];
                        keep = dd - M < thr2 && (dd - M < tu2 || dd - M < tv * tv);
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                    if (keep) sh.queue[warp][qn + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)u << 16) | (uint32_t)vc;
                    qn += __popc(bal);
                    if (qn > ZT_Q - 32) {
                        n_ex += (unsigned long long)qn;
                        zt_flush<Z>(xs, a, sh.queue[warp], qn, sh.A, sh.B, sh.rkey, sh.ckey, lane);
                        qn = 0;
                    }
                }
            }
            n_ex += (unsigned long long)qn;
            zt_flush<Z>(xs, a, sh.queue[warp], qn, sh.A, sh.B, sh.rkey, sh.ckey, lane);
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            if (tid < ZG_B) {
                bool lowered = false;
                if (sh.rkey[tid] != PN_EMPTY_KEY) lowered |= atomicMin(&prow[sh.A.s[tid]], sh.rkey[tid]) > sh.rkey[tid];
                if (sh.ckey[tid] != PN_EMPTY_KEY) lowered |= atomicMin(&prow[sh.B.s[tid]], sh.ckey[tid]) > sh.ckey[tid];
                if (lowered) atomicOr(improved, 1ull);
            }
            tl = tn;
        }
        if (sh.fail) break;
    }
    __syncthreads();
    if (sh.fail && tid == 0) {
        atomicExch(v.err, PN_ERR_TC_TIMEOUT);
        mbar_wait(smem_u32(&sh.mbar), phase ^ 1u, ZG_SPIN);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ZG_TMEM_COLS));
    if (lane == 0 && v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], n_ex);
}

template <class Z>
cudaError_t sieve_zgram_t(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int a_max,
                          int grid_blocks, cudaStream_t st) {
    uint32_t *cnt = nullptr, *off = nullptr, *tot = nullptr;
    unsigned long long *tot64 = nullptr;
    uint4 *tiles = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&cnt, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&off, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot, 4, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot64, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tot64, 0, 2 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_zg_tile_count<<<(unsigned)((ncls + 255) / 256), 256, 0, st>>>(cls, ncls, cnt, tot64,
                                                                     reinterpret_cast<int *>(tot64 + 1));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(cnt, off, ncls, tot, st);
    unsigned long long h[2] = {0ull, 0ull};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, tot64, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int64_t ntiles = (int64_t)h[0];
    if (e == cudaSuccess && (h[1] != 0ull || ntiles > 0x7FFFFFFFll)) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && ntiles > 0) e = cudaMallocAsync((void **)&tiles, sizeof(uint4) * (size_t)ntiles, st);
    unsigned long long *work = tot64;
    if (e == cudaSuccess && ntiles > 0) e = cudaMemsetAsync(work, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess && ntiles > 0) {
        k_zg_tile_fill<<<(unsigned)(((int64_t)ncls * 32 + 255) / 256), 256, 0, st>>>(cls, ncls, off, tiles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && ntiles > 0) {
        const int kpad = (a_max + 15) & ~15;
        const int atoms = (kpad + 63) >> 6;
        const size_t sm = 1024 + (size_t)atoms * 2 * ZG_B * 128;
        const int64_t g = std::min<int64_t>((ntiles + ZG_RUN - 1) / ZG_RUN, (int64_t)grid_blocks);
        e = pn_allow_smem(k_sieve_zgram<Z>, sm);
        if (e == cudaSuccess) {
            k_sieve_zgram<Z><<<(unsigned)g, ZG_THREADS, sm, st>>>(v, cls, tiles, ntiles, vals, kpad, work);
            e = cudaGetLastError();
        }
    }
    for (void *p : {(void *)cnt, (void *)off, (void *)tot, (void *)tot64, (void *)tiles})
        if (p) cudaFreeAsync(p, st);
    return e;
}

// The top-k sieve: members re-sorted by their pivot distance, the tile table
// pruned by the triangle inequality, then k_sieve_topk over the kept tiles.
template <class Z>
cudaError_t sieve_topk_t(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int64_t nmem,
                         int a_max, int grid_blocks, const float *thr_a, int *improved, cudaStream_t st) {
    if (nmem <= 0) return cudaSuccess;
    const int64_t nrows_max = nmem / ZG_B + ncls + 1;           // sum of ceil(size / 128) over the classes
    float *r = nullptr;
    uint32_t *keys = nullptr, *idx = nullptr, *nb = nullptr, *roff = nullptr, *tot = nullptr;
    uint32_t *tcnt = nullptr, *toff = nullptr;
    unsigned long long *tot64 = nullptr;
    uint4 *rec = nullptr, *tiles = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&r, 4 * (size_t)nmem, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&keys, 4 * (size_t)nmem, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&idx, 4 * (size_t)nmem, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&rec, sizeof(uint4) * (size_t)nmem, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&nb, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&roff, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot, 8, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tcnt, 4 * (size_t)nrows_max, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&toff, 4 * (size_t)nrows_max, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot64, 3 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(tot64, 0, 3 * sizeof(unsigned long long), st);
    if (e == cudaSuccess) {
        k_zt_pivot<Z><<<(unsigned)((nmem * 32 + 255) / 256), 256, 0, st>>>(v, cls, ncls, vals, nmem, r, keys, idx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = radix_sort_pairs(keys, idx, nmem, 32, st);
    int cbits = 1;
    while (cbits < 32 && ((int64_t)1 << cbits) <= ncls) ++cbits;
    if (e == cudaSuccess) {
        k_zt_rekey<<<(unsigned)((nmem + 255) / 256), 256, 0, st>>>(cls, ncls, nmem, keys, idx);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = radix_sort_pairs(keys, idx, nmem, cbits, st);
    if (e == cudaSuccess) {
        // after the class sort keys[q] is the class of position q
        k_zt_records<Z><<<(unsigned)((nmem + 255) / 256), 256, 0, st>>>(v, cls, vals, r, idx, keys, nmem, rec);
        k_zt_blocks<<<(unsigned)((ncls + 255) / 256), 256, 0, st>>>(cls, ncls, nb);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(nb, roff, ncls, tot, st);             // tot[0] = rows
    if (e == cudaSuccess) {
        k_zt_row_count<<<(unsigned)((nrows_max + 255) / 256), 256, 0, st>>>(cls, ncls, roff, tot, nrows_max, rec,
                                                                           thr_a, tcnt, tot64);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(tcnt, toff, nrows_max, tot + 1, st);
    unsigned long long h = 0ull;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, tot64, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    const int64_t ntiles = (int64_t)h;
    if (e == cudaSuccess && ntiles > 0x7FFFFFFFll) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess && ntiles > 0) e = cudaMallocAsync((void **)&tiles, sizeof(uint4) * (size_t)ntiles, st);
    unsigned long long *work = tot64 + 1;
    if (e == cudaSuccess && ntiles > 0) {
        k_zt_row_fill<<<(unsigned)((nrows_max * 32 + 255) / 256), 256, 0, st>>>(cls, ncls, roff, tot, rec, thr_a,
                                                                               toff, tiles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && ntiles > 0) {
        const int kpad = (a_max + 15) & ~15;
        const int atoms = (kpad + 63) >> 6;
        const size_t sm = 1024 + (size_t)atoms * 2 * ZG_B * 128;
        const int64_t g = std::min<int64_t>((ntiles + ZT_RUN - 1) / ZT_RUN, (int64_t)grid_blocks);
        e = pn_allow_smem(k_sieve_topk<Z>, sm);
        if (e == cudaSuccess) {
            k_sieve_topk<Z><<<(unsigned)g, ZT_THREADS, sm, st>>>(v, cls, tiles, ntiles, rec, kpad, work, thr_a,
                                                                 tot64 + 2);
            e = cudaGetLastError();
        }
    }
    // whether any cell went down (the emit stage after the sieve is needed only then)
    unsigned long long himp = 0ull;
    if (e == cudaSuccess && ntiles > 0) e = cudaMemcpyAsync(&himp, tot64 + 2, sizeof(himp), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ntiles > 0) e = cudaStreamSynchronize(st);
    if (improved && himp) *improved = 1;
    for (void *p : {(void *)r, (void *)keys, (void *)idx, (void *)rec, (void *)nb, (void *)roff, (void *)tot,
                    (void *)tcnt, (void *)toff, (void *)tot64, (void *)tiles})
        if (p) cudaFreeAsync(p, st);
    return e;
}

}  // namespace

bool sieve_gram_supported(int a_max) { return a_max <= ZG_AMAX; }

cudaError_t launch_sieve_gram(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int64_t nmem,
                              int a_max, int grid_blocks, cudaStream_t st, const float *topk_thr, int *improved) {
    if (ncls <= 0) return cudaSuccess;
    if (topk_thr) {
        if (v.x1) return sieve_topk_t<ZMix1>(v, cls, ncls, vals, nmem, a_max, grid_blocks, topk_thr, improved, st);
        return sieve_topk_t<ZMix2>(v, cls, ncls, vals, nmem, a_max, grid_blocks, topk_thr, improved, st);
    }
    if (v.x1) return sieve_zgram_t<ZMix1>(v, cls, ncls, vals, a_max, grid_blocks, st);
    return sieve_zgram_t<ZMix2>(v, cls, ncls, vals, a_max, grid_blocks, st);
}

}  // namespace pn
