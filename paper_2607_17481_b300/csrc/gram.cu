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

// TOPK: the top-k sieve.  Instead of the row and column rules, a pair is
// evaluated exactly only when its estimate minus the margin is below thr2
// (the square of a distance the top list already holds) and below one of
// its two cells: the pass looks only for pairs that can enter the list.
template <class Z, bool TOPK>
__global__ void __launch_bounds__(ZG_THREADS) k_sieve_zgram(PnView v, const PnClass *cls, const uint4 *tiles,
                                                            int64_t ntiles, const uint32_t *members, int kpad_max,
                                                            unsigned long long *work, float thr2) {
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
            for (int c0 = 0; !TOPK && c0 < ZG_B; c0 += 32) {
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
                        if constexpr (TOPK) {
                            s = dd - M < thr2 && (dd - M < tu2 || dd - M < tv * tv);
                        } else {
                            const bool keep_u = dd - M < tu2 && dd <= rmin + tol_row;
                            const bool keep_v = dd - M < tv * tv && dd <= __int_as_float(sh.colmin[vc]) +
                                                                              0.00390625f * (nv_ + nmax_a) + 2.0f * mabs;
                            s = keep_u || keep_v;
                        }
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

// The top-k sieve as its own kernel: eight warps (warps w and w + 4 read the
// same accumulator lanes, columns 0-63 and 64-127), and a fast test per pair
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
    float zref[ZG_AMAX];
    float2 nbt[ZG_B];                          // ((1 - 2^-9) |y_v|^2, P[v]^2) of the column block
    unsigned long long rkey[ZG_B], ckey[ZG_B];
    uint32_t queue[ZT_WARPS][ZT_Q];
    int nmax_a, nmax_b;
    int fail;
    uint32_t taddr;
    __align__(8) uint64_t mbar;
    unsigned long long run;
};

template <class Z>
__global__ void __launch_bounds__(ZT_THREADS) k_sieve_topk(PnView v, const PnClass *cls, const uint4 *tiles,
                                                           int64_t ntiles, const uint32_t *members, int kpad_max,
                                                           unsigned long long *work, float thr2) {
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
    uint32_t staged_cls = 0xFFFFFFFFu, staged_bu = 0xFFFFFFFFu;
    const int quarter = warp & 3, half = warp >> 2;
    const int u = quarter * 32 + lane;

    for (;;) {
        __syncthreads();
        if (tid == 0) sh.run = atomicAdd(work, (unsigned long long)ZT_RUN);
        __syncthreads();
        const int64_t run0 = (int64_t)sh.run;
        if (run0 >= ntiles || sh.fail) break;
        const int64_t run1 = min(ntiles, run0 + ZT_RUN);
        for (int64_t t = run0; t < run1; ++t) {
            const uint4 tl = tiles[t];
            const PnClass c = cls[tl.x];
            const PnAnchor &A = v.anchors[c.anchor];
            const PnSeries &S = v.series[A.series];
            const int a = A.a;
            const int kp = (a + 15) & ~15;
            const int excl = S.excl;
            const int u0 = (int)tl.y * ZG_B, v0 = (int)tl.z * ZG_B;
            const int nu = min(ZG_B, (int)c.size - u0), nv = min(ZG_B, (int)c.size - v0);
            const bool diag = tl.y == tl.z;
            unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
            __syncthreads();
            const bool new_row = tl.x != staged_cls || tl.y != staged_bu;
            if (tid == 0) {
                if (new_row) sh.nmax_a = 0;
                sh.nmax_b = 0;
            }
            if (tid < ZG_B) {
                sh.rkey[tid] = PN_EMPTY_KEY;
                sh.ckey[tid] = PN_EMPTY_KEY;
            }
            if (new_row) {
                const uint32_t cr = members[(int64_t)c.moff + u0];
                const auto mref = Z::load(v, A.win_off + cr);
                const auto *xref = Z::samples(v, S.x_off + cr);
                for (int k = tid; k < kp; k += ZT_THREADS) sh.zref[k] = k < a ? Z::z(mref, xref[k]) : 0.0f;
                __syncthreads();
                zg_stage<Z, ZT_WARPS>(v, A, S, members, (int64_t)c.moff + u0, nu, a, kp, tA, sh.A, &sh.nmax_a, prow,
                                      sh.zref, warp, lane);
            } else {
                __syncthreads();
            }
            zg_stage<Z, ZT_WARPS>(v, A, S, members, (int64_t)c.moff + v0, nv, a, kp, tB, sh.B, &sh.nmax_b, prow,
                                  sh.zref, warp, lane);
            staged_cls = tl.x;
            staged_bu = tl.y;
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncthreads();
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (tid < ZG_B) sh.nbt[tid] = make_float2(0.998046875f * sh.B.n[tid], sh.B.t[tid] * sh.B.t[tid]);
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
            // fast bound: (1 - 2^-9) |y_v|^2 - 2 G < min(thr2, max(P[u]^2, P[v]^2)) + cu, with
            // cu = a 2^-14 - (1 - 2^-9) |y_u|^2 and a slack of 2^-20 of the magnitudes involved
            const float slack = 9.5367432e-07f * (thr2 + mabs + nu_ + 1.0f);
            const float cu = urow ? mabs - 0.998046875f * nu_ + slack : -__int_as_float(0x7f800000);
            const float kt = thr2 + cu, ku = tu2 + cu;
            const int64_t pu = (int64_t)sh.A.s[u];
            const auto *xs = Z::samples(v, S.x_off);
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
                uint32_t hit = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float2 nt = sh.nbt[c0 + j];
                    const float lim = fminf(kt, fmaxf(ku, nt.y + cu));
                    hit |= (fmaf(-2.0f, __uint_as_float(r[j]), nt.x) < lim ? 1u : 0u) << j;
                }
                if (!__any_sync(0xffffffffu, hit != 0u)) continue;        // the common case: no pair near the list
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int vc = c0 + j;
                    bool keep = ((hit >> j) & 1u) && vc < nv && (!diag || u < vc) && sh.B.m[vc].x != 0.0f;
                    if (keep) keep = llabs(pu - (int64_t)sh.B.s[vc]) >= excl;
                    if (keep) {
                        const float nv_ = sh.B.n[vc];
                        const float dd = fmaxf(0.0f, nu_ + nv_ - 2.0f * __uint_as_float(r[j]));
                        const float M = 0.001953125f * (nu_ + nv_) + mabs;
                        const float tv = sh.B.t[vc];
                        keep = dd - M < thr2 && (dd - M < tu2 || dd - M < tv * tv);
                    }
                    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
                    if (keep) sh.queue[warp][qn + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)u << 16) | (uint32_t)vc;
                    qn += __popc(bal);
                    if (qn > ZT_Q - 32) {
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
            __syncthreads();
            if (tid < ZG_B) {
                if (sh.rkey[tid] != PN_EMPTY_KEY) atomicMin(&prow[sh.A.s[tid]], sh.rkey[tid]);
                if (sh.ckey[tid] != PN_EMPTY_KEY) atomicMin(&prow[sh.B.s[tid]], sh.ckey[tid]);
            }
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

template <class Z, bool TOPK>
cudaError_t sieve_zgram_t(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int a_max,
                          int grid_blocks, float thr2, cudaStream_t st) {
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
        const int run = TOPK ? ZT_RUN : ZG_RUN;
        const int64_t g = std::min<int64_t>((ntiles + run - 1) / run, (int64_t)grid_blocks);
        if constexpr (TOPK) {
            e = pn_allow_smem(k_sieve_topk<Z>, sm);
            if (e == cudaSuccess) {
                k_sieve_topk<Z><<<(unsigned)g, ZT_THREADS, sm, st>>>(v, cls, tiles, ntiles, vals, kpad, work, thr2);
                e = cudaGetLastError();
            }
        } else {
            e = pn_allow_smem(k_sieve_zgram<Z, false>, sm);
            if (e == cudaSuccess) {
                k_sieve_zgram<Z, false><<<(unsigned)g, ZG_THREADS, sm, st>>>(v, cls, tiles, ntiles, vals, kpad, work,
                                                                             thr2);
                e = cudaGetLastError();
            }
        }
    }
    for (void *p : {(void *)cnt, (void *)off, (void *)tot, (void *)tot64, (void *)tiles})
        if (p) cudaFreeAsync(p, st);
    return e;
}

}  // namespace

bool sieve_gram_supported(int a_max) { return a_max <= ZG_AMAX; }

cudaError_t launch_sieve_gram(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int a_max,
                              int grid_blocks, cudaStream_t st, double topk_thr) {
    if (ncls <= 0) return cudaSuccess;
    if (topk_thr >= 0.0) {
        const float t = (float)topk_thr;
        const float thr2 = t * t * (1.0f + 1e-6f) + 1e-12f;       // FP32 rounding of the square
        if (v.x1) return sieve_zgram_t<ZMix1, true>(v, cls, ncls, vals, a_max, grid_blocks, thr2, st);
        return sieve_zgram_t<ZMix2, true>(v, cls, ncls, vals, a_max, grid_blocks, thr2, st);
    }
    if (v.x1) return sieve_zgram_t<ZMix1, false>(v, cls, ncls, vals, a_max, grid_blocks, 0.0f, st);
    return sieve_zgram_t<ZMix2, false>(v, cls, ncls, vals, a_max, grid_blocks, 0.0f, st);
}

}  // namespace pn
