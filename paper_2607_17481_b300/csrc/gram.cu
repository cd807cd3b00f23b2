// Exhaustive hot-class sieve with a tensor-core Gram filter (Sec. 3.6's
// hot-class sieve, every valid pair of each class; the Parseval bound of
// Lemma 2 decides which pairs are evaluated exactly).
//
// For a tile of 128 x 128 members (u, v) of one class at anchor length a,
// the bound is LB^2 = (2/a) (|F_u|^2 + |F_v|^2 - 2 <F_u, F_v>) over the 30
// stored feature floats.  The Gram block <F_u, F_v> is one dense
// contraction [128 x 32] x [32 x 128]: the rows are staged in shared memory
// in the K-major no-swizzle canonical layout, split into TF32 hi + lo
// parts, and one thread issues 4 K-steps x 3 tcgen05.mma kind::tf32
// (hi*hi + hi*lo + lo*hi) into a 128 x 128 FP32 accumulator in tensor
// memory.  Each warp then reads its 32 rows back with tcgen05.ld and tests
// every pair against max(P[u], P[v]) with the (1 - lambda) shrink of
// Algorithm 1 and an additive error margin; the survivors are evaluated
// exactly (FP32, the search's arithmetic) and lower both cells.
//
// Error margin.  With x = hi + lo, hi = rna-TF32(x) (|x - hi| <= 2^-11|x|)
// and lo truncated to TF32 by the MMA (<= 2^-21 |x|), each product is
// carried to within ~2^-19.7 |x_k y_k|; FP32 accumulation of the 96 partial
// products adds at most 96 * 2^-24 of their magnitudes.  So
// |G - <F_u, F_v>| <= 2^-17 |F_u||F_v| <= 2^-17 (n_u + n_v) / 2, and the
// FP32 norms n = |F|^2 are within 2^-19 n.  The computed LB^2 is therefore
// within (2/a)(n_u + n_v)(2^-17 + 2^-19) of the exact one; the test uses
// the margin (2/a)(n_u + n_v) 2^-15, about three times that.  A pair is
// skipped only when (1 - lambda)^2 (LB^2 - margin) >= max(P[u], P[v])^2, so
// every pair the exact bound keeps is evaluated.
//
// Waits on the MMA's completion are bounded: on timeout the kernel records
// the error word, waits once more (bounded), frees its tensor memory and
// returns; the request reports ETIMEOUT.
#include <type_traits>

#include "emit.cuh"
#include "prims.cuh"
#include "tcgen05.cuh"
#include "zops.cuh"

namespace pn {
namespace {

constexpr int GR_B = 128;          // members per tile side (MMA M and N)
constexpr int GR_K = 32;           // feature floats per row (30 used)
constexpr int GR_THREADS = 128;    // 4 warps: warp w owns tile rows / TMEM lanes 32w..32w+31
constexpr int GR_Q = 256;          // survivor queue per warp
constexpr int GR_SPIN = 1 << 22;   // try_wait iterations before giving up

__global__ void k_gram_tile_count(const PnClass *cls, int32_t ncls, uint32_t *cnt) {
    const int ci = blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= ncls) return;
    const uint32_t nb = (cls[ci].size + GR_B - 1) / GR_B;
    cnt[ci] = nb * (nb + 1) / 2;
}

// One warp per class writes its upper-triangular tiles (class, bu, bv).
__global__ void k_gram_tile_fill(const PnClass *cls, int32_t ncls, const uint32_t *off, uint4 *tiles) {
    const int ci = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (ci >= ncls) return;
    const uint32_t nb = (cls[ci].size + GR_B - 1) / GR_B;
    const uint32_t total = nb * (nb + 1) / 2;
    for (uint32_t t = lane; t < total; t += 32) {
        uint32_t bu = 0, rem = t;
        while (rem >= nb - bu) {
            rem -= nb - bu;
            ++bu;
        }
        tiles[off[ci] + t] = make_uint4((uint32_t)ci, bu, bu + rem, 0u);
    }
}

// Exact distances of up to four queued pairs at once, by the whole warp
// (lanes over samples, four independent sums); each key lowers the tile's
// shared row and column minima, which are written to the cells once per tile.
template <class Z>
__device__ __forceinline__ void gram_eval4(const typename Z::X *xs, int a, const uint32_t *q, int nq,
                                           const uint32_t *su, const uint32_t *sv, const float2 *mA,
                                           const float2 *mB, unsigned long long *rmin, unsigned long long *cmin,
                                           int lane) {
    typename Z::M zu[4], zv[4];
    uint32_t uu[4], vv[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t e = q[p < nq ? p : 0];
        uu[p] = e >> 16;
        vv[p] = e & 0xFFFFu;
        zu[p].x = mA[uu[p]].x;
        zu[p].y = mA[uu[p]].y;
        zv[p].x = mB[vv[p]].x;
        zv[p].y = mB[vv[p]].y;
    }
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int r = lane; r < a; r += 32) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float d = Z::z(zu[p], xs[su[uu[p]] + r]) - Z::z(zv[p], xs[sv[vv[p]] + r]);
            acc[p] = fmaf(d, d, acc[p]);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const float d = sqrtf(pn_warp_sum(acc[p]));
        if (lane == p && p < nq) {
            atomicMin(&rmin[uu[p]], pn_pack_f(d, sv[vv[p]]));
            atomicMin(&cmin[vv[p]], pn_pack_f(d, su[uu[p]]));
        }
    }
}

template <class Z>
__global__ void __launch_bounds__(GR_THREADS) k_sieve_gram(PnView v, const PnClass *cls, const uint4 *tiles,
                                                        int64_t ntiles, const uint32_t *members) {
    extern __shared__ __align__(128) float gsm[];
    float *Ahi = gsm;                                 // [128 x 32] canonical, each
    float *Alo = Ahi + GR_B * GR_K;
    float *Bhi = Alo + GR_B * GR_K;
    float *Blo = Bhi + GR_B * GR_K;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t taddr_s;
    __shared__ int fail_s;
    __shared__ float nA[GR_B], nB[GR_B], tA[GR_B], tB[GR_B];
    __shared__ uint32_t su[GR_B], sv[GR_B];
    __shared__ float2 mA[GR_B], mB[GR_B];
    __shared__ uint32_t queue[GR_THREADS / 32][GR_Q];
    __shared__ unsigned long long rmin[GR_B], cmin[GR_B];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kg = GR_K / 4;
    if (tid == 0) {
        fail_s = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&taddr_s)),
                     "r"(GR_B));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = taddr_s;
    const uint32_t idesc = umma_idesc_tf32(GR_B, GR_B);
    const float shrink = 1.0f - v.lam;
    const float shrink2 = shrink * shrink;
    uint32_t phase = 0;
    bool ok = true;
    unsigned long long n_ex = 0;

    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const uint4 tl = tiles[t];
        const PnClass c = cls[tl.x];
        const PnAnchor &A = v.anchors[c.anchor];
        const PnSeries &S = v.series[A.series];
        const int a = A.a;
        const int u0 = (int)tl.y * GR_B, v0 = (int)tl.z * GR_B;
        const int nu = min(GR_B, (int)c.size - u0), nv = min(GR_B, (int)c.size - v0);
        const bool diag = tl.y == tl.z;
        unsigned long long *prow = v.prof + S.row_off + (int64_t)(a - S.m_min) * S.ld;
        const float *Fa = v.F + A.row_off * PN_FEAT;
        const uint32_t nch = (uint32_t)A.nchunk;
        __syncthreads();                                  // the previous tile's staging and queues are done
        {
            const int i = tid;                            // GR_THREADS == GR_B: one member per side per thread
            const uint32_t xu = i < nu ? members[c.moff + u0 + i] : 0u;
            const uint32_t xv = i < nv ? members[c.moff + v0 + i] : 0u;
            su[i] = xu;
            sv[i] = xv;
            const auto mu = Z::load(v, A.win_off + xu), mv = Z::load(v, A.win_off + xv);
            mA[i] = i < nu ? make_float2(mu.x, mu.y) : make_float2(0.0f, 0.0f);
            mB[i] = i < nv ? make_float2(mv.x, mv.y) : make_float2(0.0f, 0.0f);
            tA[i] = i < nu ? pn_key_distf(__ldcg(&prow[xu])) : 0.0f;
            tB[i] = i < nv ? pn_key_distf(__ldcg(&prow[xv])) : 0.0f;
            // squared row norms (fixed FMA order)
            float na = 0.0f, nb = 0.0f;
            if (i < nu) {
                const float4 *r4 = reinterpret_cast<const float4 *>(Fa + (size_t)pn_row32(xu, v.cshift, nch) * PN_FEAT);
#pragma unroll
                for (int k = 0; k < GR_K / 4; ++k) {
                    const float4 f = r4[k];
                    na = fmaf(f.x, f.x, fmaf(f.y, f.y, fmaf(f.z, f.z, fmaf(f.w, f.w, na))));
                }
            }
            if (i < nv) {
                const float4 *r4 = reinterpret_cast<const float4 *>(Fa + (size_t)pn_row32(xv, v.cshift, nch) * PN_FEAT);
#pragma unroll
                for (int k = 0; k < GR_K / 4; ++k) {
                    const float4 f = r4[k];
                    nb = fmaf(f.x, f.x, fmaf(f.y, f.y, fmaf(f.z, f.z, fmaf(f.w, f.w, nb))));
                }
            }
            nA[i] = na;
            nB[i] = nb;
            rmin[i] = PN_EMPTY_KEY;
            cmin[i] = PN_EMPTY_KEY;
        }
        __syncthreads();
        // operands: member rows split into TF32 hi + lo (zero rows past the class)
        for (int e = tid; e < GR_B * GR_K; e += GR_THREADS) {
            const int i = e / GR_K, k = e - i * GR_K;
            const float fu = i < nu ? Fa[(size_t)pn_row32(su[i], v.cshift, nch) * PN_FEAT + k] : 0.0f;
            const float fv = i < nv ? Fa[(size_t)pn_row32(sv[i], v.cshift, nch) * PN_FEAT + k] : 0.0f;
            const float hu = tf32_hi(fu), hv = tf32_hi(fv);
            Ahi[kmaj(i, k, kg)] = hu;
            Alo[kmaj(i, k, kg)] = fu - hu;
            Bhi[kmaj(i, k, kg)] = hv;
            Blo[kmaj(i, k, kg)] = fv - hv;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t lbo = 128, sbo = kg * 128;
            for (int s = 0; s < GR_K / 8; ++s) {
                const uint32_t off = (uint32_t)(s * 2 * 32 * sizeof(float));
                const uint64_t ah = umma_desc(smem_u32(Ahi) + off, lbo, sbo);
                const uint64_t al = umma_desc(smem_u32(Alo) + off, lbo, sbo);
                const uint64_t bh = umma_desc(smem_u32(Bhi) + off, lbo, sbo);
                const uint64_t bl = umma_desc(smem_u32(Blo) + off, lbo, sbo);
                const uint32_t acc0 = s > 0 ? 1u : 0u;
                asm volatile("{ .reg .pred p; setp.ne.u32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }"
                             ::"r"(taddr), "l"(ah), "l"(bh), "r"(idesc), "r"(acc0));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(taddr), "l"(ah), "l"(bl),
                             "r"(idesc));
                asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;" ::"r"(taddr), "l"(al), "l"(bh),
                             "r"(idesc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar))
                         : "memory");
        }
        if (!mbar_wait(smem_u32(&mbar), phase, GR_SPIN)) {
            if (lane == 0) atomicExch(&fail_s, 1);
        }
        phase ^= 1u;
        __syncthreads();
        if (fail_s) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // epilogue: row u = 32 warp + lane against the tile's columns
        const int u = warp * 32 + lane;
        const bool urow = u < nu && mA[u].x != 0.0f;
        const float nu_ = nA[u], tu = tA[u];
        const int64_t pu = (int64_t)su[u];
        const float scale = 2.0f / (float)a;
        const auto *xs = Z::samples(v, S.x_off);
        int qn = 0;
        for (int c0 = 0; c0 < nv; c0 += 32) {
            uint32_t r[32];
            const uint32_t ta = taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"
                "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int vc = c0 + j;
                bool s = urow && vc < nv && (!diag || u < vc) && mB[vc].x != 0.0f;
                if (s) s = llabs(pu - (int64_t)sv[vc]) >= S.excl;
                if (s) {
                    const float n2 = nu_ + nB[vc];
                    const float lb2 = fmaxf(0.0f, scale * (n2 - 2.0f * __uint_as_float(r[j])));
                    const float margin = scale * n2 * 3.0517578e-5f;          // (2/a)(n_u + n_v) 2^-15
                    const float thr = fmaxf(tu, tB[vc]);
                    s = !(shrink2 * (lb2 - margin) >= thr * thr);            // an infinite threshold keeps it
                }
                const uint32_t bal = __ballot_sync(0xffffffffu, s);
                if (s) queue[warp][qn + __popc(bal & ((1u << lane) - 1u))] = ((uint32_t)u << 16) | (uint32_t)vc;
                qn += __popc(bal);
                if (qn > GR_Q - 32) {                     // warp-uniform: evaluate the queued pairs
                    __syncwarp();
                    for (int e = 0; e < qn; e += 4)
                        gram_eval4<Z>(xs, a, &queue[warp][e], min(4, qn - e), su, sv, mA, mB, rmin, cmin, lane);
                    n_ex += (unsigned long long)qn;
                    qn = 0;
                    __syncwarp();
                }
            }
        }
        __syncwarp();
        for (int e = 0; e < qn; e += 4)
            gram_eval4<Z>(xs, a, &queue[warp][e], min(4, qn - e), su, sv, mA, mB, rmin, cmin, lane);
        n_ex += (unsigned long long)qn;
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();                                   // every warp's keys are in the tile minima
        if (rmin[tid] != PN_EMPTY_KEY) atomicMin(&prow[su[tid]], rmin[tid]);
        if (cmin[tid] != PN_EMPTY_KEY) atomicMin(&prow[sv[tid]], cmin[tid]);
    }
    if (!ok && tid == 0) {
        atomicExch(v.err, PN_ERR_TC_TIMEOUT);
        mbar_wait(smem_u32(&mbar), phase ^ 1u, GR_SPIN);   // let an MMA still in flight finish (bounded)
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(GR_B));
    if (lane == 0 && v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_SIEVE], n_ex);
}

template <class Z>
cudaError_t sieve_gram_t(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals, int grid_blocks,
                         cudaStream_t st) {
    uint32_t *cnt = nullptr, *off = nullptr, *tot = nullptr;
    uint4 *tiles = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&cnt, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&off, 4 * (size_t)ncls, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&tot, 4, st);
    if (e == cudaSuccess) {
        k_gram_tile_count<<<(unsigned)((ncls + 255) / 256), 256, 0, st>>>(cls, ncls, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = excl_scan_u32(cnt, off, ncls, tot, st);
    uint32_t ntiles = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ntiles, tot, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ntiles > 0) e = cudaMallocAsync((void **)&tiles, sizeof(uint4) * (size_t)ntiles, st);
    if (e == cudaSuccess && ntiles > 0) {
        k_gram_tile_fill<<<(unsigned)(((int64_t)ncls * 32 + 255) / 256), 256, 0, st>>>(cls, ncls, off, tiles);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && ntiles > 0) {
        const size_t sm = sizeof(float) * 4 * GR_B * GR_K;
        e = pn_allow_smem(k_sieve_gram<Z>, sm);
        if (e == cudaSuccess) {
            const int64_t g = std::min<int64_t>((int64_t)ntiles, (int64_t)grid_blocks);
            k_sieve_gram<Z><<<(unsigned)g, GR_THREADS, sm, st>>>(v, cls, tiles, (int64_t)ntiles, vals);
            e = cudaGetLastError();
        }
    }
    for (void *p : {(void *)cnt, (void *)off, (void *)tot, (void *)tiles})
        if (p) cudaFreeAsync(p, st);
    return e;
}

}  // namespace

cudaError_t launch_sieve_gram(const PnView &v, const PnClass *cls, int32_t ncls, const uint32_t *vals,
                              int grid_blocks, cudaStream_t st) {
    if (ncls <= 0) return cudaSuccess;
    if (v.x1) return sieve_gram_t<ZMix1>(v, cls, ncls, vals, grid_blocks, st);
    return sieve_gram_t<ZMix2>(v, cls, ncls, vals, grid_blocks, st);
}

}  // namespace pn
