// Index construction: constant-window runs, FP64 prefix moments, sliding-DFT
// features with SimHash keys, non-constant ranks and the per-depth
// directories of every anchor (Sec. 3.1-3.4, Algorithm 1 phase A).
#include "kernels.cuh"
#include "prims.cuh"

namespace pn {
namespace {

__device__ __forceinline__ int series_of(const PnView &v, int64_t t) {
    return pn_find(v.series, v.nseries, t, [](const PnSeries &s) { return s.x_off; });
}

// Length of the run of equal samples starting at t, capped at the series' m_max.
// Window (q, m) is constant (max == min) exactly when runlen[q] >= m.
__global__ void k_runlen(PnView v, int64_t total, int32_t *runlen) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int s = series_of(v, t);
    const PnSeries &se = v.series[s];
    int64_t end = se.x_off + se.n;
    double x0 = v.x[t];
    int r = 1;
    while (r < se.m_max && t + r < end && v.x[t + r] == x0) ++r;
    runlen[t] = r;
}

// (v, v^2) with v = x - x[series start], and a head flag at each series start.
__global__ void k_moment_terms(PnView v, int64_t total, double2 *terms, uint8_t *head, double *shift) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int s = series_of(v, t);
    int64_t x0 = v.series[s].x_off;
    double c = v.x[x0];
    double d = v.x[t] - c;
    terms[t] = make_double2(d, d * d);
    head[t] = (uint8_t)(t == x0);
    if (t == x0) shift[s] = c;
}

// Places the inclusive sums at n+1 slots per series (slot 0 of a series is 0).
__global__ void k_moment_place(PnView v, int64_t total, const double2 *incl, double2 *sq) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int s = series_of(v, t);
    int64_t x0 = v.series[s].x_off;
    sq[t + s + 1] = incl[t];
    if (t == x0) sq[t + s] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------------------
// Features and signatures (Sec. 3.2 online update, Sec. 3.4 SimHash key).
//
// One thread advances one chunk of C consecutive windows of one anchor.  The
// chunk starts from a direct FP64 DFT of its first window (the periodic
// recompute of Sec. 3.2, here every C slides), then slides C-1 times:
//   X_{q+1,k} = e^{+2 pi i k/a} (X_{q,k} - t_q + t_{q+a}),
// in FP64 (plain form) or FP32 (mixed form).  Each window's bins 1..K' are
// scaled by 1/sigma (Lemma 1) into an FP32 row, and its B-bit key is
// bit l = 1{<g_{a,l}, F> >= 0}.  Rows of the 32 chunks of a warp are staged
// in shared memory and written as one contiguous 4 KB run (row layout
// pn_row()).
// ---------------------------------------------------------------------------
constexpr int FT_THREADS = 128;
constexpr int FT_WARPS = FT_THREADS / 32;

template <typename ST>
__global__ void __launch_bounds__(FT_THREADS) k_features(PnView v, const int32_t *blk_anchor,
                                                         const int32_t *blk_chunk0) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ai = blk_anchor[blockIdx.x];
    const PnAnchor A = v.anchors[ai];
    const PnSeries S = v.series[A.series];
    const int a = A.a, kp = A.kp, B = v.B, C = v.C;
    const int dims = 2 * (v.K - 1);
    double2 *tw = reinterpret_cast<double2 *>(smem);                 // (cos, sin)(2 pi t / a)
    float *gs = reinterpret_cast<float *>(tw + a);                   // B rows of PN_FEAT
    float *stage = gs + B * PN_FEAT;                                 // [warps][32][33]
    for (int t = threadIdx.x; t < a; t += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)t / (double)a, &sn, &cs);
        tw[t] = make_double2(cs, sn);
    }
    const float *gsrc = v.g + (int64_t)ai * (B + 1) * PN_FEAT;
    for (int t = threadIdx.x; t < B * PN_FEAT; t += blockDim.x) gs[t] = gsrc[t];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blk_chunk0[blockIdx.x] + threadIdx.x;
    const bool chunk_ok = c < A.nchunk;
    const int64_t q0 = c * C;
    const int64_t qend = chunk_ok ? min(A.nw, q0 + C) : q0;
    const double *xs = v.x + S.x_off;
    const double shift = v.shift[A.series];
    const int32_t *rl = v.runlen + S.x_off;
    const double2 *sqp = v.sq + S.x_off + A.series;
    const double inv_a = 1.0 / (double)a;

    ST Xr[PN_MAXK - 1], Xi[PN_MAXK - 1];
#pragma unroll
    for (int k = 0; k < PN_MAXK - 1; ++k) {
        Xr[k] = 0;
        Xi[k] = 0;
    }
    if constexpr (sizeof(ST) == 4) {
        if (q0 < qend && v.anc) {      // mixed form: chunk anchor from the tensor-core kernel
            const float *an = v.anc + (A.chunk_off + c) * PN_FEAT;
#pragma unroll
            for (int k = 0; k < PN_MAXK - 1; ++k) {
                Xr[k] = an[2 * k];
                Xi[k] = an[2 * k + 1];
            }
        }
    }
    if (q0 < qend && !(sizeof(ST) == 4 && v.anc)) {
        double dr[PN_MAXK - 1], di[PN_MAXK - 1];
        int idx[PN_MAXK - 1];
#pragma unroll
        for (int k = 0; k < PN_MAXK - 1; ++k) {
            dr[k] = 0.0;
            di[k] = 0.0;
            idx[k] = 0;
        }
        for (int r = 0; r < a; ++r) {
            const double t = xs[q0 + r] - shift;
#pragma unroll
            for (int k = 0; k < PN_MAXK - 1; ++k) {
                if (k < kp) {
                    const double2 w = tw[idx[k]];
                    dr[k] = fma(t, w.x, dr[k]);
                    di[k] = fma(-t, w.y, di[k]);
                    idx[k] += k + 1;
                    if (idx[k] >= a) idx[k] -= a;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < PN_MAXK - 1; ++k) {
            Xr[k] = (ST)dr[k];
            Xi[k] = (ST)di[k];
        }
    }

    float *st_w = stage + warp * 32 * 33;
    const int64_t warp_c0 = (int64_t)blk_chunk0[blockIdx.x] + warp * 32;
    float *Fa = v.F + A.row_off * PN_FEAT;
    for (int s = 0; s < C; ++s) {
        const int64_t q = q0 + s;
        const bool act = q < qend;
        float f[PN_FEAT];
#pragma unroll
        for (int t = 0; t < PN_FEAT; ++t) f[t] = 0.0f;
        if (act) {
            // moments from the FP64 prefix sums; the mixed form normalises in FP32
            const double2 pa = sqp[q], pb = sqp[q + a];
            const double ms = (pb.x - pa.x) * inv_a;
            const double var = (pb.y - pa.y) * inv_a - ms * ms;
            const double mu = ms + shift;
            const bool nonconst = rl[q] < a;
            const bool ok = nonconst && var > 0.0;
            if (v.precision == 0) {
                const double inv = ok ? 1.0 / sqrt(var) : 0.0;
                v.wmd[A.win_off + q] = make_double2(inv, -mu * inv);
                if (ok) {
#pragma unroll
                    for (int k = 0; k < PN_MAXK - 1; ++k) {
                        if (k < kp) {
                            f[2 * k] = (float)((double)Xr[k] * inv);
                            f[2 * k + 1] = (float)((double)Xi[k] * inv);
                        }
                    }
                }
            } else {
                const float invf = ok ? rsqrtf((float)var) : 0.0f;
                // z = fma(x, 1/sigma, -mu/sigma): one rounding, no cancellation for |mu| >> sigma
                v.wmf[A.win_off + q] = make_float2(invf, (float)(-mu * (double)invf));
                if (ok) {
#pragma unroll
                    for (int k = 0; k < PN_MAXK - 1; ++k) {
                        if (k < kp) {
                            f[2 * k] = (float)Xr[k] * invf;
                            f[2 * k + 1] = (float)Xi[k] * invf;
                        }
                    }
                }
            }
            uint32_t key = 0;
            if (nonconst) {
                for (int l = 0; l < B; ++l) {
                    float mg = pn_margin(gs + l * PN_FEAT, f, dims);
                    key |= (mg >= 0.0f ? 1u : 0u) << (B - 1 - l);
                }
            }
            v.sig[A.win_off + q] = key;
        }
        // stage the 32 rows of this warp and write them as one contiguous run
#pragma unroll
        for (int t = 0; t < PN_FEAT; ++t) st_w[lane * 33 + t] = f[t];
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int r = 4 * j + (lane >> 3);
            const int f4 = lane & 7;
            const int64_t cr = warp_c0 + r;
            if (cr < A.nchunk) {
                float4 o;
                o.x = st_w[r * 33 + 4 * f4 + 0];
                o.y = st_w[r * 33 + 4 * f4 + 1];
                o.z = st_w[r * 33 + 4 * f4 + 2];
                o.w = st_w[r * 33 + 4 * f4 + 3];
                reinterpret_cast<float4 *>(Fa + ((int64_t)s * A.nchunk + cr) * PN_FEAT)[f4] = o;
            }
        }
        __syncwarp();
        if (act && q + 1 < qend) {
            const ST delta = (ST)(xs[q + a] - xs[q]);
#pragma unroll
            for (int k = 0; k < PN_MAXK - 1; ++k) {
                if (k < kp) {
                    const double2 w = tw[k + 1];
                    const ST re = Xr[k] + delta;
                    const ST im = Xi[k];
                    if constexpr (sizeof(ST) == 8) {
                        Xr[k] = re * (ST)w.x - im * (ST)w.y;
                        Xi[k] = re * (ST)w.y + im * (ST)w.x;
                    } else {
                        // FP32 state: the rotation factor as a float-float pair, so its
                        // rounding does not compound into a phase drift over the chunk
                        const float ch = (float)w.x, sh = (float)w.y;
                        const float cl = (float)(w.x - (double)ch), sl = (float)(w.y - (double)sh);
                        Xr[k] = fmaf(re, ch, fmaf(-im, sh, fmaf(re, cl, -im * sl)));
                        Xi[k] = fmaf(re, sh, fmaf(im, ch, fmaf(re, sl, im * cl)));
                    }
                }
            }
        }
    }
}

// Non-constant flags per window and anchor heads for the rank scan.
__global__ void k_nonconst(PnView v, int64_t total, uint32_t *flag, uint8_t *head) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= total) return;
    int ai = pn_find(v.anchors, v.nanchors, w, [](const PnAnchor &A) { return A.win_off; });
    const PnAnchor &A = v.anchors[ai];
    int64_t q = w - A.win_off;
    flag[w] = q < A.nw ? (uint32_t)(v.runlen[v.series[A.series].x_off + q] < A.a) : 0u;
    head[w] = (uint8_t)(q == 0);
}

__global__ void k_nclist(PnView v, int64_t total, const uint32_t *flag) {
    int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= total || !flag[w]) return;
    int ai = pn_find(v.anchors, v.nanchors, w, [](const PnAnchor &A) { return A.win_off; });
    const PnAnchor &A = v.anchors[ai];
    v.nclist[A.win_off + v.cnt[w] - 1] = (uint32_t)(w - A.win_off);
}

// ---------------------------------------------------------------------------
// Directories (Sec. 3.4).  Level d of an anchor holds its first
// min(N, alpha 2^d) non-constant windows in stream order, addressed by the
// d-bit prefix of their keys: exactly the global-depth directory of the
// serial stream while its population is in (alpha 2^(d-1), alpha 2^d].
// One stable radix sort over the global bucket ids of all levels of all
// anchors leaves every bucket's entries in ascending start order.
// ---------------------------------------------------------------------------
__global__ void k_dir_items(PnView v, int64_t total, uint32_t *hist) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int li = pn_find(v.levels, v.nlevels, t, [](const PnLevel &L) { return L.item_off; });
    const PnLevel &L = v.levels[li];
    const PnAnchor &A = v.anchors[L.anchor];
    int64_t r = t - L.item_off;
    uint32_t N = A.nw > 0 ? v.cnt[A.win_off + A.nw - 1] : 0u;
    uint32_t key = 0xFFFFFFFFu, val = 0xFFFFFFFFu;
    if (r < (int64_t)N) {
        uint32_t q = v.nclist[A.win_off + r];
        uint32_t sg = v.sig[A.win_off + q];
        uint32_t pre = L.d > 0 ? (sg >> (v.B - L.d)) : 0u;
        key = (uint32_t)(L.bucket_base + pre);
        val = q;
        atomicAdd(&hist[key], 1u);
    }
    v.dir_keys[t] = key;
    v.dir_vals[t] = val;
}

// Search order: every query is keyed by the global bucket it probes first
// (its level's d-bit prefix), so warps running close together read the
// same candidate rows.  Constant windows and windows without an earlier
// valid partner sort last with key 0xFFFFFFFF.  Without a range table the
// query space is every window; with one, entry t is the window its range
// places there.
__global__ void k_query_keys(PnView v, int64_t total, uint32_t *keys, const PnQRange *rng, int32_t nrng) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= total) return;
    int ai;
    int64_t w;
    if (rng) {
        const int ri = pn_find(rng, nrng, t, [](const PnQRange &r) { return r.off; });
        ai = rng[ri].anchor;
        w = v.anchors[ai].win_off + rng[ri].q_lo + (t - rng[ri].off);
    } else {
        w = t;
        ai = pn_find(v.anchors, v.nanchors, w, [](const PnAnchor &A) { return A.win_off; });
    }
    const PnAnchor &A = v.anchors[ai];
    const PnSeries &S = v.series[A.series];
    const int64_t q = w - A.win_off;
    uint32_t key = 0xFFFFFFFFu;
    if (v.runlen[S.x_off + q] < A.a && q >= S.excl) {
        const int beta = (v.beta > 0 && v.beta < S.excl) ? v.beta : S.excl;
        const int64_t tau = q + A.a - 1;
        const int64_t tend = min(S.n - 1, (tau / beta + 1) * beta - 1);
        const uint32_t P = v.cnt[A.win_off + tend - A.a + 1];
        const int d = pn_depth(P, v.alpha, v.B);
        const uint32_t sg = v.sig[w];
        key = (uint32_t)(v.levels[A.level_begin + d].bucket_base + (d > 0 ? (sg >> (v.B - d)) : 0u));
    }
    keys[t] = key;
    v.qorder[t] = (uint32_t)w;
}

inline unsigned grid_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_runlen(const PnView &v, int64_t total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    k_runlen<<<grid_for(total, 256), 256, 0, st>>>(v, total, const_cast<int32_t *>(v.runlen));
    return cudaGetLastError();
}

cudaError_t launch_moments(const PnView &v, int64_t total, double2 *sq_out, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    double2 *terms = nullptr;
    uint8_t *head = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&terms, sizeof(double2) * total, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&head, total, st);
    if (e == cudaSuccess) {
        k_moment_terms<<<grid_for(total, 256), 256, 0, st>>>(v, total, terms, head, const_cast<double *>(v.shift));
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = seg_scan_d2(terms, head, terms, total, st);
    if (e == cudaSuccess) {
        k_moment_place<<<grid_for(total, 256), 256, 0, st>>>(v, total, terms, sq_out);
        e = cudaGetLastError();
    }
    if (terms) cudaFreeAsync(terms, st);
    if (head) cudaFreeAsync(head, st);
    return e;
}

size_t features_smem(int a_max, int B) {
    return sizeof(double2) * a_max + sizeof(float) * B * PN_FEAT + sizeof(float) * FT_WARPS * 32 * 33;
}

cudaError_t launch_features(const PnView &v, const int32_t *blk_anchor, const int32_t *blk_chunk0,
                            int32_t nblocks, int a_max, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    size_t sm = features_smem(a_max, v.B);
    cudaError_t e;
    if (v.precision == 0) {
        e = cudaFuncSetAttribute(k_features<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_features<double><<<nblocks, FT_THREADS, sm, st>>>(v, blk_anchor, blk_chunk0);
    } else {
        e = cudaFuncSetAttribute(k_features<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_features<float><<<nblocks, FT_THREADS, sm, st>>>(v, blk_anchor, blk_chunk0);
    }
    return cudaGetLastError();
}

cudaError_t launch_ranks(const PnView &v, int64_t total, cudaStream_t st) {
    if (total <= 0) return cudaSuccess;
    uint32_t *flag = nullptr;
    uint8_t *head = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&flag, sizeof(uint32_t) * total, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&head, total, st);
    if (e == cudaSuccess) {
        k_nonconst<<<grid_for(total, 256), 256, 0, st>>>(v, total, flag, head);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = seg_scan_u32(flag, head, v.cnt, total, st);
    if (e == cudaSuccess) {
        k_nclist<<<grid_for(total, 256), 256, 0, st>>>(v, total, flag);
        e = cudaGetLastError();
    }
    if (flag) cudaFreeAsync(flag, st);
    if (head) cudaFreeAsync(head, st);
    return e;
}

cudaError_t launch_directory(const PnView &v, int64_t total_items, int64_t total_buckets, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(v.bstart, 0, sizeof(uint32_t) * (total_buckets + 1), st);
    if (e != cudaSuccess || total_items <= 0) return e;
    k_dir_items<<<grid_for(total_items, 256), 256, 0, st>>>(v, total_items, v.bstart);
    e = cudaGetLastError();
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= total_buckets) ++bits;
    if (e == cudaSuccess) e = radix_sort_pairs(v.dir_keys, v.dir_vals, total_items, bits, st);
    if (e == cudaSuccess) e = excl_scan_u32(v.bstart, v.bstart, total_buckets + 1, nullptr, st);
    return e;
}

cudaError_t launch_query_order(const PnView &v, int64_t total, int64_t total_buckets, cudaStream_t st,
                               const PnQRange *rng, int32_t nrng) {
    if (total <= 0) return cudaSuccess;
    uint32_t *keys = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&keys, sizeof(uint32_t) * total, st);
    if (e != cudaSuccess) return e;
    k_query_keys<<<grid_for(total, 256), 256, 0, st>>>(v, total, keys, rng, nrng);
    e = cudaGetLastError();
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= total_buckets) ++bits;
    if (e == cudaSuccess) e = radix_sort_pairs(keys, v.qorder, total, bits, st);
    cudaFreeAsync(keys, st);
    return e;
}

}  // namespace pn
