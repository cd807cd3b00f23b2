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
// Window moments table (Sec. 3.2: mu = S/m, sigma^2 = Q/m - mu^2 from the
// FP64 prefix sums): per window (1/sigma, -mu/sigma), FP32 in the mixed form
// and FP64 in the plain form; 1/sigma = 0 marks a constant or degenerate
// window.  One thread per window.
// ---------------------------------------------------------------------------
__global__ void k_moment_table(PnView v, int64_t total) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= total) return;
    const int ai = pn_find(v.anchors, v.nanchors, w, [](const PnAnchor &A) { return A.win_off; });
    const PnAnchor &A = v.anchors[ai];
    const int64_t q = w - A.win_off;
    if (q >= A.nw) return;
    const PnSeries &S = v.series[A.series];
    const int a = A.a;
    const double2 *sqp = v.sq + S.x_off + A.series;
    const double2 pa = sqp[q], pb = sqp[q + a];
    const double inv_a = 1.0 / (double)a;
    const double ms = (pb.x - pa.x) * inv_a;
    const double var = (pb.y - pa.y) * inv_a - ms * ms;
    const double mu = ms + v.shift[A.series];
    const bool ok = v.runlen[S.x_off + q] < a && var > 0.0;
    if (v.precision == 0) {
        const double inv = ok ? 1.0 / sqrt(var) : 0.0;
        v.wmd[w] = make_double2(inv, -mu * inv);
    } else {
        const float invf = ok ? rsqrtf((float)var) : 0.0f;
        // z = fma(x, 1/sigma, -mu/sigma): one rounding, no cancellation for |mu| >> sigma
        v.wmf[w] = make_float2(invf, (float)(-mu * (double)invf));
    }
}

// ---------------------------------------------------------------------------
// Features and signatures (Sec. 3.2 online update, Sec. 3.4 SimHash key).
//
// One warp advances one chunk of C consecutive windows of one anchor: lane k
// (k < K') carries bin k+1 of the spectral state.  The chunk starts from a
// direct DFT of its first window (the periodic recompute of Sec. 3.2, here
// every C slides: tensor-core anchors in the mixed form, an FP64 direct DFT
// otherwise), then slides C-1 times,
//   X_{q+1,k} = e^{+2 pi i k/a} (X_{q,k} - t_q + t_{q+a}),
// in FP64 (plain form) or FP32 with a float-float rotation factor (mixed).
// Per window the bins are scaled by 1/sigma (Lemma 1) into an FP32 row
// written by the whole warp as one 128-byte store, and lane l < B computes
// <g_{a,l}, F>: the B-bit key is the warp's ballot of the signs.  Every lane
// works on every window, so the per-window latency is a few dozen warp
// instructions rather than a thread's whole projection loop.
// ---------------------------------------------------------------------------
constexpr int FT_WARPS = PN_FT_CHUNKS;
constexpr int FT_THREADS = FT_WARPS * 32;

template <typename ST>
__global__ void __launch_bounds__(FT_THREADS) k_features(PnView v, const int32_t *blk_anchor,
                                                         const int32_t *blk_chunk0) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(16) float frow[FT_WARPS][PN_FEAT];
    const int ai = blk_anchor[blockIdx.x];
    const PnAnchor A = v.anchors[ai];
    const PnSeries S = v.series[A.series];
    const int a = A.a, kp = A.kp, B = v.B, C = v.C;
    const int dims = 2 * (v.K - 1);
    // (cos, sin)(2 pi t / a) for t < a, needed only where chunk anchors come
    // from the FP64 direct DFT (plain form, or mixed form without
    // tensor-core anchors); otherwise each lane takes its own bin's factor
    double2 *tw = reinterpret_cast<double2 *>(smem);
    const bool direct = sizeof(ST) == 8 || !v.anc;
    if (direct) {
        for (int t = threadIdx.x; t < a; t += blockDim.x) {
            double sn, cs;
            sincospi(2.0 * (double)t / (double)a, &sn, &cs);
            tw[t] = make_double2(cs, sn);
        }
    }
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t c = (int64_t)blk_chunk0[blockIdx.x] + warp;
    const int64_t q0 = c * C;
    if (c >= A.nchunk || q0 >= A.nw) return;                         // warp-uniform
    const int64_t qend = min(A.nw, q0 + C);
    const double *xs = v.x + S.x_off;
    const double shift = v.shift[A.series];
    const int32_t *rl = v.runlen + S.x_off;
    float *Fa = v.F ? v.F + A.row_off * PN_FEAT : nullptr;
    __half *Fha = v.Fh ? v.Fh + A.row_off * PN_FEAT : nullptr;
    float *fr = frow[warp];
    const bool bin = lane < kp;

    // projection row of lane l (l < B; lane B: the sieve direction), in registers
    float g[PN_FEAT - 2];
    {
        const float *gsrc = v.g + ((int64_t)ai * (B + 1) + (lane <= B ? lane : 0)) * PN_FEAT;
#pragma unroll
        for (int t = 0; t < PN_FEAT - 2; ++t) g[t] = gsrc[t];
    }
    // chunk anchor of bin lane+1
    ST Xr = 0, Xi = 0;
    bool have = false;
    if constexpr (sizeof(ST) == 4) {
        if (v.anc) {
            const float *an = v.anc + (A.chunk_off + c) * PN_FEAT;
            if (bin) {
                Xr = an[2 * lane];
                Xi = an[2 * lane + 1];
            }
            have = true;
        }
    }
    if (!have && bin) {
        double dr = 0.0, di = 0.0;
        int idx = 0;
        for (int r = 0; r < a; ++r) {
            const double t = xs[q0 + r] - shift;
            const double2 w = tw[idx];
            dr = fma(t, w.x, dr);
            di = fma(-t, w.y, di);
            idx += lane + 1;
            if (idx >= a) idx -= a;
        }
        Xr = (ST)dr;
        Xi = (ST)di;
    }
    // rotation factor of bin lane+1 (the table's arithmetic, bit for bit)
    double2 wk;
    if (direct) {
        wk = tw[bin ? lane + 1 : 0];
    } else {
        double sn, cs;
        sincospi(2.0 * (double)(bin ? lane + 1 : 0) / (double)a, &sn, &cs);
        wk = make_double2(cs, sn);
    }
    const float ch = (float)wk.x, sh = (float)wk.y;
    const float cl = (float)(wk.x - (double)ch), sl = (float)(wk.y - (double)sh);

    // sample differences t_{q+a} - t_q of the slide after window q, taken in
    // FP64 (exact for float32 series) and rounded to the state type once:
    // lane l computes the one of window q + l for 32 windows at a time, and
    // each slide takes its own by a shuffle
    ST dlane = 0;
    for (int64_t q = q0; q < qend; ++q) {
        if (((q - q0) & 31) == 0) {
            const int64_t ql = q + lane;
            dlane = ql + 1 < qend ? (ST)(xs[ql + a] - xs[ql]) : (ST)0;
        }
        const bool nonconst = rl[q] < a;
        float f_re = 0.0f, f_im = 0.0f;
        if (v.precision == 0) {
            const double inv = v.wmd[A.win_off + q].x;
            if (bin && inv != 0.0) {
                f_re = (float)((double)Xr * inv);
                f_im = (float)((double)Xi * inv);
            }
        } else {
            const float invf = v.wmf[A.win_off + q].x;
            if (bin && invf != 0.0f) {
                f_re = (float)Xr * invf;
                f_im = (float)Xi * invf;
            }
        }
        if (lane < PN_FEAT / 2) {
            fr[2 * lane] = f_re;
            fr[2 * lane + 1] = f_im;
        }
        __syncwarp();
        if (Fha) Fha[(int64_t)pn_row(q, C, A.nchunk) * PN_FEAT + lane] = __float2half_rn(fr[lane]);
        else Fa[(int64_t)pn_row(q, C, A.nchunk) * PN_FEAT + lane] = fr[lane];
        // <g_l, F> in the fixed FMA order of pn_margin, then the key by ballot
        float mg = 0.0f;
        const float4 *f4 = reinterpret_cast<const float4 *>(fr);
#pragma unroll
        for (int t4 = 0; t4 < (PN_FEAT - 2 + 3) / 4; ++t4) {
            const float4 f = f4[t4];
            const float fv[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int t = 4 * t4 + u;
                if (t < PN_FEAT - 2 && t < dims) mg = fmaf(g[t], fv[u], mg);
            }
        }
        const uint32_t bits = __ballot_sync(0xffffffffu, lane < B && mg >= 0.0f);
        if (lane == 0) v.sig[A.win_off + q] = nonconst ? (__brev(bits) >> (32 - B)) : 0u;
        if (lane == B) v.sproj[A.win_off + q] = mg;          // the sieve's sort key
        __syncwarp();
        const ST delta = __shfl_sync(0xffffffffu, dlane, (int)((q - q0) & 31));
        if (q + 1 < qend) {
            if (bin) {
                const ST re = Xr + delta;
                const ST im = Xi;
                if constexpr (sizeof(ST) == 8) {
                    Xr = re * (ST)wk.x - im * (ST)wk.y;
                    Xi = re * (ST)wk.y + im * (ST)wk.x;
                } else {
                    // FP32 state: the rotation factor as a float-float pair, so its
                    // rounding does not compound into a phase drift over the chunk
                    Xr = fmaf(re, ch, fmaf(-im, sh, fmaf(re, cl, -im * sl)));
                    Xi = fmaf(re, sh, fmaf(im, ch, fmaf(re, sl, im * cl)));
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
    (void)B;
    return sizeof(double2) * a_max;
}

cudaError_t launch_moment_table(const PnView &v, int64_t total_windows, cudaStream_t st) {
    if (total_windows <= 0) return cudaSuccess;
    k_moment_table<<<grid_for(total_windows, 256), 256, 0, st>>>(v, total_windows);
    return cudaGetLastError();
}

cudaError_t launch_features(const PnView &v, const int32_t *blk_anchor, const int32_t *blk_chunk0,
                            int32_t nblocks, int a_max, cudaStream_t st) {
    if (nblocks <= 0) return cudaSuccess;
    size_t sm = features_smem(a_max, v.B);
    cudaError_t e;
    if (v.precision == 0) {
        e = pn_allow_smem(k_features<double>, sm);
        if (e != cudaSuccess) return e;
        k_features<double><<<nblocks, FT_THREADS, sm, st>>>(v, blk_anchor, blk_chunk0);
    } else {
        e = pn_allow_smem(k_features<float>, sm);
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
                               const PnQRange *rng, int32_t nrng, uint32_t **keys_out) {
    if (keys_out) *keys_out = nullptr;
    if (total <= 0) return cudaSuccess;
    uint32_t *keys = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&keys, sizeof(uint32_t) * total, st);
    if (e != cudaSuccess) return e;
    k_query_keys<<<grid_for(total, 256), 256, 0, st>>>(v, total, keys, rng, nrng);
    e = cudaGetLastError();
    int bits = 1;
    while (bits < 32 && ((int64_t)1 << bits) <= total_buckets) ++bits;
    if (e == cudaSuccess) e = radix_sort_pairs(keys, v.qorder, total, bits, st);
    if (e == cudaSuccess && keys_out) *keys_out = keys;
    else cudaFreeAsync(keys, st);
    return e;
}

}  // namespace pn
