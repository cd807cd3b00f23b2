// Spectral-width calibration (Sec. 3.2, "Spectral width selection").
//
// The width K is fixed before insertion: the smallest K whose retained bins
// hold a fraction eta of the normalised spectral energy of sampled windows,
// E[(2/m^2) sum_{k<=K'} |X^_k|^2] >= eta, and whose expected accidental
// signature collisions stay within twice the verification budget,
// n E[(1 - theta_K/pi)^B] <= 2 gamma alpha.  This file computes the two
// sample means for every K = 2..K_max on the device:
//   k_cal_features  one warp per sampled window: FP64 moments, max/min, and
//                   the direct DFT bins 1..K_max-1 of the z-normalised window;
//   k_cal_pairs     one block per (length, window a): every later window b of
//                   the same length, near-duplicates (full-width bound below
//                   0.1 sqrt(2m)) skipped, the angle at each width from
//                   running sums over the bins, block sums in a fixed tree;
//   k_cal_reduce    one block: the per-window energies and the per-row pair
//                   sums, in a fixed order (run-to-run identical results).
#include "kernels.cuh"

namespace pn {
namespace {

constexpr int CAL_NK = PN_MAXK - 1;            // widths K = 2..K_max
constexpr int CAL_BINS = PN_MAXK - 1;          // bins 1..K_max-1
constexpr int CAL_THREADS = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_min_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__global__ void k_cal_features(const double *x, const PnCalWin *win, int nwin, double *F, int *valid,
                               double *energy) {
    const int lane = threadIdx.x & 31;
    const int wi = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (wi >= nwin) return;
    const PnCalWin w = win[wi];
    const int m = w.m;
    const double *xs = x + w.start;
    double s = 0.0, mx = -1.0 / 0.0, mn = 1.0 / 0.0;
    for (int r = lane; r < m; r += 32) {
        const double t = xs[r];
        s += t;
        mx = fmax(mx, t);
        mn = fmin(mn, t);
    }
    s = warp_sum_d(s);
    mx = warp_max_d(mx);
    mn = warp_min_d(mn);
    const double mu = s / m;
    double q = 0.0;
    for (int r = lane; r < m; r += 32) {
        const double d = xs[r] - mu;
        q = fma(d, d, q);
    }
    q = warp_sum_d(q);
    const double sigma = sqrt(q / m);
    const bool ok = mx != mn && sigma > 0.0;
    const int kp = pn_kprime(m, PN_MAXK);
    double re[CAL_BINS], im[CAL_BINS];
#pragma unroll
    for (int k = 0; k < CAL_BINS; ++k) {
        re[k] = 0.0;
        im[k] = 0.0;
    }
    if (ok) {
        for (int r = lane; r < m; r += 32) {
            const double z = (xs[r] - mu) / sigma;
#pragma unroll
            for (int k = 0; k < CAL_BINS; ++k) {
                if (k < kp) {
                    const int ph = (int)(((int64_t)(k + 1) * r) % m);
                    double sn, cs;
                    sincospi(2.0 * (double)ph / (double)m, &sn, &cs);
                    re[k] = fma(z, cs, re[k]);
                    im[k] = fma(-z, sn, im[k]);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < CAL_BINS; ++k) {
        re[k] = warp_sum_d(re[k]);
        im[k] = warp_sum_d(im[k]);
    }
    if (lane == 0) {
        double *f = F + (int64_t)wi * 2 * CAL_BINS;
        const double scale = 2.0 / ((double)m * (double)m);
        int t = 0;
        for (int k = 0; k < CAL_BINS; ++k) {
            f[2 * k] = re[k];
            f[2 * k + 1] = im[k];
        }
        // energy retained at every width K = 2..K_max (bins 1..K'(m, K))
        for (int K = 2; K <= PN_MAXK; ++K, ++t) {
            const int kk = pn_kprime(m, K);
            double acc = 0.0;
            for (int k = 0; k < kk; ++k) acc += re[k] * re[k] + im[k] * im[k];
            energy[(int64_t)wi * CAL_NK + t] = ok ? scale * acc : 0.0;
        }
        valid[wi] = ok ? 1 : 0;
    }
}

// Block (g, a): pairs (a, b), a < b, of the windows of length group g.
__global__ void __launch_bounds__(CAL_THREADS) k_cal_pairs(const double *F, const int *valid, const PnCalWin *win,
                                                           const int *g_off, const int *g_cnt, const int *row_g,
                                                           const int *row_a, int B, double *row_sum,
                                                           unsigned long long *row_cnt) {
    __shared__ double s_sum[CAL_THREADS];
    __shared__ unsigned long long s_cnt[CAL_THREADS];
    const int g = row_g[blockIdx.x], a = row_a[blockIdx.x];
    const int off = g_off[g], S = g_cnt[g];
    const int ia = off + a;
    const int m = win[ia].m;
    const double *fa = F + (int64_t)ia * 2 * CAL_BINS;
    const double dup = 0.1 * sqrt(2.0 * (double)m);
    double term[CAL_NK];
#pragma unroll
    for (int t = 0; t < CAL_NK; ++t) term[t] = 0.0;
    unsigned long long cnt = 0;
    if (valid[ia]) {
        for (int b = a + 1 + (int)threadIdx.x; b < S; b += blockDim.x) {
            const int ib = off + b;
            if (!valid[ib]) continue;
            const double *fb = F + (int64_t)ib * 2 * CAL_BINS;
            double d2 = 0.0;
            for (int t = 0; t < 2 * CAL_BINS; ++t) {
                const double d = fa[t] - fb[t];
                d2 += d * d;
            }
            if (sqrt((2.0 / m) * d2) < dup) continue;          // near-duplicate pair
            ++cnt;
            double dot = 0.0, na = 0.0, nb = 0.0;
            int kdone = 0;
#pragma unroll
            for (int t = 0; t < CAL_NK; ++t) {
                const int kk = pn_kprime(m, t + 2);
                for (int k = kdone; k < kk; ++k) {
                    dot += fa[2 * k] * fb[2 * k] + fa[2 * k + 1] * fb[2 * k + 1];
                    na += fa[2 * k] * fa[2 * k] + fa[2 * k + 1] * fa[2 * k + 1];
                    nb += fb[2 * k] * fb[2 * k] + fb[2 * k + 1] * fb[2 * k + 1];
                }
                kdone = kk > kdone ? kk : kdone;
                double c = (na > 0.0 && nb > 0.0) ? dot / (sqrt(na) * sqrt(nb)) : 0.0;
                c = fmin(1.0, fmax(-1.0, c));
                const double th = acos(c);
                term[t] += pow(1.0 - th / 3.141592653589793, (double)B);
            }
        }
    }
    // fixed-tree block sums, one width at a time
    for (int t = 0; t <= CAL_NK; ++t) {
        if (t < CAL_NK) s_sum[threadIdx.x] = term[t];
        else s_cnt[threadIdx.x] = cnt;
        __syncthreads();
        for (int h = CAL_THREADS / 2; h > 0; h >>= 1) {
            if ((int)threadIdx.x < h) {
                if (t < CAL_NK) s_sum[threadIdx.x] += s_sum[threadIdx.x + h];
                else s_cnt[threadIdx.x] += s_cnt[threadIdx.x + h];
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (t < CAL_NK) row_sum[(int64_t)blockIdx.x * CAL_NK + t] = s_sum[0];
            else row_cnt[blockIdx.x] = s_cnt[0];
        }
        __syncthreads();
    }
}

// Means over the valid windows (energy) and over the counted pairs (collision).
__global__ void k_cal_reduce(const double *energy, const int *valid, int nwin, const double *row_sum,
                             const unsigned long long *row_cnt, int nrows, double *out) {
    const int t = threadIdx.x;
    if (t < CAL_NK) {
        double e = 0.0;
        long long nv = 0;
        for (int w = 0; w < nwin; ++w) {
            if (!valid[w]) continue;
            e += energy[(int64_t)w * CAL_NK + t];
            ++nv;
        }
        double c = 0.0;
        unsigned long long np = 0;
        for (int r = 0; r < nrows; ++r) {
            c += row_sum[(int64_t)r * CAL_NK + t];
            np += row_cnt[r];
        }
        out[t] = nv ? e / (double)nv : 0.0;
        out[CAL_NK + t] = np ? c / (double)np : 0.0;
        if (t == 0) out[2 * CAL_NK] = (double)np;
    }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

cudaError_t launch_calibration(const double *x, const PnCalWin *win, int nwin, const int *g_off, const int *g_cnt,
                               const int *row_g, const int *row_a, int nrows, int B, double *out, cudaStream_t st) {
    double *F = nullptr, *energy = nullptr, *row_sum = nullptr;
    int *valid = nullptr;
    unsigned long long *row_cnt = nullptr;
    const int nw = nwin > 0 ? nwin : 1, nr = nrows > 0 ? nrows : 1;
    cudaError_t e = cudaMallocAsync((void **)&F, sizeof(double) * 2 * CAL_BINS * nw, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&energy, sizeof(double) * CAL_NK * nw, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&valid, sizeof(int) * nw, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&row_sum, sizeof(double) * CAL_NK * nr, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&row_cnt, sizeof(unsigned long long) * nr, st);
    if (e == cudaSuccess && nwin > 0) {
        k_cal_features<<<blocks_for((int64_t)nwin * 32, 128), 128, 0, st>>>(x, win, nwin, F, valid, energy);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && nrows > 0) {
        k_cal_pairs<<<nrows, CAL_THREADS, 0, st>>>(F, valid, win, g_off, g_cnt, row_g, row_a, B, row_sum, row_cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_cal_reduce<<<1, 32, 0, st>>>(energy, valid, nwin, row_sum, row_cnt, nrows, out);
        e = cudaGetLastError();
    }
    if (F) cudaFreeAsync(F, st);
    if (energy) cudaFreeAsync(energy, st);
    if (valid) cudaFreeAsync(valid, st);
    if (row_sum) cudaFreeAsync(row_sum, st);
    if (row_cnt) cudaFreeAsync(row_cnt, st);
    return e;
}

}  // namespace pn
