// Exact row refinement of the top cells (emit stage, after local completion).
//
// The streaming search, the hot-class sieve and local completion evaluate
// the pairs their rules admit (Algorithms 1-2); a cell whose nearest valid
// neighbour no rule brought up keeps a larger value, and if that cell is
// reported, its motif carries a partner that is not its nearest neighbour.
// The paper's emit never rescans a length row.  On the GPU one row costs
// n m multiply-adds (a few tens of microseconds at n = 5M), so the cells of
// the current top list are refined by scanning every valid partner j
// (|i - j| >= excl, j non-constant) at the cell's own length with the
// arithmetic of the in-stream distances, and the smallest packed key lowers
// the cell by atomicMin.  The host reselects and refines new cells until the
// list no longer changes (capi.cu); every reported cell then holds its exact
// nearest neighbour up to in-stream rounding, and the FP64 verification
// gives its distance.  Only the target cell is written (the partner's own
// cell is left to the other rules).
//
// Window moments come from the FP64 prefix sums at the target's length with
// the moment table's arithmetic (mu, sigma^2 = Q/m - mu^2; the mixed form
// takes 1/sigma in FP32), so any length works, anchored or not.
#include <algorithm>

#include "emit.cuh"
#include "zops.cuh"

namespace pn {
namespace {

constexpr int RF_THREADS = 256;

template <class Z>
__device__ __forceinline__ typename Z::M ref_moments(const PnView &v, const PnSeries &S, int s, int64_t j, int m);

template <>
__device__ __forceinline__ double2 ref_moments<ZPlain>(const PnView &v, const PnSeries &S, int s, int64_t j, int m) {
    const double2 *sqp = v.sq + S.x_off + s;
    const double2 pa = sqp[j], pb = sqp[j + m];
    const double inv_m = 1.0 / (double)m;
    const double ms = (pb.x - pa.x) * inv_m;
    const double var = (pb.y - pa.y) * inv_m - ms * ms;
    const double mu = ms + v.shift[s];
    const bool ok = v.runlen[S.x_off + j] < m && var > 0.0;
    const double inv = ok ? 1.0 / sqrt(var) : 0.0;
    return make_double2(inv, -mu * inv);
}

template <class Z>
__device__ __forceinline__ float2 ref_moments_mixed(const PnView &v, const PnSeries &S, int s, int64_t j, int m) {
    const double2 *sqp = v.sq + S.x_off + s;
    const double2 pa = sqp[j], pb = sqp[j + m];
    const double inv_m = 1.0 / (double)m;
    const double ms = (pb.x - pa.x) * inv_m;
    const double var = (pb.y - pa.y) * inv_m - ms * ms;
    const double mu = ms + v.shift[s];
    const bool ok = v.runlen[S.x_off + j] < m && var > 0.0;
    const float invf = ok ? rsqrtf((float)var) : 0.0f;
    return make_float2(invf, (float)(-mu * (double)invf));
}

template <>
__device__ __forceinline__ float2 ref_moments<ZMix2>(const PnView &v, const PnSeries &S, int s, int64_t j, int m) {
    return ref_moments_mixed<ZMix2>(v, S, s, j, m);
}

template <>
__device__ __forceinline__ float2 ref_moments<ZMix1>(const PnView &v, const PnSeries &S, int s, int64_t j, int m) {
    return ref_moments_mixed<ZMix1>(v, S, s, j, m);
}

// A persistent kernel: work item w is part (w mod parts) of target
// (w / parts); a part scans partners j = part * RF_THREADS + tid + k parts
// RF_THREADS.  The target count may live on the device (device-driven
// passes), so the grid is fixed and the items are counted there.
template <class Z>
__global__ void __launch_bounds__(RF_THREADS) k_refine(PnView v, const PnSeed *tg, int32_t ntg_max,
                                                       const int32_t *ntg_dev, int32_t parts, int *improved) {
    using ZT = typename Z::T;
    if (pn_gated(v)) return;
    extern __shared__ __align__(16) unsigned char rsm[];
    ZT *zq = reinterpret_cast<ZT *>(rsm);
    __shared__ unsigned long long wbest[RF_THREADS / 32];
    const int32_t ntg = ntg_dev ? min(*ntg_dev, ntg_max) : ntg_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long n_ex = 0;
    for (int64_t w = blockIdx.x; w < (int64_t)ntg * parts; w += gridDim.x) {
        const PnSeed t = tg[w / parts];
        const int part = (int)(w % parts);
        const int s = t.series, m = t.m;
        const PnSeries &S = v.series[s];
        const int64_t i = t.i, last = S.n - m;
        const auto mq = ref_moments<Z>(v, S, s, i, m);
        if (Z::degenerate(mq)) continue;                     // block-uniform
        __syncthreads();                                     // the previous item's window is no longer read
        const auto *xi = Z::samples(v, S.x_off + i);
        for (int r = threadIdx.x; r < m; r += RF_THREADS) zq[r] = Z::z(mq, xi[r]);
        __syncthreads();
        unsigned long long best = PN_EMPTY_KEY;
        for (int64_t j = (int64_t)part * RF_THREADS + threadIdx.x; j <= last; j += (int64_t)parts * RF_THREADS) {
            if (j - i < S.excl && i - j < S.excl) continue;
            const auto mj = ref_moments<Z>(v, S, s, j, m);
            if (Z::degenerate(mj)) continue;
            const auto *xj = Z::samples(v, S.x_off + j);
            ZT acc = 0;
#pragma unroll 4
            for (int r = 0; r < m; ++r) {
                const ZT d = zq[r] - Z::z(mj, xj[r]);
                acc = fma(d, d, acc);
            }
            const unsigned long long key = Z::pack(Z::root(acc), (uint32_t)j);
            best = key < best ? key : best;
            n_ex += 1;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other < best ? other : best;
        }
        if (lane == 0) wbest[warp] = best;
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long b = wbest[0];
            for (int q = 1; q < RF_THREADS / 32; ++q) b = wbest[q] < b ? wbest[q] : b;
            if (b != PN_EMPTY_KEY) {
                unsigned long long *row = v.prof + S.row_off + (int64_t)(m - S.m_min) * S.ld;
                if (atomicMin(&row[i], b) > b) atomicExch(improved, 1);
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_ex += __shfl_xor_sync(0xffffffffu, n_ex, o);
    if (lane == 0 && v.stats && n_ex) atomicAdd(&v.stats[PN_ST_EXACT_REFINE], n_ex);
}

template <class Z>
cudaError_t refine_t(const PnView &v, const PnSeed *tg, int32_t ntg, const int32_t *ntg_dev, int64_t max_windows,
                     int m_max, int *improved, int blocks_per_target, cudaStream_t st) {
    const size_t sm = sizeof(typename Z::T) * (size_t)m_max;
    cudaError_t e = pn_allow_smem(k_refine<Z>, sm);
    if (e != cudaSuccess) return e;
    int64_t parts = (max_windows + RF_THREADS - 1) / RF_THREADS;
    if (parts > blocks_per_target) parts = blocks_per_target;
    if (parts < 1) parts = 1;
    // enough resident blocks for every SM; the items beyond are looped over
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t items = (int64_t)ntg * parts;
    const int64_t grid = std::min<int64_t>(items, (int64_t)sms * 8);
    k_refine<Z><<<(unsigned)std::max<int64_t>(1, grid), RF_THREADS, sm, st>>>(v, tg, ntg, ntg_dev, (int32_t)parts,
                                                                          improved);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refine(const PnView &v, const PnSeed *tg, int32_t ntg, const int32_t *ntg_dev, int64_t max_windows,
                          int m_max, int *improved, int blocks_per_target, cudaStream_t st) {
    if (ntg <= 0 || max_windows <= 0) return cudaSuccess;
    if (v.precision == 0)
        return refine_t<ZPlain>(v, tg, ntg, ntg_dev, max_windows, m_max, improved, blocks_per_target, st);
    if (v.x1) return refine_t<ZMix1>(v, tg, ntg, ntg_dev, max_windows, m_max, improved, blocks_per_target, st);
    return refine_t<ZMix2>(v, tg, ntg, ntg_dev, max_windows, m_max, improved, blocks_per_target, st);
}

}  // namespace pn
