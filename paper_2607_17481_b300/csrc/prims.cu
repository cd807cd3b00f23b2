// Segmented scans and a stable LSD radix sort, written for sm_103a.
//
// Scans: three launches (tile reduce, single-block scan of tile carries,
// tile scan with carry-in).  The association order is fixed by the tile
// layout, so floating-point results are identical from run to run.
//
// Radix sort: 8-bit digits, tiles of 4096 items (8 warps x 512).  Per tile a
// digit histogram; an exclusive scan over (digit, tile) gives each tile's
// output base per digit; in the scatter pass every warp walks its 512 items
// in order and ranks equal digits with __match_any_sync, so the sort is
// stable.
#include "prims.cuh"

namespace pn {
namespace {

constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;   // 2048

struct AddU32 {
    __device__ static uint32_t zero() { return 0u; }
    __device__ static uint32_t add(uint32_t a, uint32_t b) { return a + b; }
};
struct AddD2 {
    __device__ static double2 zero() { return make_double2(0.0, 0.0); }
    __device__ static double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
};

// (flag, value) pairs under the segmented-sum operator:
// (f1, v1) (+) (f2, v2) = (f1 | f2, f2 ? v2 : v1 + v2).
template <class Op, class T>
struct Seg {
    T v;
    int f;
};

template <class Op, class T>
__device__ __forceinline__ Seg<Op, T> seg_op(Seg<Op, T> a, Seg<Op, T> b) {
    Seg<Op, T> r;
    r.f = a.f | b.f;
    r.v = b.f ? b.v : Op::add(a.v, b.v);
    return r;
}

template <class T>
__device__ __forceinline__ T shfl_up(T v, int d);
template <>
__device__ __forceinline__ uint32_t shfl_up<uint32_t>(uint32_t v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
template <>
__device__ __forceinline__ double2 shfl_up<double2>(double2 v, int d) {
    return make_double2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}

// Inclusive block scan of one Seg per thread.  Returns the inclusive value;
// *block_total receives the block aggregate (valid in every thread).
template <class Op, class T>
__device__ Seg<Op, T> block_scan(Seg<Op, T> x, Seg<Op, T> *block_total) {
    __shared__ T s_v[SC_THREADS / 32];
    __shared__ int s_f[SC_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Seg<Op, T> y;
        y.v = shfl_up<T>(x.v, d);
        y.f = __shfl_up_sync(0xffffffffu, x.f, d);
        if (lane >= d) x = seg_op<Op, T>(y, x);
    }
    if (lane == 31) {
        s_v[warp] = x.v;
        s_f[warp] = x.f;
    }
    __syncthreads();
    Seg<Op, T> pre;
    pre.v = Op::zero();
    pre.f = 0;
    for (int w = 0; w < warp; ++w) {
        Seg<Op, T> y;
        y.v = s_v[w];
        y.f = s_f[w];
        pre = seg_op<Op, T>(pre, y);
    }
    Seg<Op, T> tot;
    tot.v = Op::zero();
    tot.f = 0;
    for (int w = 0; w < SC_THREADS / 32; ++w) {
        Seg<Op, T> y;
        y.v = s_v[w];
        y.f = s_f[w];
        tot = seg_op<Op, T>(tot, y);
    }
    *block_total = tot;
    __syncthreads();
    return seg_op<Op, T>(pre, x);
}

template <class Op, class T>
__device__ __forceinline__ Seg<Op, T> load_seg(const T *in, const uint8_t *head, int64_t i, int64_t n) {
    Seg<Op, T> s;
    if (i < n) {
        s.v = in[i];
        s.f = head ? (int)head[i] : 0;
    } else {
        s.v = Op::zero();
        s.f = 0;
    }
    return s;
}

// Pass 1: aggregate of each tile.
template <class Op, class T>
__global__ void k_seg_reduce(const T *in, const uint8_t *head, int64_t n, T *tv, int *tf) {
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    Seg<Op, T> acc;
    acc.v = Op::zero();
    acc.f = 0;
    for (int t = 0; t < SC_ITEMS; ++t) acc = seg_op<Op, T>(acc, load_seg<Op, T>(in, head, base + t, n));
    Seg<Op, T> tot;
    block_scan<Op, T>(acc, &tot);
    if (threadIdx.x == 0) {
        tv[blockIdx.x] = tot.v;
        tf[blockIdx.x] = tot.f;
    }
}

// Pass 2: exclusive scan of the tile aggregates by one block (in place).
template <class Op, class T>
__global__ void k_seg_carries(T *tv, int *tf, int64_t ntiles) {
    __shared__ T s_carry;
    __shared__ int s_cf;
    if (threadIdx.x == 0) {
        s_carry = Op::zero();
        s_cf = 0;
    }
    __syncthreads();
    for (int64_t b0 = 0; b0 < ntiles; b0 += SC_THREADS) {
        int64_t i = b0 + threadIdx.x;
        Seg<Op, T> x;
        if (i < ntiles) {
            x.v = tv[i];
            x.f = tf[i];
        } else {
            x.v = Op::zero();
            x.f = 0;
        }
        Seg<Op, T> tot;
        Seg<Op, T> inc = block_scan<Op, T>(x, &tot);
        Seg<Op, T> carry;
        carry.v = s_carry;
        carry.f = s_cf;
        // exclusive value for tile i = carry (+) (inclusive - own)
        Seg<Op, T> ex;
        {
            // recompute exclusive by shifting the inclusive result one lane up the block
            __shared__ T s_inc_v[SC_THREADS];
            __shared__ int s_inc_f[SC_THREADS];
            s_inc_v[threadIdx.x] = inc.v;
            s_inc_f[threadIdx.x] = inc.f;
            __syncthreads();
            Seg<Op, T> prev;
            if (threadIdx.x == 0) {
                prev.v = Op::zero();
                prev.f = 0;
            } else {
                prev.v = s_inc_v[threadIdx.x - 1];
                prev.f = s_inc_f[threadIdx.x - 1];
            }
            ex = seg_op<Op, T>(carry, prev);
            __syncthreads();
        }
        if (i < ntiles) {
            tv[i] = ex.v;
            tf[i] = ex.f;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Seg<Op, T> nc = seg_op<Op, T>(carry, tot);
            s_carry = nc.v;
            s_cf = nc.f;
        }
        __syncthreads();
    }
}

// Pass 3: inclusive scan of each tile with its carry-in.
template <class Op, class T>
__global__ void k_seg_final(const T *in, const uint8_t *head, T *out, int64_t n, const T *tv) {
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    Seg<Op, T> items[SC_ITEMS];
    Seg<Op, T> acc;
    acc.v = Op::zero();
    acc.f = 0;
#pragma unroll
    for (int t = 0; t < SC_ITEMS; ++t) {
        items[t] = load_seg<Op, T>(in, head, base + t, n);
        acc = seg_op<Op, T>(acc, items[t]);
    }
    Seg<Op, T> tot;
    Seg<Op, T> inc = block_scan<Op, T>(acc, &tot);
    // exclusive prefix of this thread inside the tile = inc minus own aggregate:
    // rebuild it by scanning again with the thread's items removed.
    __shared__ T s_v[SC_THREADS];
    __shared__ int s_f[SC_THREADS];
    s_v[threadIdx.x] = inc.v;
    s_f[threadIdx.x] = inc.f;
    __syncthreads();
    Seg<Op, T> run;
    run.v = tv[blockIdx.x];
    run.f = 0;
    if (threadIdx.x > 0) {
        Seg<Op, T> p;
        p.v = s_v[threadIdx.x - 1];
        p.f = s_f[threadIdx.x - 1];
        run = seg_op<Op, T>(run, p);
    }
#pragma unroll
    for (int t = 0; t < SC_ITEMS; ++t) {
        run = seg_op<Op, T>(run, items[t]);
        if (base + t < n) out[base + t] = run.v;
    }
}

template <class Op, class T>
cudaError_t seg_scan_impl(const T *in, const uint8_t *head, T *out, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int64_t ntiles = (n + SC_TILE - 1) / SC_TILE;
    T *tv = nullptr;
    int *tf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&tv, sizeof(T) * ntiles, st);
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync((void **)&tf, sizeof(int) * ntiles, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(tv, st);
        return e;
    }
    k_seg_reduce<Op, T><<<(unsigned)ntiles, SC_THREADS, 0, st>>>(in, head, n, tv, tf);
    k_seg_carries<Op, T><<<1, SC_THREADS, 0, st>>>(tv, tf, ntiles);
    k_seg_final<Op, T><<<(unsigned)ntiles, SC_THREADS, 0, st>>>(in, head, out, n, tv);
    e = cudaGetLastError();
    cudaFreeAsync(tv, st);
    cudaFreeAsync(tf, st);
    return e;
}

// ---------------------------------------------------------------------------
// Radix sort
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ROUNDS = 16;                        // 16 x 32 = 512 items per warp
constexpr int RS_TILE = RS_WARPS * RS_ROUNDS * 32;   // 4096 items per block

__global__ void k_rs_upsweep(const uint32_t *keys, int64_t n, int shift, uint32_t *hist, int64_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_ROUNDS * 32;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t p = wbase + r * 32 + lane;
        bool ok = p < n;
        uint32_t dg = ok ? ((keys[p] >> shift) & 255u) : (256u + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (ok && lane == __ffs(peers) - 1) atomicAdd(&h[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void k_rs_downsweep(const uint32_t *kin, const uint32_t *vin, uint32_t *kout, uint32_t *vout,
                               int64_t n, int shift, const uint32_t *hist, int64_t ntiles) {
    __shared__ uint32_t wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < RS_WARPS * 256; t += RS_THREADS) (&wcnt[0][0])[t] = 0;
    __syncthreads();
    const int64_t wbase = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * RS_ROUNDS * 32;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t p = wbase + r * 32 + lane;
        bool ok = p < n;
        uint32_t dg = ok ? ((kin[p] >> shift) & 255u) : (256u + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][dg] += (uint32_t)__popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {
        const int dg = threadIdx.x;
        uint32_t run = hist[(int64_t)dg * ntiles + blockIdx.x];
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wcnt[w][dg];
            wcnt[w][dg] = run;
            run += c;
        }
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    for (int r = 0; r < RS_ROUNDS; ++r) {
        int64_t p = wbase + r * 32 + lane;
        bool ok = p < n;
        uint32_t k = ok ? kin[p] : 0u;
        uint32_t dg = ok ? ((k >> shift) & 255u) : (256u + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        uint32_t base = ok ? wcnt[warp][dg] : 0u;
        __syncwarp();
        if (ok) {
            uint32_t pos = base + (uint32_t)__popc(peers & lt);
            kout[pos] = k;
            vout[pos] = vin[p];
            if (lane == __ffs(peers) - 1) wcnt[warp][dg] = base + (uint32_t)__popc(peers);
        }
        __syncwarp();
    }
}

}  // namespace

cudaError_t seg_scan_u32(const uint32_t *in, const uint8_t *head, uint32_t *out, int64_t n, cudaStream_t st) {
    return seg_scan_impl<AddU32, uint32_t>(in, head, out, n, st);
}

cudaError_t seg_scan_d2(const double2 *in, const uint8_t *head, double2 *out, int64_t n, cudaStream_t st) {
    return seg_scan_impl<AddD2, double2>(in, head, out, n, st);
}

namespace {
__global__ void k_shift_excl(const uint32_t *inc, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        uint32_t v = inc[i];
        out[i] = v - in[i];
        if (i == n - 1 && total) *total = v;
    }
}
}  // namespace

cudaError_t excl_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, uint32_t *total, cudaStream_t st) {
    if (n <= 0) {
        if (total) return cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
        return cudaSuccess;
    }
    uint32_t *inc = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&inc, sizeof(uint32_t) * n, st);
    if (e != cudaSuccess) return e;
    e = seg_scan_u32(in, nullptr, inc, n, st);
    if (e == cudaSuccess) {
        k_shift_excl<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(inc, in, out, n, total);
        e = cudaGetLastError();
    }
    cudaFreeAsync(inc, st);
    return e;
}

cudaError_t radix_sort_pairs(uint32_t *keys, uint32_t *vals, int64_t n, int bits, cudaStream_t st) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    int64_t ntiles = (n + RS_TILE - 1) / RS_TILE;
    uint32_t *k2 = nullptr, *v2 = nullptr, *hist = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&k2, sizeof(uint32_t) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&v2, sizeof(uint32_t) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync((void **)&hist, sizeof(uint32_t) * 256 * ntiles, st);
    uint32_t *ka = keys, *va = vals, *kb = k2, *vb = v2;
    int passes = (bits + 7) / 8;
    for (int p = 0; p < passes && e == cudaSuccess; ++p) {
        k_rs_upsweep<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(ka, n, 8 * p, hist, ntiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = excl_scan_u32(hist, hist, 256 * ntiles, nullptr, st);
        if (e == cudaSuccess) {
            k_rs_downsweep<<<(unsigned)ntiles, RS_THREADS, 0, st>>>(ka, va, kb, vb, n, 8 * p, hist, ntiles);
            e = cudaGetLastError();
        }
        uint32_t *t = ka; ka = kb; kb = t;
        t = va; va = vb; vb = t;
    }
    if (e == cudaSuccess && ka != keys) {
        e = cudaMemcpyAsync(keys, ka, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
    }
    if (k2) cudaFreeAsync(k2, st);
    if (v2) cudaFreeAsync(v2, st);
    if (hist) cudaFreeAsync(hist, st);
    return e;
}

}  // namespace pn
