// Top-k selection of one profile row with no device allocation.
//
// The regular selection (emit.cu) takes its histogram, candidate pool and
// counters from the stream-ordered allocator.  Callers that cannot allocate
// device memory -- code running inside another framework's memory pool or
// under a memory budget that forbids new allocations, or an embedded caller
// that must not touch the allocator from its context -- use this variant.
// All of its scratch lives in one file-scope __device__ array of fixed size
// (NaScratch below, about 145 KB), which every GPU that loads this library
// holds until the process exits.
//
// The steps are those of the regular selection (Sec. 2 top-k rule, Sec. 3.6
// zero-snap), for a single length: a two-level radix select of the
// k (m + 1) smallest keys (plus one bin of slack), FP64 two-pass distances of
// the pooled cells evaluated in (min, max) order, a bitonic sort by (d, i)
// and a greedy scan under the m/2 rule.
#include <mutex>

#include "common.cuh"
#include "panache.h"

namespace {

constexpr int NA_BINS = 4096;
constexpr int NA_POOL_MAX = 8192;       // pooled cells; k (m + 1) + slack must fit
constexpr int NA_MAX_DEVICES = 64;
// The largest k (m + 1) accepted: the pool must hold it plus the regular
// selection's slack (a quarter more and one bin's worth, 256).
static_assert(PANACHE_NOALLOC_NEED_MAX + PANACHE_NOALLOC_NEED_MAX / 4 + 256 <= NA_POOL_MAX,
              "the pool must hold the largest accepted request with its slack");

struct NaEntry {
    double d;
    uint32_t i;
    uint32_t j;
};

struct NaScratch {
    uint32_t hist[NA_BINS];
    uint32_t b1, b2, carry, pool_cnt;
    int overflow;
    int _pad[3];
    NaEntry pool[NA_POOL_MAX];
};

// The scratch.  Host code must not pass this symbol to a kernel: on the host
// its name is a stand-in, not a device address.  The address comes from
// cudaGetSymbolAddress, once per device, with that device current.
static __device__ __align__(256) NaScratch g_na_scratch;

__device__ __forceinline__ uint32_t na_bits(unsigned long long key, double eps0, int level) {
    const double d = pn_key_dist(key);
    const unsigned long long b = d < eps0 ? 0ull : (key & ~PN_IDX_MASK);
    return level == 0 ? (uint32_t)(b >> 51) & 0xFFFu : (uint32_t)(b >> 39) & 0xFFFu;
}

__global__ void k_na_clear(NaScratch *s) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < NA_BINS; t += gridDim.x * blockDim.x) s->hist[t] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        s->b1 = s->b2 = s->carry = s->pool_cnt = 0;
        s->overflow = 0;
    }
}

__global__ void k_na_hist(const unsigned long long *keys, int64_t n, double eps0, int level, NaScratch *s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long key = t < n ? keys[t] : PN_EMPTY_KEY;
    bool ok = key != PN_EMPTY_KEY;
    if (ok && level == 1) ok = na_bits(key, eps0, 0) == s->b1;
    const uint32_t bin = ok ? na_bits(key, eps0, level) : (0x1000u + (threadIdx.x & 31));
    const unsigned peers = __match_any_sync(0xffffffffu, bin);
    if (ok && (threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&s->hist[bin], (uint32_t)__popc(peers));
}

// First bin whose cumulative count reaches `need`; then clears the histogram.
__global__ void k_na_pick(NaScratch *s, uint32_t need, int level) {
    if (threadIdx.x == 0) {
        uint32_t run = level == 0 ? 0u : s->carry, b = NA_BINS - 1;
        for (int t = 0; t < NA_BINS; ++t) {
            const uint32_t c = s->hist[t];
            if (run + c >= need) {
                b = t;
                break;
            }
            run += c;
        }
        if (level == 0) {
            s->b1 = b;
            s->carry = run;
        } else {
            s->b2 = b;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < NA_BINS; t += blockDim.x) s->hist[t] = 0;
}

__global__ void k_na_pool(const unsigned long long *keys, int64_t n, int m, double eps0, NaScratch *s) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n - m) return;                       // cells past the last window hold no motif
    const unsigned long long key = keys[t];
    if (key == PN_EMPTY_KEY || (int64_t)pn_key_idx(key) > n - m) return;
    const uint32_t h = (na_bits(key, eps0, 0) << 12) | na_bits(key, eps0, 1);
    if (h > ((s->b1 << 12) | s->b2) + 1u) return;
    const uint32_t slot = atomicAdd(&s->pool_cnt, 1u);
    if (slot >= (uint32_t)NA_POOL_MAX) {
        s->overflow = 1;
        return;
    }
    NaEntry e;
    e.d = pn_key_dist(key);
    e.i = (uint32_t)t;
    e.j = pn_key_idx(key);
    s->pool[slot] = e;
}

// FP64 two-pass distance of every pooled cell, pair taken in (min, max) order.
__global__ void k_na_verify(const double *x, int m, double eps0, NaScratch *s) {
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    const int cnt = (int)min(s->pool_cnt, (uint32_t)NA_POOL_MAX);
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < cnt; e += nwarp) {
        NaEntry &pe = s->pool[e];
        const int64_t i = pe.i < pe.j ? pe.i : pe.j, j = pe.i < pe.j ? pe.j : pe.i;
        const double *xi = x + i, *xj = x + j;
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

__device__ __forceinline__ bool na_less(const NaEntry &a, const NaEntry &b) {
    return a.d < b.d || (a.d == b.d && a.i < b.i);
}

// One block: bitonic sort of the pool in shared memory, greedy m/2 scan by warp 0.
__global__ void k_na_greedy(NaScratch *s, int m, int k, panache_motif *out, int32_t *out_count) {
    extern __shared__ __align__(16) unsigned char smem[];
    NaEntry *e = reinterpret_cast<NaEntry *>(smem);
    int64_t *acc_i = reinterpret_cast<int64_t *>(e + NA_POOL_MAX);
    if (s->overflow) {
        if (threadIdx.x == 0) *out_count = PANACHE_EPOOL;
        return;
    }
    const int cnt = (int)min(s->pool_cnt, (uint32_t)NA_POOL_MAX);
    int np2 = 1;
    while (np2 < cnt) np2 <<= 1;
    for (int t = threadIdx.x; t < np2; t += blockDim.x) {
        if (t < cnt) {
            e[t] = s->pool[t];
        } else {
            e[t].d = __longlong_as_double(0x7ff0000000000000ll);
            e[t].i = 0xFFFFFFFFu;
            e[t].j = 0;
        }
    }
    __syncthreads();
    for (int kk = 2; kk <= np2; kk <<= 1) {
        for (int jj = kk >> 1; jj > 0; jj >>= 1) {
            for (int t = threadIdx.x; t < np2; t += blockDim.x) {
                const int p = t ^ jj;
                if (p > t) {
                    const bool up = (t & kk) == 0;
                    const NaEntry A = e[t], B = e[p];
                    if (na_less(B, A) == up) {
                        e[t] = B;
                        e[p] = A;
                    }
                }
            }
            __syncthreads();
        }
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int nacc = 0;
        for (int t = 0; t < cnt && nacc < k; ++t) {
            const int64_t i = e[t].i;
            bool clash = false;
            for (int u = lane; u < nacc; u += 32)
                if (2 * llabs(i - acc_i[u]) <= m) clash = true;
            clash = __any_sync(0xffffffffu, clash);
            if (!clash) {
                if (lane == 0) {
                    acc_i[nacc] = i;
                    panache_motif mo;
                    mo.m = m;
                    mo._pad = 0;
                    mo.i = i;
                    mo.j = e[t].j;
                    mo.d = e[t].d;
                    out[nacc] = mo;
                }
                ++nacc;
                __syncwarp();
            }
        }
        if (lane == 0) *out_count = nacc;
    }
}

std::mutex g_na_mu;
NaScratch *g_na_ptr[NA_MAX_DEVICES] = {};

// Once per device, with that device current: the scratch's device address
// and the sort kernel's shared-memory limit.
int na_setup(int dev, NaScratch **out) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return PANACHE_ECUDA;
        const int sm = (int)(sizeof(NaEntry) * NA_POOL_MAX + sizeof(int64_t) * 1024);
        if (cudaFuncSetAttribute(k_na_greedy, cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess)
            return PANACHE_ECUDA;
        g_na_ptr[dev] = reinterpret_cast<NaScratch *>(p);
    }
    *out = g_na_ptr[dev];
    return PANACHE_OK;
}

}  // namespace

extern "C" int panache_topk_row_noalloc(const double *x, int64_t n, int32_t m, const uint64_t *keys, int32_t k,
                                        double eps0, panache_motif *out, int32_t *out_count, void *stream) {
    if (!x || !keys || !out || !out_count) return PANACHE_EINVAL;
    if (n < 1 || n > PN_MAX_SERIES_LEN || m < 3 || m > n || m > 1024 || k < 1 || k > 1024 || !(eps0 >= 0.0))
        return PANACHE_EINVAL;
    const int64_t need = (int64_t)k * (m + 1);
    if (need > PANACHE_NOALLOC_NEED_MAX) return PANACHE_EINVAL;
    // An error left pending by earlier work on this thread is not ours to
    // report or to clear: refuse to enqueue anything and leave it in place.
    if (cudaPeekAtLastError() != cudaSuccess) return PANACHE_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return PANACHE_ENODEV;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return PANACHE_ENODEV;
    NaScratch *s = nullptr;
    const int rc = na_setup(dev, &s);
    if (rc != PANACHE_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned long long *kk = reinterpret_cast<const unsigned long long *>(keys);
    const unsigned g = (unsigned)((n + 255) / 256);
    k_na_clear<<<16, 256, 0, st>>>(s);
    k_na_hist<<<g, 256, 0, st>>>(kk, n, eps0, 0, s);
    k_na_pick<<<1, 256, 0, st>>>(s, (uint32_t)need, 0);
    k_na_hist<<<g, 256, 0, st>>>(kk, n, eps0, 1, s);
    k_na_pick<<<1, 256, 0, st>>>(s, (uint32_t)need, 1);
    k_na_pool<<<g, 256, 0, st>>>(kk, n, m, eps0, s);
    k_na_verify<<<64, 256, 0, st>>>(x, m, eps0, s);
    const int sm = (int)(sizeof(NaEntry) * NA_POOL_MAX + sizeof(int64_t) * 1024);
    k_na_greedy<<<1, 1024, sm, st>>>(s, m, k, out, out_count);
    // only this call's launches can have set an error since the check above
    return cudaGetLastError() == cudaSuccess ? PANACHE_OK : PANACHE_ECUDA;
}
