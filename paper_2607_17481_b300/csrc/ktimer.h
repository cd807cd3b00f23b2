// Device time of the kernels the per-kernel roofline report names, taken
// with CUDA events on the launching stream around each launch
// (PANACHE_FLAG_TIMING) and summed per kernel when the request's results are
// read.  Host code only.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>
#include <vector>

enum PnKernelId {
    PN_KT_ANCHOR_TC = 0,   // tensor-core chunk anchors
    PN_KT_FEATURES,        // sliding DFT, normalisation, keys
    PN_KT_SEARCH,          // streaming search
    PN_KT_SIEVE,           // hot-class sieve evaluation (after its sorts)
    PN_KT_COMPLETE,        // local completion rounds
    PN_KT_SELECT,          // selection kernels (seed selections and the final top-k)
    PN_KT_REFINE,          // exact row refinement of the top list
    PN_KT_TOPK,            // top-k sieve after the emit stage (focused or every anchor; with its pre-pass)
    PN_KT_COUNT
};

struct PnKTimer {
    bool on = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PN_KT_COUNT];
    double ms[PN_KT_COUNT] = {};
    uint64_t launches[PN_KT_COUNT] = {};

    ~PnKTimer() { release(); }
    void release() {
        for (auto &v : ev) {
            for (auto &p : v) {
                cudaEventDestroy(p.first);
                cudaEventDestroy(p.second);
            }
            v.clear();
        }
    }
    // Starts a request: clears the sums; timing is on when `enable`.
    void reset(bool enable) {
        release();
        on = enable;
        for (int k = 0; k < PN_KT_COUNT; ++k) {
            ms[k] = 0.0;
            launches[k] = 0;
        }
    }
    void begin(int k, cudaStream_t st) {
        if (!on) return;
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess) return;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return;
        }
        cudaEventRecord(a, st);
        ev[k].push_back({a, b});
    }
    void end(int k, cudaStream_t st) {
        if (!on || ev[k].empty()) return;
        cudaEventRecord(ev[k].back().second, st);
        ++launches[k];
    }
    // Adds up the recorded launches (waits for the last event of each kernel).
    void collect() {
        if (!on) return;
        for (int k = 0; k < PN_KT_COUNT; ++k) {
            for (auto &p : ev[k]) {
                float t = 0.0f;
                if (cudaEventSynchronize(p.second) == cudaSuccess &&
                    cudaEventElapsedTime(&t, p.first, p.second) == cudaSuccess)
                    ms[k] += t;
            }
        }
        release();
    }
};

inline void pn_kt_begin(PnKTimer *t, int k, cudaStream_t st) {
    if (t) t->begin(k, st);
}
inline void pn_kt_end(PnKTimer *t, int k, cudaStream_t st) {
    if (t) t->end(k, st);
}
