// Request server: continuous batching of pan-motif requests under an HBM
// budget, with live streams whose samples stay resident on the device.
//
// Slots: every slot is a host worker thread with its own context and CUDA
// stream, so the requests of different slots run concurrently on the GPU.
// Admission: a request reserves its device footprint (the planner's
// estimate) from the server budget before it runs and releases it when its
// results are on the host; a request larger than the whole budget is refused
// at submission (PANACHE_EBUDGET).
// Continuous batching: a free slot takes, in arrival order, every queued
// request that still fits both the free budget and the slot's share of it,
// and runs them as one batch (one set of launches); requests that arrive
// while others are on the GPU wait only for the next free slot.
// Latency of a request: from submission to its motifs being on the host.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "panache.h"
#include "runtime.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct Job {
    uint64_t ticket = 0;
    std::vector<unsigned char> host;          // caller's samples, copied at submission
    PnSeriesIn s{};
    uint64_t footprint = 0;
    double t_submit = 0.0;
};

struct Result {
    int rc = PANACHE_OK;
    std::vector<panache_motif> motifs;
    double latency_ms = 0.0;
};

// A live stream: its whole index stays resident on the device (a resident
// panache_stream on a context, and so a CUDA stream, of its own).  Appends
// and snapshots run in the calling thread and overlap the slots' batches on
// the GPU.  The resident state, plus the row copy a snapshot works on, is
// reserved from the server's budget; an append that would grow it past the
// budget is refused (EBUDGET).
struct LiveStream {
    std::mutex mu;
    panache_ctx *ctx = nullptr;
    panache_stream *h = nullptr;
    uint64_t reserved = 0;
    int32_t m_min, m_max, k, excl;
    ~LiveStream() {
        if (h) panache_stream_close(h);
        if (ctx) panache_destroy(ctx);
    }
};

}  // namespace

struct panache_server {
    panache_config cfg{};
    int device = 0;
    int slots = 1;
    uint64_t budget = 0, in_use = 0, peak_in_use = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job> queue;
    std::unordered_map<uint64_t, Result> done;
    std::vector<std::thread> workers;
    std::vector<panache_ctx *> ctxs;
    bool stop = false;
    uint64_t next_ticket = 1, next_stream = 1;
    std::unordered_map<uint64_t, std::unique_ptr<LiveStream>> streams;
    std::mutex streams_mu;
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, batches = 0, wl = 0;
    std::vector<double> latencies;
    double t_first = 0.0, t_last = 0.0;
    int max_concurrent = 0, running = 0;

    void worker(int slot);
};

static int64_t windows_lengths(const PnSeriesIn &s) {
    int64_t w = 0;
    for (int m = s.m_min; m <= s.m_max; ++m) w += std::max<int64_t>(0, s.n - m + 1);
    return w;
}

void panache_server::worker(int slot) {
    cudaSetDevice(device);
    panache_ctx *ctx = ctxs[slot];
    const uint64_t share = std::max<uint64_t>(budget / (uint64_t)slots, 1);
    for (;;) {
        std::vector<Job> batch;
        uint64_t fp = 0;
        {
            std::unique_lock<std::mutex> lk(mu);
            // a request that does not fit while no batch runs can only wait for
            // live streams to close: it is refused (EBUDGET) instead of waiting
            cv_work.wait(lk, [&] {
                return (!queue.empty() && (in_use + queue.front().footprint <= budget || running == 0)) ||
                       (stop && queue.empty());
            });
            if (queue.empty()) return;                    // stopping and drained
            if (in_use + queue.front().footprint > budget) {
                Result r;
                r.rc = PANACHE_EBUDGET;
                r.latency_ms = now_ms() - queue.front().t_submit;
                ++failed;
                done[queue.front().ticket] = std::move(r);
                queue.pop_front();
                cv_done.notify_all();
                continue;
            }
            while (!queue.empty()) {
                const Job &j = queue.front();
                const bool fits = in_use + fp + j.footprint <= budget;
                const bool in_share = batch.empty() || fp + j.footprint <= share;
                if (!fits || !in_share) break;
                fp += j.footprint;
                batch.push_back(std::move(queue.front()));
                queue.pop_front();
            }
            in_use += fp;
            peak_in_use = std::max(peak_in_use, in_use);
            ++running;
            max_concurrent = std::max(max_concurrent, running);
            ++batches;
        }
        std::vector<PnSeriesIn> in;
        for (auto &j : batch) {
            PnSeriesIn s = j.s;
            s.ptr = (const void *)j.host.data();
            in.push_back(s);
        }
        std::vector<std::vector<panache_motif>> res;
        const int rc = pn_rt::run(ctx, in, res);
        const double t = now_ms();
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use -= fp;
            --running;
            for (size_t b = 0; b < batch.size(); ++b) {
                Result r;
                r.rc = rc;
                if (rc == PANACHE_OK) r.motifs = std::move(res[b]);
                r.latency_ms = t - batch[b].t_submit;
                if (rc == PANACHE_OK) {
                    ++completed;
                    wl += (uint64_t)windows_lengths(batch[b].s);
                    latencies.push_back(r.latency_ms);
                } else {
                    ++failed;
                }
                t_last = t;
                done[batch[b].ticket] = std::move(r);
            }
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

static int enqueue(panache_server *sv, Job &&j, uint64_t *ticket) {
    uint64_t fp = 0;
    const int rc = pn_rt::footprint(sv->ctxs[0], j.s, &fp);
    if (rc != PANACHE_OK) return rc;
    if (fp > sv->budget) return PANACHE_EBUDGET;
    j.footprint = fp;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        j.ticket = sv->next_ticket++;
        j.t_submit = now_ms();
        if (!sv->submitted) sv->t_first = j.t_submit;
        ++sv->submitted;
        *ticket = j.ticket;
        sv->queue.push_back(std::move(j));
    }
    sv->cv_work.notify_all();
    return PANACHE_OK;
}

extern "C" {

int panache_server_create(const panache_config *cfg, int32_t slots, uint64_t hbm_budget_bytes,
                          panache_server **out) {
    if (!out || slots < 1 || slots > 64) return PANACHE_EINVAL;
    *out = nullptr;
    std::unique_ptr<panache_server> sv(new (std::nothrow) panache_server());
    if (!sv) return PANACHE_ENOMEM;
    if (cfg) sv->cfg = *cfg;
    if (cudaGetDevice(&sv->device) != cudaSuccess) return PANACHE_ENODEV;
    sv->slots = slots;
    if (!hbm_budget_bytes) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return PANACHE_ECUDA;
        hbm_budget_bytes = (uint64_t)(0.6 * (double)fr);
    }
    sv->budget = hbm_budget_bytes;
    for (int s = 0; s < slots; ++s) {
        panache_ctx *c = nullptr;
        const int rc = panache_create(cfg, &c);
        if (rc != PANACHE_OK) {
            for (auto *x : sv->ctxs) panache_destroy(x);
            return rc;
        }
        sv->ctxs.push_back(c);
    }
    for (int s = 0; s < slots; ++s) sv->workers.emplace_back(&panache_server::worker, sv.get(), s);
    *out = sv.release();
    return PANACHE_OK;
}

void panache_server_destroy(panache_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    for (auto &t : sv->workers) t.join();
    cudaSetDevice(sv->device);
    {
        std::lock_guard<std::mutex> lk(sv->streams_mu);
        sv->streams.clear();
    }
    for (auto *c : sv->ctxs) panache_destroy(c);
    delete sv;
}

int panache_server_submit(panache_server *sv, const void *series, int32_t dtype, int64_t n, int32_t m_min,
                          int32_t m_max, int32_t k, int32_t excl, uint64_t *ticket) {
    if (!sv || !ticket || (n > 0 && !series) || n < 0) return PANACHE_EINVAL;
    const int dt = dtype & 0xFF;
    if ((dt != PANACHE_F32 && dt != PANACHE_F64) || (dtype & PANACHE_DEVICE)) return PANACHE_EINVAL;
    Job j;
    const size_t es = dt == PANACHE_F32 ? 4 : 8;
    j.host.resize((size_t)n * es);
    if (n) memcpy(j.host.data(), series, (size_t)n * es);
    j.s = PnSeriesIn{nullptr, dt, n, m_min, m_max, k, excl};
    return enqueue(sv, std::move(j), ticket);
}

int panache_server_wait(panache_server *sv, uint64_t ticket, int32_t timeout_ms, panache_motif *out, int64_t cap,
                        int64_t *out_len, double *latency_ms) {
    if (!sv || !out_len) return PANACHE_EINVAL;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto ready = [&] { return sv->done.count(ticket) != 0; };
    if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
    else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) return PANACHE_ETIMEOUT;
    Result &r = sv->done[ticket];
    if (r.rc != PANACHE_OK) {
        const int rc = r.rc;
        sv->done.erase(ticket);
        return rc;
    }
    *out_len = (int64_t)r.motifs.size();
    if (latency_ms) *latency_ms = r.latency_ms;
    if ((int64_t)r.motifs.size() > cap) return PANACHE_ETRUNC;
    if (!r.motifs.empty()) {
        if (!out) return PANACHE_EINVAL;
        memcpy(out, r.motifs.data(), sizeof(panache_motif) * r.motifs.size());
    }
    sv->done.erase(ticket);
    return PANACHE_OK;
}

int panache_server_stream_open(panache_server *sv, int32_t m_min, int32_t m_max, int32_t k, int32_t excl,
                               uint64_t *stream_id) {
    if (!sv || !stream_id) return PANACHE_EINVAL;
    if (m_min < 3 || m_max < m_min || m_max > 1024 || k < 1 || excl < 1) return PANACHE_EINVAL;
    std::unique_ptr<LiveStream> ls(new (std::nothrow) LiveStream());
    if (!ls) return PANACHE_ENOMEM;
    ls->m_min = m_min;
    ls->m_max = m_max;
    ls->k = k;
    ls->excl = excl;
    cudaSetDevice(sv->device);
    panache_config c = sv->cfg;
    c.hbm_budget_bytes = 0;                       // the server's budget governs
    int rc = panache_create(&c, &ls->ctx);
    if (rc == PANACHE_OK) rc = panache_stream_open(ls->ctx, m_min, m_max, k, excl, &ls->h);
    if (rc != PANACHE_OK) return rc;
    std::lock_guard<std::mutex> lk(sv->streams_mu);
    *stream_id = sv->next_stream++;
    sv->streams[*stream_id] = std::move(ls);
    return PANACHE_OK;
}

static LiveStream *find_stream(panache_server *sv, uint64_t id) {
    std::lock_guard<std::mutex> lk(sv->streams_mu);
    auto it = sv->streams.find(id);
    return it == sv->streams.end() ? nullptr : it->second.get();
}

int panache_server_append(panache_server *sv, uint64_t stream_id, const void *chunk, int32_t dtype, int64_t len) {
    if (!sv || len < 0 || (len > 0 && !chunk)) return PANACHE_EINVAL;
    const int dt = dtype & 0xFF;
    if ((dt != PANACHE_F32 && dt != PANACHE_F64) || (dtype & PANACHE_DEVICE)) return PANACHE_EINVAL;
    LiveStream *ls = find_stream(sv, stream_id);
    if (!ls) return PANACHE_EINVAL;
    if (!len) return PANACHE_OK;
    cudaSetDevice(sv->device);
    std::lock_guard<std::mutex> lk(ls->mu);
    const int64_t have = panache_stream_length(ls->h), cap = pn_rt::stream_capacity(ls->h);
    const int64_t ncap = pn_rt::grow_capacity(cap, have + len);
    if (ncap != cap) {
        // reserve the grown state (and its snapshot row copy) before growing
        uint64_t fp = 0;
        const PnSeriesIn s{chunk, dt, ncap, ls->m_min, ls->m_max, ls->k, ls->excl};
        int rc = pn_rt::footprint(ls->ctx, s, &fp);
        if (rc != PANACHE_OK) return rc;
        fp += (uint64_t)(ls->m_max - ls->m_min + 1) * (uint64_t)ncap * 8u;
        std::lock_guard<std::mutex> g(sv->mu);
        if (sv->in_use - ls->reserved + fp > sv->budget) return PANACHE_EBUDGET;
        sv->in_use = sv->in_use - ls->reserved + fp;
        sv->peak_in_use = std::max(sv->peak_in_use, sv->in_use);
        ls->reserved = fp;
    }
    return panache_append(ls->h, chunk, dtype, len);
}

int panache_server_stream_topk(panache_server *sv, uint64_t stream_id, uint64_t *ticket) {
    if (!sv || !ticket) return PANACHE_EINVAL;
    LiveStream *ls = find_stream(sv, stream_id);
    if (!ls) return PANACHE_EINVAL;
    cudaSetDevice(sv->device);
    const double t0 = now_ms();
    Result r;
    int64_t n = 0;
    {
        std::lock_guard<std::mutex> lk(ls->mu);
        n = panache_stream_length(ls->h);
        if (n == 0) return PANACHE_ESTATE;
        std::vector<panache_motif> out((size_t)ls->k * (size_t)(ls->m_max - ls->m_min + 1));
        int64_t got = 0;
        r.rc = panache_stream_topk(ls->h, out.data(), (int64_t)out.size(), &got);
        if (r.rc == PANACHE_OK) r.motifs.assign(out.begin(), out.begin() + got);
    }
    const double t = now_ms();
    r.latency_ms = t - t0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        *ticket = sv->next_ticket++;
        if (!sv->submitted) sv->t_first = t0;
        ++sv->submitted;
        if (r.rc == PANACHE_OK) {
            ++sv->completed;
            sv->wl += (uint64_t)windows_lengths(PnSeriesIn{nullptr, 0, n, ls->m_min, ls->m_max, ls->k, ls->excl});
            sv->latencies.push_back(r.latency_ms);
        } else {
            ++sv->failed;
        }
        sv->t_last = t;
        sv->done[*ticket] = std::move(r);
    }
    sv->cv_done.notify_all();
    return PANACHE_OK;
}

int panache_server_stream_close(panache_server *sv, uint64_t stream_id) {
    if (!sv) return PANACHE_EINVAL;
    std::unique_ptr<LiveStream> ls;
    {
        std::lock_guard<std::mutex> lk(sv->streams_mu);
        auto it = sv->streams.find(stream_id);
        if (it == sv->streams.end()) return PANACHE_EINVAL;
        ls = std::move(it->second);
        sv->streams.erase(it);
    }
    {
        std::lock_guard<std::mutex> lk(ls->mu);     // no append or snapshot of this stream in flight
    }
    cudaSetDevice(sv->device);
    const uint64_t r = ls->reserved;
    ls.reset();
    std::lock_guard<std::mutex> g(sv->mu);
    sv->in_use -= r;
    return PANACHE_OK;
}

int panache_server_get_stats(panache_server *sv, panache_server_stats *out) {
    if (!sv || !out) return PANACHE_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    memset(out, 0, sizeof(*out));
    out->submitted = sv->submitted;
    out->completed = sv->completed;
    out->failed = sv->failed;
    out->queued = sv->queue.size();
    out->batches = sv->batches;
    out->windows_lengths = sv->wl;
    out->budget_bytes = sv->budget;
    out->peak_reserved_bytes = sv->peak_in_use;
    out->max_concurrent_batches = (uint32_t)sv->max_concurrent;
    out->span_ms = sv->completed ? sv->t_last - sv->t_first : 0.0;
    if (!sv->latencies.empty()) {
        std::vector<double> l = sv->latencies;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {
            const double pos = p * (double)(l.size() - 1);
            const size_t lo = (size_t)pos, hi = std::min(lo + 1, l.size() - 1);
            return l[lo] + (l[hi] - l[lo]) * (pos - (double)lo);
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        double s = 0;
        for (double v : l) s += v;
        out->mean_ms = s / (double)l.size();
    }
    return PANACHE_OK;
}

}  // extern "C"
