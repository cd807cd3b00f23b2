// Request server: continuous batching of pan-motif requests under an HBM
// budget, with live streams whose samples stay resident on the device.
//
// Slots: every slot is a host worker thread with its own context and CUDA
// stream, so the requests of different slots run concurrently on the GPU.
// Admission: a request reserves its device footprint (the planner's
// estimate) from the server budget before it runs and releases it when its
// results are on the host; a request larger than the whole budget is refused
// at submission (PANACHE_EBUDGET).  With a deadline set, a request whose
// predicted wait -- the work on the GPU and queued ahead of it and its own,
// in windows x lengths, over the server's measured throughput -- exceeds the
// deadline is refused at submission (PANACHE_EBUSY): above capacity the
// server sheds load instead of letting every request's latency grow.  A
// stream snapshot is refused the same way when the snapshots queued ahead
// of it, at the measured time per snapshot, would keep it past the deadline.
// Continuous batching: a free slot takes, in arrival order, every queued
// request that still fits both the free budget and the slot's share of it,
// and runs them as one batch (one set of launches); requests that arrive
// while others are on the GPU wait only for the next free slot.
// Live streams: appends and snapshots are queued per stream and applied by
// stream worker threads, each stream on a context (and CUDA stream) of its
// own, so they overlap one another and the slots' batches; consecutive
// pending appends of a stream are applied as one.
// Latency of a request: from submission to its motifs being on the host; of
// a snapshot: from its call to its motifs being on the host.
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

#define PN_STREAM_MAX_LEN ((int64_t)((1ull << 26) - 1))

// Share of a deadline that a predicted wait may use (the rest covers the
// error of the throughput estimate).
static constexpr double kDeadlineShare = 0.75;

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

// One pending operation of a live stream, applied in order by a stream worker.
struct StreamOp {
    bool snapshot = false;
    std::vector<double> samples;             // an append's samples (FP64)
    int64_t cap_after = 0;                   // the capacity reserved for the stream after this append
    uint64_t ticket = 0;                     // a snapshot's ticket
    double t_enq = 0.0;
};

// A live stream: its whole index stays resident on the device (a resident
// panache_stream on a context, and so a CUDA stream, of its own).  Appends
// and snapshots are queued (ops) and applied by a stream worker.  The
// resident state, plus the row copy a snapshot works on, is reserved from the
// server's budget when an append is accepted; an append that would grow it
// past the budget is refused (EBUDGET) at the call.
struct LiveStream {
    std::mutex ops_mu;                       // ops, accepted, planned_cap, scheduled, err
    std::deque<StreamOp> ops;
    int64_t accepted = 0;                    // samples accepted (applied or pending)
    int64_t planned_cap = 0;                 // capacity after every accepted append
    bool scheduled = false;                  // on the server's stream work list
    int err = PANACHE_OK;                    // first failure of an applied append (sticky)
    std::mutex exec_mu;                      // held while a worker applies ops
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
    std::unordered_map<uint64_t, std::shared_ptr<LiveStream>> streams;
    std::mutex streams_mu;
    // stream workers: streams with pending ops, in the order they were scheduled
    std::deque<std::shared_ptr<LiveStream>> stream_work;
    std::condition_variable cv_stream;
    std::vector<std::thread> stream_workers;
    // deadline admission: work in flight and queued, and the measured throughput
    double deadline_ms = 0.0;
    uint64_t queued_wl = 0;
    uint64_t inflight_wl = 0;                // windows x lengths of the batches on the GPU
    double rate_wl_per_ms = 0.0;             // per batch, smoothed; times the slots for the server
    std::deque<std::pair<double, uint64_t>> recent;   // (completion time, windows x lengths), last 2 s
    uint64_t snaps_queued = 0;               // snapshots accepted and not yet served
    double snap_ms = 0.0;                    // smoothed time a stream worker spends on one snapshot
    int n_stream_workers = 2;

    // Requests' throughput in windows x lengths per ms: what completed in the
    // last two seconds (it includes every other use of the GPU), or, before
    // that window fills, the smoothed per-batch rate times the slots.
    double request_rate(double now) const {
        if (recent.size() >= 3 && now - recent.front().first >= 250.0) {
            uint64_t w = 0;
            for (auto &e : recent) w += e.second;
            return (double)w / (now - recent.front().first);
        }
        return rate_wl_per_ms * (double)slots;
    }
    // statistics
    uint64_t submitted = 0, completed = 0, failed = 0, refused = 0, refused_snaps = 0, batches = 0, wl = 0;
    std::vector<double> latencies, snap_latencies;
    double t_first = 0.0, t_last = 0.0;
    int max_concurrent = 0, running = 0;

    void worker(int slot);
    void stream_worker();
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
                queued_wl -= std::min<uint64_t>(queued_wl, (uint64_t)windows_lengths(j.s));
                inflight_wl += (uint64_t)windows_lengths(j.s);
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
        const double t_start = now_ms();
        const int rc = pn_rt::run(ctx, in, res);
        const double t = now_ms();
        {
            std::lock_guard<std::mutex> lk(mu);
            in_use -= fp;
            --running;
            for (auto &j : batch) inflight_wl -= std::min<uint64_t>(inflight_wl, (uint64_t)windows_lengths(j.s));
            if (rc == PANACHE_OK && t > t_start) {
                uint64_t bw = 0;
                for (auto &j : batch) bw += (uint64_t)windows_lengths(j.s);
                const double r = (double)bw / (t - t_start);
                rate_wl_per_ms = rate_wl_per_ms > 0.0 ? 0.8 * rate_wl_per_ms + 0.2 * r : r;
            }
            for (size_t b = 0; b < batch.size(); ++b) {
                Result r;
                r.rc = rc;
                if (rc == PANACHE_OK) r.motifs = std::move(res[b]);
                r.latency_ms = t - batch[b].t_submit;
                if (rc == PANACHE_OK) {
                    ++completed;
                    wl += (uint64_t)windows_lengths(batch[b].s);
                    latencies.push_back(r.latency_ms);
                    recent.emplace_back(t, (uint64_t)windows_lengths(batch[b].s));
                } else {
                    ++failed;
                }
                t_last = t;
                done[batch[b].ticket] = std::move(r);
            }
            while (!recent.empty() && t - recent.front().first > 2000.0) recent.pop_front();
        }
        cv_done.notify_all();
        cv_work.notify_all();
    }
}

// Files a stream snapshot's result under its ticket.
static void file_snapshot(panache_server *sv, uint64_t ticket, Result &&r, int64_t n, const LiveStream &ls) {
    const double t = now_ms();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (r.rc == PANACHE_OK) {
            ++sv->completed;
            sv->wl += (uint64_t)windows_lengths(PnSeriesIn{nullptr, 0, n, ls.m_min, ls.m_max, ls.k, ls.excl});
            sv->snap_latencies.push_back(r.latency_ms);
        } else {
            ++sv->failed;
        }
        sv->t_last = t;
        sv->done[ticket] = std::move(r);
    }
    sv->cv_done.notify_all();
}

// Applies the pending ops of one stream at a time: runs of consecutive
// appends as one append (to the capacity reserved for the last of them),
// snapshots in their place in the order.
void panache_server::stream_worker() {
    cudaSetDevice(device);
    for (;;) {
        std::shared_ptr<LiveStream> ls;
        {
            std::unique_lock<std::mutex> lk(streams_mu);
            cv_stream.wait(lk, [&] { return !stream_work.empty() || stop; });
            if (stream_work.empty()) return;             // stopping and drained
            ls = std::move(stream_work.front());
            stream_work.pop_front();
        }
        std::lock_guard<std::mutex> ex(ls->exec_mu);
        for (;;) {
            std::vector<StreamOp> run;
            {
                std::lock_guard<std::mutex> o(ls->ops_mu);
                if (ls->ops.empty()) {
                    ls->scheduled = false;
                    break;
                }
                if (ls->ops.front().snapshot) {
                    run.push_back(std::move(ls->ops.front()));
                    ls->ops.pop_front();
                } else {
                    while (!ls->ops.empty() && !ls->ops.front().snapshot) {
                        run.push_back(std::move(ls->ops.front()));
                        ls->ops.pop_front();
                    }
                }
            }
            if (run[0].snapshot) {
                const double t_snap = now_ms();
                Result r;
                int64_t n = panache_stream_length(ls->h);
                {
                    std::lock_guard<std::mutex> o(ls->ops_mu);
                    r.rc = ls->err;
                }
                if (r.rc == PANACHE_OK && n == 0) r.rc = PANACHE_ESTATE;
                if (r.rc == PANACHE_OK) {
                    std::vector<panache_motif> out((size_t)ls->k * (size_t)(ls->m_max - ls->m_min + 1));
                    int64_t got = 0;
                    r.rc = panache_stream_topk(ls->h, out.data(), (int64_t)out.size(), &got);
                    if (r.rc == PANACHE_OK) r.motifs.assign(out.begin(), out.begin() + got);
                }
                const double t_end = now_ms();
                r.latency_ms = t_end - run[0].t_enq;
                {
                    std::lock_guard<std::mutex> lk(mu);
                    const double took = t_end - t_snap;
                    snap_ms = snap_ms > 0.0 ? 0.8 * snap_ms + 0.2 * took : took;
                    if (snaps_queued) --snaps_queued;
                }
                file_snapshot(this, run[0].ticket, std::move(r), n, *ls);
                continue;
            }
            size_t total = 0;
            for (auto &op : run) total += op.samples.size();
            std::vector<double> buf;
            const double *src = run[0].samples.data();
            if (run.size() > 1) {
                buf.reserve(total);
                for (auto &op : run) buf.insert(buf.end(), op.samples.begin(), op.samples.end());
                src = buf.data();
            }
            const int rc = pn_rt::append_to(ls->h, src, PANACHE_F64, (int64_t)total, run.back().cap_after);
            if (rc != PANACHE_OK) {
                std::lock_guard<std::mutex> o(ls->ops_mu);
                if (ls->err == PANACHE_OK) ls->err = rc;
            }
        }
    }
}

static int enqueue(panache_server *sv, Job &&j, uint64_t *ticket) {
    uint64_t fp = 0;
    const int rc = pn_rt::footprint(sv->ctxs[0], j.s, &fp);
    if (rc != PANACHE_OK) return rc;
    if (fp > sv->budget) return PANACHE_EBUDGET;
    j.footprint = fp;
    const uint64_t w = (uint64_t)windows_lengths(j.s);
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        const double rate = sv->request_rate(now_ms());
        if (sv->deadline_ms > 0.0 && rate > 0.0) {
            // predicted wait: the work on the GPU and queued ahead and this
            // request's own, at the server's measured throughput; a quarter of
            // the deadline is kept for the error of that estimate (the live
            // streams share the GPU and move the rate)
            if ((double)(sv->inflight_wl + sv->queued_wl + w) / rate > kDeadlineShare * sv->deadline_ms) {
                ++sv->refused;
                return PANACHE_EBUSY;
            }
        }
        j.ticket = sv->next_ticket++;
        j.t_submit = now_ms();
        if (!sv->submitted) sv->t_first = j.t_submit;
        ++sv->submitted;
        sv->queued_wl += w;
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
    sv->n_stream_workers = std::max(4, 2 * slots);
    for (int s = 0; s < sv->n_stream_workers; ++s)
        sv->stream_workers.emplace_back(&panache_server::stream_worker, sv.get());
    *out = sv.release();
    return PANACHE_OK;
}

void panache_server_destroy(panache_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        std::lock_guard<std::mutex> ls(sv->streams_mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->cv_stream.notify_all();
    for (auto &t : sv->workers) t.join();
    for (auto &t : sv->stream_workers) t.join();     // pending stream ops are applied first
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
    std::shared_ptr<LiveStream> ls(new (std::nothrow) LiveStream());
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

static std::shared_ptr<LiveStream> find_stream(panache_server *sv, uint64_t id) {
    std::lock_guard<std::mutex> lk(sv->streams_mu);
    auto it = sv->streams.find(id);
    return it == sv->streams.end() ? nullptr : it->second;
}

// Queues an op and puts the stream on the work list (ops_mu held by the caller).
static void schedule(panache_server *sv, const std::shared_ptr<LiveStream> &ls) {
    if (ls->scheduled) return;
    ls->scheduled = true;
    {
        std::lock_guard<std::mutex> lk(sv->streams_mu);
        sv->stream_work.push_back(ls);
    }
    sv->cv_stream.notify_one();
}

int panache_server_append(panache_server *sv, uint64_t stream_id, const void *chunk, int32_t dtype, int64_t len) {
    if (!sv || len < 0 || (len > 0 && !chunk)) return PANACHE_EINVAL;
    const int dt = dtype & 0xFF;
    if ((dt != PANACHE_F32 && dt != PANACHE_F64) || (dtype & PANACHE_DEVICE)) return PANACHE_EINVAL;
    std::shared_ptr<LiveStream> ls = find_stream(sv, stream_id);
    if (!ls) return PANACHE_EINVAL;
    if (!len) return PANACHE_OK;
    StreamOp op;
    op.samples.resize((size_t)len);
    if (dt == PANACHE_F32) {
        const float *f = static_cast<const float *>(chunk);
        for (int64_t t = 0; t < len; ++t) op.samples[t] = (double)f[t];
    } else {
        memcpy(op.samples.data(), chunk, sizeof(double) * (size_t)len);
    }
    std::lock_guard<std::mutex> o(ls->ops_mu);
    if (ls->err != PANACHE_OK) return ls->err;
    if (ls->accepted + len > PN_STREAM_MAX_LEN) return PANACHE_EINVAL;
    const int64_t ncap = pn_rt::grow_capacity(ls->planned_cap, ls->accepted + len);
    if (ncap != ls->planned_cap) {
        // reserve the grown state (and its snapshot row copy) before accepting
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
        ls->planned_cap = ncap;
    }
    ls->accepted += len;
    op.cap_after = ls->planned_cap;
    ls->ops.push_back(std::move(op));
    schedule(sv, ls);
    return PANACHE_OK;
}

int panache_server_stream_topk(panache_server *sv, uint64_t stream_id, uint64_t *ticket) {
    if (!sv || !ticket) return PANACHE_EINVAL;
    std::shared_ptr<LiveStream> ls = find_stream(sv, stream_id);
    if (!ls) return PANACHE_EINVAL;
    StreamOp op;
    op.snapshot = true;
    op.t_enq = now_ms();
    std::lock_guard<std::mutex> o(ls->ops_mu);
    if (ls->accepted == 0) return PANACHE_ESTATE;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        // a snapshot waits for those queued before it, served by the stream workers
        if (sv->deadline_ms > 0.0 && sv->snap_ms > 0.0 &&
            (double)(sv->snaps_queued + 1) * sv->snap_ms / (double)sv->n_stream_workers > kDeadlineShare * sv->deadline_ms) {
            ++sv->refused_snaps;
            return PANACHE_EBUSY;
        }
        ++sv->snaps_queued;
        op.ticket = sv->next_ticket++;
        if (!sv->submitted) sv->t_first = op.t_enq;
        ++sv->submitted;
    }
    *ticket = op.ticket;
    ls->ops.push_back(std::move(op));
    schedule(sv, ls);
    return PANACHE_OK;
}

int panache_server_stream_close(panache_server *sv, uint64_t stream_id) {
    if (!sv) return PANACHE_EINVAL;
    std::shared_ptr<LiveStream> ls;
    {
        std::lock_guard<std::mutex> lk(sv->streams_mu);
        auto it = sv->streams.find(stream_id);
        if (it == sv->streams.end()) return PANACHE_EINVAL;
        ls = std::move(it->second);
        sv->streams.erase(it);
    }
    // the stream's pending ops are applied first (a snapshot asked for before
    // the close still gets its result)
    for (;;) {
        {
            std::lock_guard<std::mutex> ex(ls->exec_mu);
            std::lock_guard<std::mutex> o(ls->ops_mu);
            if (ls->ops.empty() && !ls->scheduled) break;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(200));
    }
    cudaSetDevice(sv->device);
    const uint64_t r = ls->reserved;
    {
        std::lock_guard<std::mutex> ex(ls->exec_mu);
        if (ls->h) panache_stream_close(ls->h);
        ls->h = nullptr;
        if (ls->ctx) panache_destroy(ls->ctx);
        ls->ctx = nullptr;
    }
    std::lock_guard<std::mutex> g(sv->mu);
    sv->in_use -= r;
    return PANACHE_OK;
}

int panache_server_set_deadline(panache_server *sv, double deadline_ms) {
    if (!sv || !(deadline_ms >= 0.0)) return PANACHE_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->deadline_ms = deadline_ms;
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
    out->refused = sv->refused;
    out->refused_snapshots = sv->refused_snaps;
    auto pct = [](std::vector<double> l, double p) {
        std::sort(l.begin(), l.end());
        const double pos = p * (double)(l.size() - 1);
        const size_t lo = (size_t)pos, hi = std::min(lo + 1, l.size() - 1);
        return l[lo] + (l[hi] - l[lo]) * (pos - (double)lo);
    };
    if (!sv->latencies.empty()) {
        out->p50_ms = pct(sv->latencies, 0.50);
        out->p99_ms = pct(sv->latencies, 0.99);
        double s = 0;
        for (double v : sv->latencies) s += v;
        out->mean_ms = s / (double)sv->latencies.size();
    }
    if (!sv->snap_latencies.empty()) {
        out->snap_p50_ms = pct(sv->snap_latencies, 0.50);
        out->snap_p99_ms = pct(sv->snap_latencies, 0.99);
    }
    return PANACHE_OK;
}

}  // extern "C"
