// Internal interface between the C ABI's request runner (capi.cu) and the
// request server (server.cu).
#pragma once
#include <stdint.h>

#include <vector>

#include "panache.h"

struct PnSeriesIn {          // one series of a request, as the caller gave it
    const void *ptr;
    int32_t dtype;           // PANACHE_F32 / PANACHE_F64, optionally | PANACHE_DEVICE
    int64_t n;
    int32_t m_min, m_max, k, excl;
};

namespace pn_rt {
// Runs the whole path for a list of series on ctx's stream; results per series.
int run(panache_ctx *ctx, const std::vector<PnSeriesIn> &in, std::vector<std::vector<panache_motif>> &res);
// Device footprint of one series under ctx's configuration (admission estimate).
int footprint(panache_ctx *ctx, const PnSeriesIn &s, uint64_t *bytes);
// Resident capacity of a stream, and the capacity an append of `need` total
// samples grows it to (the stream keeps its capacity when need fits).
int64_t stream_capacity(const panache_stream *h);
int64_t grow_capacity(int64_t cap, int64_t need);
// panache_append, except that an append that outgrows the capacity rebuilds
// the state at exactly `cap` (when cap holds the samples): several appends
// applied as one then reach the capacity reserved for them one by one.
int append_to(panache_stream *h, const void *chunk, int32_t dtype, int64_t len, int64_t cap);
}  // namespace pn_rt
