"""Throughput of the Panache pan-motif path on one B300 (windows x lengths per second).

Workload (the configuration the metric is quoted on): the precision form on
a 5,000,000-sample float32 wafer-like series (152-sample step/plateau
segments, seed 0), lengths 100..150 (51 lengths, 26 anchors), top-20
pan-motifs over the whole stack, exclusion zone 150: FP32 sliding-DFT state
re-anchored every 256 slides by 3xTF32 tensor-core contractions, FP64 prefix
sums, FP32 bounds and in-stream distances, FP64 verification of every
reported distance.  One step = one full request: samples on the device ->
index (features, keys, directories) -> streaming search -> sieve ->
completion -> FP64-verified top-20 on the host.  The plain FP64 form runs on
the same series as the comparator.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  N > 1 runs one independent replica per GPU
(the single-series path does not shard; weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "windows*lengths/sec to exact top-20 pan-motifs (recall 1.0) vs plain FP64 form; p50/p99"
UNIT = "windows*lengths/s"
WORKLOAD = dict(workload="wafer_like_5M", n=5_000_000, m_min=100, m_max=150, k=20, excl=150, seed=0,
                dtype="float32", topk="global")
STRIDE = 2                       # the paper's anchor stride (the library's default for the global top-k)


def rank_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in self.lines:
            p = [t.strip() for t in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, val in zip(names, p[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def measured_traffic(queries: int):
    """DRAM bytes per search launch from the committed ncu capture, scaled by queries.

    Null when the kernel's sources changed since the capture (hashes differ).
    """
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)["k_search"]
    except (OSError, KeyError, ValueError):
        return None
    for path, want in t["sources_sha256_16"].items():
        with open(os.path.join(ROOT, path), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest()[:16] != want:
                return None
    return t["dram_bytes_per_query"] * queries


def alu_peaks(pn) -> dict:
    """Measured arithmetic ceilings of this GPU, TFLOP/s: the library's FMA
    probes (FP32 scalar and packed two-wide, FP64) and cuBLAS TF32 (an 8192^3
    float32 matmul with TF32 tensor cores allowed, best of 5, CUDA events)."""
    import torch
    out = {"fp32_fma": pn.alu_peak(0), "fp32x2_fma": pn.alu_peak(1), "fp64_fma": pn.alu_peak(2)}
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(8192, 8192, device="cuda")
        b = torch.randn(8192, 8192, device="cuda")
        best = None
        for _ in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        out["tf32_cublas"] = 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12
        del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    out["fp32"] = max(out["fp32_fma"], out["fp32x2_fma"])
    out["how"] = ("FP32/FP64: panache_alu_peak (8 FMA chains per thread, 8 blocks of 256 per SM, ~50 ms); "
                  "TF32: torch.matmul 8192^3 float32 with allow_tf32 (cuBLAS), best of 5")
    return {k: (round(v, 2) if isinstance(v, float) else v) for k, v in out.items()}


def kernel_table(st: dict, kt: dict, n: int, anchors: list[int], peaks: dict, alu: dict, w: int = 8) -> list[dict]:
    """Per-kernel roofline: algorithmic flops and bytes of each kernel for one
    request, its CUDA-event time (library per-kernel timer, the last timed
    step), and both fractions.  Per-unit costs (unit: window-anchor unless
    stated):
      k_anchor_tc   3 TF32 MMAs of 2 a 32 flop per chunk of 256 windows; reads
                    the a samples of each chunk start (8 B each) and writes a
                    128 B anchor row per chunk
      k_features    1,650 flop (15 bins x 8 flop of complex update, 30
                    normalisations, 25 projections x 30 FMAs); 164 B (128 B row,
                    4 B key, 4 B sieve projection written; 8 B moments, 4 B run
                    length, 16 B of samples read)
      k_search      per inspected candidate a 30-wide bound (90 flop) and its
                    128 B row; per query its own 128 B row; per survivor an
                    exact distance of 5 flop per sample (normalise, subtract,
                    multiply-add) at the mean anchor length
      sieve eval    5 flop per sample per evaluated pair; each member's window
                    (4 B per sample) once per band of w pairs (the exact pairs
                    counted include the top-k sieve's, a few percent)
      k_complete    3 flop per sample per box triple (its windows are
                    normalised once in shared memory); bytes: per seed (1,053
                    triples) the two runs of m + 2 dm + 2 dp samples its box
                    covers, 8 B each
      selection     three passes of 8 B per profile cell (two histogram
                    passes, the pool pass) per selection call; flops negligible
      refine        4 flop per sample per scanned partner (normalise,
                    subtract, multiply-add); its samples (8 B) come from L1/L2
                    shared by the 256 partners of a block, so 8 m B per 256
    """
    L = 51
    a_mean = sum(anchors) / len(anchors)
    nwa = sum(n - a + 1 for a in anchors)
    q, c, e = st["queries"], st["candidates"], st["exact_stream"]
    es, ec, rounds = st["exact_sieve"], st["exact_completion"], st["completion_rounds"]
    chunks = sum((n - a + 1 + 255) // 256 for a in anchors)
    m_mean = 125.0
    rows = {
        "anchor_tc": (3.0 * 2 * a_mean * 32 * chunks, chunks * (8.0 * a_mean + 128.0), "tf32"),
        "features": (1650.0 * nwa, 164.0 * nwa, "fp32"),
        "search": (90.0 * c + 5.0 * a_mean * e, 128.0 * (q + c), "fp32"),
        "sieve": (5.0 * a_mean * es, 4.0 * a_mean * es / w, "fp32"),
        "complete": (3.0 * m_mean * ec, (ec / 1053.0) * 2 * (m_mean + 2 * 6 + 2 * 4) * 8.0, "fp32"),
        "select": (0.0, 24.0 * L * n * (rounds + 1 + st.get("refine_passes", 0)), "fp32"),
        "refine": (4.0 * m_mean * st.get("exact_refine", 0), 8.0 * m_mean * st.get("exact_refine", 0) / 256.0,
                   "fp32"),
    }
    out = []
    for name, (fl, by, pipe) in rows.items():
        ms, launches = kt.get(name, (0.0, 0))
        if ms <= 0:
            continue
        tf = fl / (ms * 1e-3) / 1e12
        gbs = by / (ms * 1e-3) / 1e9
        peak_c = alu["tf32_cublas"] if pipe == "tf32" else alu["fp32"]
        sig = lambda v: float(f"{v:.4g}")                          # noqa: E731  (4 significant digits)
        out.append({"kernel": name, "launches": launches, "ms": round(ms, 3), "flops": fl, "bytes": by,
                    "tflops": sig(tf), "gbs": sig(gbs),
                    ("tf32_frac" if pipe == "tf32" else "fp32_frac"): sig(tf / peak_c),
                    "hbm_frac": sig(gbs / peaks["hbm_gbs"])})
    ms, launches = kt.get("topk_sieve", (0.0, 0))
    if ms > 0:
        # the focused top-k sieve after the emit stage: its work is the kept
        # tiles' FP16 Gram blocks, which the request counters do not give;
        # time only (its profile summary has the counters)
        out.append({"kernel": "topk_sieve", "launches": launches, "ms": round(ms, 3),
                    "note": "FP16 Gram blocks of the pivot-kept tiles plus the pivot pre-pass; issue-bound"})
    return out


def roofline(stats_steps: list[dict], peaks: dict, peak_src: str, traffic: float | None):
    """Roofline of the dominant kernel, from the library's per-step CUDA events.

    The streaming search is one kernel launch per request.  Its algorithmic
    bytes per query window: the query's feature row (128 B) plus 128 B per
    inspected candidate row -- the Parseval test reads every candidate's
    30-float row once (the per-query figure of the search step).
    """
    ms = [s["step_ms"]["search"] for s in stats_steps]
    feat_ms = [s["step_ms"]["features"] for s in stats_steps]
    st = stats_steps[-1]
    bytes_search = 128.0 * (st["queries"] + st["candidates"])
    avg = statistics.mean(ms) / 1e3
    ach = bytes_search / avg / 1e9
    out = {"kernel": "k_search (streaming search: probe, Parseval rejection, exact distance)",
           "bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": traffic,
           "peak_source": f"{peak_src} (HBM copy GB/s)",
           "bytes_per_launch": bytes_search, "avg_launch_ms": round(statistics.mean(ms), 3),
           "features_avg_ms": round(statistics.mean(feat_ms), 3)}
    return out


def paper_recovery(ref, got) -> dict:
    """Top-k recovery as the paper's evaluation scores it (Sec. 4).

    ref and got are motif lists (fields m, i, d).  A reference cell is a
    position match when some reported cell at the same length starts within
    m/2 of it; otherwise a value match when the best reported distance at
    that length is within 5% relative or 0.05 absolute of its distance;
    otherwise missed.
    """
    best, starts = {}, {}
    for r in got:
        m = int(r["m"])
        best[m] = min(best.get(m, float("inf")), float(r["d"]))
        starts.setdefault(m, []).append(int(r["i"]))
    pos = val = 0
    for r in ref:
        m, i, d = int(r["m"]), int(r["i"]), float(r["d"])
        if any(2 * abs(j - i) <= m for j in starts.get(m, ())):
            pos += 1
        elif m in best and (abs(best[m] - d) <= 0.05 * d or abs(best[m] - d) <= 0.05):
            val += 1
    return {"position": pos, "value": val, "missed": len(ref) - pos - val, "of": len(ref)}


def cpu_baseline(x: np.ndarray, lengths=(100, 125, 150), excl=150, target_s=12.0):
    """The oracle (tier ii, all host cores) on a bounded prefix sample at three lengths.

    A 20k-sample probe sizes the sample so the timed oracle run takes about
    target_s seconds on this host (the oracle's cost grows as n^2).
    """
    from oracle import exact

    def once(n_sample):
        xs = np.asarray(x[:n_sample], dtype=np.float64)
        t = time.perf_counter()
        for m in lengths:
            exact.pmp(xs, m, m, excl, tier="diag")
        return time.perf_counter() - t

    t0 = once(20_000)
    n_sample = int(min(len(x), 300_000, max(20_000, 20_000 * (target_s / max(t0, 1e-3)) ** 0.5)))
    dt = once(n_sample)
    w = sum(n_sample - m + 1 for m in lengths)
    return {"value": w / dt, "unit": UNIT, "cores": exact.max_threads(), "kind": "oracle",
            "seconds": round(dt, 2),
            "sample": f"tier-ii exact PMP (per-diagonal FP64 sliding dot products) of the first {n_sample} "
                      f"samples at lengths {list(lengths)}; its cost grows as n^2, so on the full "
                      f"{len(x)}-sample series the oracle's rate would be about {n_sample / len(x):.3f}x this"}


def run_batched(pn, stream, n_series: int, n_loop: int, n_graph: int = 256):
    """The batched form: the first n_series series of the batched workload
    (4096 log-uniform lengths in [2000, 200000], per-series length intervals,
    top-10, exclusion m_max) in one pmp_batch call from host buffers (waves
    under the HBM budget), timed once after a warm-up on 64 of them; the
    first n_loop series run one pmp call at a time; the first n_graph series
    with the index and search steps replayed from a captured CUDA graph; and
    64 small series of one shape one call each, eager and replayed."""
    import torch
    from paper_2607_17481_b300 import shard
    t_gen = time.perf_counter()
    series = workloads.batched_workload(4096, seed=0, indices=range(n_series))
    t_gen = time.perf_counter() - t_gen
    params = [(q.m_min, q.m_max, q.k, q.excl) for q in series]
    hosts = [q.x for q in series]
    W = sum(workloads.windows_lengths(len(q.x), q.m_min, q.m_max) for q in series)
    # chunk length and search grid from the autotuner (cached per shape class)
    from paper_2607_17481_b300 import autotune
    t_tune = time.perf_counter()
    tuned = autotune.config_for_batch(hosts, params, sample=64)
    t_tune = time.perf_counter() - t_tune
    ctx = pn.Context(precision=1, topk_mode=pn.TOPK_GLOBAL, flags=pn.FLAG_TIMING, chunk=tuned["chunk"],
                     grid_mult=tuned["grid_mult"])
    ctx.set_stream(stream.cuda_stream)

    def run_all(xs, ps, c):
        # every rank runs its shard of the batch (no collective on the data path)
        return shard.run_sharded(xs, ps, lambda s_, p_: c.pmp_batch(s_, p_))

    run_all(hosts[:64], params[:64], ctx)                      # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_all(hosts, params, ctx)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0)
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    st = ctx.stats()
    out = {"series": n_series, "samples": int(sum(len(q.x) for q in series)), "windows_lengths": W,
           "value": W / (ms / 1e3), "unit": UNIT, "ms_per_batch": ms, "inputs": "host buffers (H2D inside)",
           "generation_s": round(t_gen, 1), "waves": st["waves"], "kernel_launches": st["kernel_launches"],
           "autotuned": {"chunk": tuned["chunk"], "grid_mult": tuned["grid_mult"], "tuning_s": round(t_tune, 1),
                         "search_ms_by_grid_mult": tuned["search_ms"],
                         "drift_by_chunk": {str(k): v for k, v in tuned["drift"].items()}},
           "workload": "batched_workload(4096, seed=0)[:n]: random walk / ECG-like / sine mix, 0-5 planted "
                       "motifs, lengths m_min~U{16..128} with 20-64 lengths, top-10, excl=m_max"}
    xs = [torch.from_numpy(q.x).cuda() for q in series[:max(n_loop, n_graph)]]
    if n_loop > 0:
        sub = list(range(min(n_loop, n_series)))
        Wl = sum(workloads.windows_lengths(len(series[i].x), series[i].m_min, series[i].m_max) for i in sub)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in sub:
            ctx.pmp(xs[i], *params[i])
        e1.record(stream)
        e1.synchronize()
        out["one_at_a_time"] = {"series": len(sub), "value": Wl / (e0.elapsed_time(e1) / 1e3), "unit": UNIT}
    if n_graph > 0:
        ng = min(n_graph, n_series)
        Wg = sum(workloads.windows_lengths(len(series[i].x), series[i].m_min, series[i].m_max) for i in range(ng))
        res = {}
        for name, flags in (("eager", 0), ("graph", pn.FLAG_GRAPH)):
            c = pn.Context(precision=1, topk_mode=pn.TOPK_GLOBAL, flags=flags, chunk=tuned["chunk"],
                           grid_mult=tuned["grid_mult"])
            c.set_stream(stream.cuda_stream)
            run_all(xs[:ng], params[:ng], c)                   # capture (graph) / warm-up
            gt = []
            for _ in range(2):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                run_all(xs[:ng], params[:ng], c)
                torch.cuda.synchronize()
                gt.append(1e3 * (time.perf_counter() - t0))
            res[name] = {"value": Wg / (statistics.mean(gt) / 1e3), "ms_per_batch": statistics.mean(gt)}
        out["device_inputs_first"] = {"series": ng, "unit": UNIT, **res}
    # many small series of one shape, one call each: eager launches vs graph replay
    fleet = [workloads.random_walk(np.random.default_rng([77, i]), 8192) for i in range(64)]
    fl = [torch.from_numpy(f).cuda() for f in fleet]
    Wf = len(fl) * workloads.windows_lengths(8192, 32, 64)
    res = {}
    for name, flags in (("eager", 0), ("graph", pn.FLAG_GRAPH)):
        c = pn.Context(precision=1, topk_mode=pn.TOPK_GLOBAL, flags=flags)
        c.set_stream(stream.cuda_stream)
        c.pmp(fl[0], 32, 64, 20, 64)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for f in fl:
            c.pmp(f, 32, 64, 20, 64)
        torch.cuda.synchronize()
        res[name] = Wf / (time.perf_counter() - t0)
    out["fleet_8192"] = {"series": len(fl), "n": 8192, "lengths": "32..64", "unit": UNIT,
                         "eager_value": res["eager"], "graph_value": res["graph"]}
    return out


def run_walk(pn, stream):
    """The small exact case: the planted random walk (n = 8,192 float64, 3
    planted pairs, lengths 32..64, exclusion 64), top-20 per length (660
    motifs) and over the whole stack, both precision forms, per call with the
    series resident on the device.  Per-length mode runs at the library's
    default anchor stride for that mode (1) and, for comparison, at the
    paper's 2."""
    import torch
    s = workloads.planted_random_walk()
    x = torch.from_numpy(s.x).cuda()
    W = workloads.windows_lengths(len(s.x), s.m_min, s.m_max)
    out = {"n": len(s.x), "lengths": f"{s.m_min}..{s.m_max}", "k": s.k, "excl": s.excl, "unit": UNIT}
    for name, over in (("per_length_mixed", dict(precision=1, topk_mode=pn.TOPK_PER_LENGTH)),
                       ("per_length_plain", dict(precision=0, topk_mode=pn.TOPK_PER_LENGTH)),
                       ("per_length_mixed_stride2", dict(precision=1, topk_mode=pn.TOPK_PER_LENGTH, stride=2)),
                       ("global_mixed", dict(precision=1, topk_mode=pn.TOPK_GLOBAL)),
                       ("global_plain", dict(precision=0, topk_mode=pn.TOPK_GLOBAL))):
        c = pn.Context(**over)
        c.set_stream(stream.cuda_stream)
        for _ in range(3):
            got = c.pmp(x, s.m_min, s.m_max, s.k, s.excl)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(10):
            got = c.pmp(x, s.m_min, s.m_max, s.k, s.excl)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / 10
        out[name] = {"ms": round(ms, 3), "value": W / (ms / 1e3), "motifs": int(len(got))}
    return out


def run_served(pn, args, rate=None):
    """The served form: Poisson arrivals of batched-workload series plus live
    streams (random walk or ECG-like, starting at 50,000 samples, lengths
    64..128, top-20, exclusion 128) receiving 1,024-sample appends at 50 Hz,
    each stream asked for its top-20 once a second; one request server with
    4 slots under a 120 GB budget and a request deadline (submissions whose
    predicted wait exceeds it are refused, EBUSY).  Appends and snapshots are
    queued and applied by the server's stream workers.  Latency: submission
    to motifs on the host (requests), call to motifs on the host
    (snapshots)."""
    import numpy as np
    rate = args.served_rate if rate is None else rate
    rng = np.random.default_rng(99)
    n_req = int(rate * args.served_seconds * 1.3) + 8
    reqs = workloads.batched_workload(n_req, seed=5)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    arrivals = arrivals[arrivals < args.served_seconds]
    live = []
    for sidx in range(args.served_streams):
        g = np.random.default_rng([123, sidx])
        kind = "random_walk" if sidx % 2 == 0 else "ecg_like"
        total = 50_000 + 1024 * int(50 * args.served_seconds + 2)
        x = workloads.random_walk(g, total) if kind == "random_walk" else workloads.ecg_like(g, total)
        live.append(x.astype(np.float32))
    sv = pn.Server(slots=4, hbm_budget_bytes=120 * 10 ** 9, precision=1, topk_mode=pn.TOPK_GLOBAL,
                   flags=pn.FLAG_HALF_FEATURES if args.served_half else 0)
    # live streams reserve their resident state from the budget; one that
    # does not fit is refused (EBUDGET) and left out, and a stream whose
    # growth is refused keeps its samples and stops taking appends
    sids, kept, refused, opened_refused = [], [], 0, 0
    for x in live:
        sid = sv.stream_open(64, 128, 20, 128)
        try:
            sv.append(sid, x[:50_000])
        except pn.PanacheError:
            opened_refused += 1
            sv.stream_close(sid)
            continue
        sids.append(sid)
        kept.append(x)
    live = kept
    for sid in sids:                                   # the initial index of every stream is built
        sv.wait(sv.stream_topk(sid))
    sv.set_deadline(args.served_deadline_ms)
    growing = [True] * len(live)
    tickets, busy = [], 0
    t0 = time.perf_counter()
    next_req, tick = 0, 0
    fed = [50_000] * len(live)
    while True:
        now = time.perf_counter() - t0
        if now >= args.served_seconds:
            break
        while next_req < len(arrivals) and arrivals[next_req] <= now:
            q = reqs[next_req]
            try:
                tickets.append(sv.submit(q.x, q.m_min, q.m_max, q.k, q.excl))
            except pn.PanacheError as e:
                if e.code != pn.native.EBUSY:
                    raise
                busy += 1
            next_req += 1
        if now >= tick * 0.02:                     # 50 Hz append round
            for i, sid in enumerate(sids):
                if not growing[i]:
                    continue
                try:
                    sv.append(sid, live[i][fed[i]:fed[i] + 1024])
                    fed[i] += 1024
                except pn.PanacheError:
                    growing[i] = False
                    refused += 1
            if tick % 50 == 49:                    # once a second: top-20 of every live stream
                for sid in sids:
                    try:
                        tickets.append(sv.stream_topk(sid))
                    except pn.PanacheError as e:
                        if e.code != pn.native.EBUSY:
                            raise
            tick += 1
        time.sleep(0.0005)
    sv.set_deadline(0.0)                           # the final snapshots are always served
    tickets.extend(sv.stream_topk(sid) for sid in sids)
    failures = {}
    for t in tickets:
        try:
            sv.wait(t)
        except pn.PanacheError as e:
            failures[e.code] = failures.get(e.code, 0) + 1
    st = sv.stats()
    sv.close()
    return {"requests": int(next_req), "admitted": int(next_req - busy), "refused_by_deadline": busy,
            "deadline_ms": args.served_deadline_ms,
            "stream_topk_requests": int(len(tickets) - next_req + busy),
            "live_streams": len(live), "live_streams_requested": args.served_streams,
            "live_streams_refused_at_open": opened_refused,
            "stream_appends_refused": refused, "refused_snapshots": int(st["refused_snapshots"]),
            "failures_by_code": {str(k): v for k, v in failures.items()},
            "feature_rows": "half" if args.served_half else "fp32",
            "appended_samples": int(sum(f - 50_000 for f in fed)),
            "arrival_rate_per_s": rate, "window_s": args.served_seconds,
            "completed": int(st["completed"]), "failed": int(st["failed"]),
            "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
            "snapshot_p50_ms": st["snap_p50_ms"], "snapshot_p99_ms": st["snap_p99_ms"],
            "windows_lengths": int(st["windows_lengths"]),
            "sustained_value": st["windows_lengths"] / (st["span_ms"] / 1e3) if st["span_ms"] else None,
            "unit": UNIT, "batches": int(st["batches"]), "max_concurrent_batches": int(st["max_concurrent_batches"]),
            "peak_reserved_bytes": int(st["peak_reserved_bytes"]), "budget_bytes": int(st["budget_bytes"]),
            "note": "stream top-k requests process each stream's samples received so far; p50/p99 are of "
                    "admitted requests"}


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, each step a bounded sample of the workload."""
    rank, world, _ = rank_env()
    if rank != 0:
        return 0
    s = workloads.wafer_like(WORKLOAD["n"], seed=WORKLOAD["seed"])
    times = []
    w = 0
    n_sample = 50_000
    lengths = (100, 125, 150)
    from oracle import exact
    xs = np.asarray(s.x[:n_sample], dtype=np.float64)
    for step in range(args.warmup + args.steps):
        t = time.perf_counter()
        for m in lengths:
            exact.pmp(xs, m, m, WORKLOAD["excl"], tier="diag")
        dt = time.perf_counter() - t
        if step >= args.warmup:
            times.append(dt)
    w = sum(n_sample - m + 1 for m in lengths)
    value = w / statistics.mean(times)
    sample = (f"tier-ii exact PMP of the first {n_sample} samples at lengths {list(lengths)} per step "
              f"(oracle, FP64, all host cores)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, sample=sample),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": exact.max_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="panache", choices=("panache", "reference"))
    ap.add_argument("--precision", type=int, default=1, help="1 mixed (default), 0 plain FP64")
    ap.add_argument("--plain-steps", type=int, default=1, help="timed steps of the plain FP64 form")
    ap.add_argument("--half-steps", type=int, default=2, help="timed steps with half-precision feature rows")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--batched", type=int, default=4096,
                    help="series of the batched workload timed as one pmp_batch (0: skip)")
    ap.add_argument("--served-seconds", type=float, default=2.0, help="arrival window of the served leg (0: skip)")
    ap.add_argument("--served-rate", type=float, default=200.0, help="Poisson request arrivals per second")
    ap.add_argument("--served-streams", type=int, default=256, help="live streams")
    ap.add_argument("--served-fp32", dest="served_half", action="store_false",
                    help="served leg with FP32 feature rows (default: half-precision rows)")
    ap.add_argument("--served-deadline-ms", type=float, default=1000.0,
                    help="server deadline: requests predicted to wait longer are refused (0: off)")
    ap.add_argument("--batched-loop", type=int, default=64,
                    help="series of the same batch timed one pmp call at a time (0: skip)")
    ap.add_argument("--n", type=int, default=WORKLOAD["n"])
    ap.add_argument("--fast-steps", type=int, default=1,
                    help="timed steps of the paper's fastest settings (s=6, alpha=4, one completion round; "
                         "K=4, s=8), 0: skip")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = rank_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import paper_2607_17481_b300 as pn
    wl = dict(WORKLOAD, n=args.n)
    s = workloads.wafer_like(wl["n"], seed=wl["seed"] + rank)
    x_host = torch.from_numpy(s.x).pin_memory()
    x_dev = x_host.cuda()
    W = workloads.windows_lengths(wl["n"], wl["m_min"], wl["m_max"])
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def make_ctx(precision, **over):
        over = dict(over)
        flags = pn.FLAG_TIMING | over.pop("flags", 0)
        ctx = pn.Context(precision=precision, topk_mode=pn.TOPK_GLOBAL, flags=flags, **over)
        ctx.set_stream(stream.cuda_stream)
        return ctx

    def timed(ctx, steps, warm, src, kts=None):
        for _ in range(warm):
            ctx.pmp(src, wl["m_min"], wl["m_max"], wl["k"], wl["excl"])
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ms, stats, motifs = [], [], None
        for _ in range(steps):
            flush.fill_(1.0)                      # L2 flush between steps (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            motifs = ctx.pmp(src, wl["m_min"], wl["m_max"], wl["k"], wl["excl"])
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            stats.append(ctx.stats())
            if kts is not None:
                kts.append(ctx.kernel_times())
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        return ms, stats, motifs

    ctx = make_ctx(args.precision)
    kts = []
    with ClockSampler(local) as clk:
        ms, stats, motifs = timed(ctx, args.steps, args.warmup, x_dev, kts)
    clocks = clk.summary()
    # end to end through the C ABI with host buffers: the H2D copy of the series
    # and the D2H copy of the motifs happen inside every call
    e2e_ms = ms if args.no_e2e else timed(ctx, max(2, args.steps // 2), 1, x_host.numpy())[0]
    total = sum(ms) / 1e3
    if dist:
        t = torch.tensor([total], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    value = W * world * args.steps / total
    e2e_value = W * world / (statistics.mean(e2e_ms) / 1e3)

    plain = None
    if args.plain_steps > 0 and args.precision != 0:
        pctx = make_ctx(0)
        pms, pstats, pmot = timed(pctx, args.plain_steps, 1, x_dev)
        plain_mot = pmot
        plain = {"value": W * world / (statistics.mean(pms) / 1e3), "ms_per_step": statistics.mean(pms),
                 "same_motifs": bool(np.array_equal(pmot[["m", "i", "j"]], motifs[["m", "i", "j"]])),
                 "step_ms": pstats[-1]["step_ms"]}
    half = None
    if args.half_steps > 0 and args.precision != 0:
        hctx = make_ctx(args.precision, flags=pn.FLAG_HALF_FEATURES)
        hms, hst, hmot = timed(hctx, args.half_steps, 1, x_dev)
        half = {"value": W * world / (statistics.mean(hms) / 1e3), "ms_per_step": statistics.mean(hms),
                "same_motifs": bool(np.array_equal(hmot[["m", "i", "j"]], motifs[["m", "i", "j"]])),
                "device_bytes": int(hst[-1]["device_bytes"]),
                "device_bytes_fp32_rows": int(stats[-1]["device_bytes"]),
                "exact_distances": int(hst[-1]["exact_stream"]),
                "exact_distances_fp32_rows": int(stats[-1]["exact_stream"]), "step_ms": hst[-1]["step_ms"]}
    fast = None
    if args.fast_steps > 0:
        fast = {}
        for name, over in (("s6_alpha4_rounds1", dict(stride=6, alpha=4, rounds=1)),
                           ("topk_sieve", dict(flags=pn.FLAG_TOPK_SIEVE)),
                           ("no_focus_sieve", dict(flags=pn.FLAG_NO_FOCUS_SIEVE)),
                           ("K4_s8", dict(K=4, stride=8))):
            fctx = make_ctx(args.precision, **over)
            fms, fst, fmot = timed(fctx, args.fast_steps, 1, x_dev)
            ref_cells = {(int(r["m"]), int(r["i"]), int(r["j"])) for r in motifs}
            got_cells = {(int(r["m"]), int(r["i"]), int(r["j"])) for r in fmot}
            over = {k: v for k, v in over.items() if k != "flags"} | ({name: True} if "flags" in over else {})
            fast[name] = {"value": W * world / (statistics.mean(fms) / 1e3), "ms_per_step": statistics.mean(fms),
                          "same_motifs": bool(np.array_equal(fmot[["m", "i", "j"]], motifs[["m", "i", "j"]])),
                          "recall_vs_default": len(ref_cells & got_cells) / max(1, len(ref_cells)),
                          "best_d": float(fmot["d"][0]) if len(fmot) else None,
                          "kth_d": float(fmot["d"][-1]) if len(fmot) else None,
                          "config": over}
            if name == "topk_sieve":
                # every pair of every hot class estimated on the tensor cores
                # (the dense exhaustive sieve's motifs in the tests): the
                # default's cells it also reports, and both lists' k-th distances
                fast[name]["default_recall_vs_this"] = fast[name]["recall_vs_default"]
                fast[name]["default_kth_d"] = float(motifs["d"][-1]) if len(motifs) else None
                # the default's list scored against this one by the paper's recovery rule
                fast[name]["default_recovery_sec4"] = paper_recovery(fmot, motifs)
                topk_mot = fmot
            if name == "no_focus_sieve" and plain is not None:
                # the plain FP64 form has no focused sieve (it needs the FP16
                # Gram blocks): its lists against the mixed form's without it
                plain["same_motifs_as_mixed_without_focus"] = bool(
                    np.array_equal(plain_mot[["m", "i", "j"]], fmot[["m", "i", "j"]]))
            if name == "no_focus_sieve" and "topk_sieve" in fast:
                # without the default's focused sieve: its cells against the whole
                # top-k sieve's, by identity and by the paper's rule
                tc = {(int(r["m"]), int(r["i"]), int(r["j"])) for r in topk_mot}
                fast[name]["recall_vs_topk_sieve"] = len(tc & got_cells) / max(1, len(tc))
                fast[name]["recovery_sec4_vs_topk_sieve"] = paper_recovery(topk_mot, fmot)
    walk = run_walk(pn, stream) if rank == 0 else None
    batched = run_batched(pn, stream, args.batched, args.batched_loop) if args.batched > 0 else None
    served = run_served(pn, args) if args.served_seconds > 0 and rank == 0 else None
    # the same mix at a quarter of the arrival rate: latency when the server is not saturated
    served_light = run_served(pn, args, args.served_rate / 4) if args.served_seconds > 0 and rank == 0 else None
    if rank != 0:
        return 0
    peaks, psrc = measured_peaks()
    alu = alu_peaks(pn)
    anchors = list(range(wl["m_min"], wl["m_max"] + 1, STRIDE))
    if anchors[-1] != wl["m_max"]:
        anchors.append(wl["m_max"])
    rl = roofline(stats, peaks, psrc, measured_traffic(stats[-1]["queries"]))
    rl["kernels"] = kernel_table(stats[-1], kts[-1], wl["n"], anchors, peaks, alu)
    rl["alu_peaks_tflops"] = alu
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 recurrence/bound/in-stream distance, f64 prefix sums/anchors/verification"
        if args.precision else "f64",
        "data": "synthetic",
        "config": dict(wl, form="mixed" if args.precision else "plain_fp64", l2="flushed between steps",
                       replicas=world),
        "latency_ms": {"p50": float(np.percentile(ms, 50)), "p99": float(np.percentile(ms, 99))},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(s.x.nbytes),
                "d2h_bytes_per_step": int(len(motifs) * 32)},
        "gpu_launches": int(sum(st["kernel_launches"] for st in stats)),
        "roofline": rl,
        "clocks": clocks,
        "plain_fp64": plain,
        "half_feature_rows": half,
        "fast_settings": fast,
        "planted_walk": walk,
        "batched": batched,
        "served": served,
        "served_quarter_rate": served_light,
        "step_ms": stats[-1]["step_ms"],
        "counters": {k: v for k, v in stats[-1].items() if k != "step_ms"},
        "motifs": [[int(r["m"]), int(r["i"]), int(r["j"]), float(r["d"])] for r in motifs],
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s.x)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
