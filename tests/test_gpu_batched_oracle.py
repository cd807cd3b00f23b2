"""The batched and served forms against the oracle on the batched workload itself.

Eight series of batched_workload(4096, seed=0) -- all three generators,
10k to 58k samples, one series of 53k samples at lengths 18..42 and one of
57k at 100..126, several intervals with m_min >= 100 -- with the oracle's
global top-10 and per-length top-10 frozen in
tests/golden/batched_subset_top10.json (tier ii exact PMP, FP64, written by
tests/golden/make_batched_subset.py).  Bar: every oracle (m, i, j) is
reported (exact ties accepted either way), distances within 1e-6 relative.

* batched: the eight series in one pmp_batch call, global and per-length top-10;
* served: the eight series submitted to a request server at once (two
  slots, continuous batching), and three of them fed to the server as live
  streams in uneven appends, each snapshot's top-10 against the oracle.
"""
import json
import os

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "batched_subset_top10.json")
SMALL = os.path.join(os.path.dirname(__file__), "golden", "batched_small_top10.json")


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_17481_b300 as pkg
    from paper_2607_17481_b300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def subset():
    with open(GOLDEN) as f:
        g = json.load(f)
    idx = [e["index"] for e in g["series"]]
    series = workloads.batched_workload(4096, seed=0, indices=idx)
    for q, e in zip(series, g["series"]):
        assert (len(q.x), q.m_min, q.m_max, q.k, q.excl) == (e["n"], e["m_min"], e["m_max"], e["k"], e["excl"])
    return series, g["series"]


def _check(q, got, ref):
    from parity import compare
    r = compare(q.x.astype(np.float64), got, [tuple(t) for t in ref])
    assert r["misses"] == 0, (q.kind, len(q.x), q.m_min, q.m_max, r["miss_list"])
    assert r["bad_dist"] == 0


def test_golden_subset_shape(subset):
    series, gold = subset
    assert any(len(q.x) >= 50_000 for q in series)
    assert sum(q.m_min >= 100 for q in series) >= 3
    assert {q.kind for q in series} == {"random_walk", "ecg_like", "sine_mix"}


def test_batched_matches_oracle(pn, subset):
    """The workload's own top-k (global top-10): exact for every series."""
    series, gold = subset
    ctx = pn.Context(precision=1, topk_mode=0)
    got = ctx.pmp_batch([q.x for q in series], [(q.m_min, q.m_max, q.k, q.excl) for q in series])
    for q, g, e in zip(series, got, gold):
        _check(q, g, e["global"])


def test_batched_per_length_recall(pn, subset):
    """Per-length top-10 of every series (2,440 cells), reported: the 53k
    ECG-like series at lengths 18..42 loses one pair at length 18 that no
    anchor's search brings up and that is not among the refined top cells of
    its length; everything else is exact."""
    from parity import compare
    series, gold = subset
    ctx = pn.Context(precision=1, topk_mode=1)
    got = ctx.pmp_batch([q.x for q in series], [(q.m_min, q.m_max, q.k, q.excl) for q in series])
    misses = total = 0
    for q, g, e in zip(series, got, gold):
        r = compare(q.x.astype(np.float64), g, [tuple(t) for t in e["per_length"]])
        assert r["bad_dist"] == 0
        misses += r["misses"]
        total += r["n"]
        if r["misses"]:
            print("per-length misses:", q.kind, len(q.x), q.m_min, q.m_max, r["miss_list"])
    print(f"batched per-length recall: {(total - misses) / total:.5f} of {total}")
    assert misses <= 0.002 * total


def test_served_matches_oracle(pn, subset):
    series, gold = subset
    sv = pn.Server(slots=2, precision=1, topk_mode=0)
    try:
        tickets = [sv.submit(q.x, q.m_min, q.m_max, q.k, q.excl) for q in series]
        # three series also arrive as live streams, in uneven appends
        live = [0, 2, 5]
        sids = []
        for li in live:
            q = series[li]
            sid = sv.stream_open(q.m_min, q.m_max, q.k, q.excl)
            cuts = [0, 1000, 1777, 5000, len(q.x) - 3333, len(q.x)]
            for a, b in zip(cuts[:-1], cuts[1:]):
                sv.append(sid, q.x[a:b])
            sids.append(sid)
        snap = [sv.stream_topk(sid) for sid in sids]
        for q, e, t in zip(series, gold, tickets):
            got, _ = sv.wait(t)
            _check(q, got, e["global"])
        for li, t in zip(live, snap):
            got, _ = sv.wait(t)
            _check(series[li], got, gold[li]["global"])
        for sid in sids:
            sv.stream_close(sid)
    finally:
        sv.close()


def test_batched_short_series_match_oracle(pn):
    """Every series of the workload with n <= 12,000 and m_min <= 24 (145
    series): global top-10 against the oracle
    (tests/golden/batched_small_top10.json, written by make_batched_small.py),
    in one pmp_batch call at the defaults, which include the focused top-k
    sieve, and without it.  Measured: 12 of 1,450 cells missed, in six
    series (pairs at lengths 16..26 that neither an anchor's search nor a hot
    class brings up); 36 in 18 series without the focused sieve.  Bar:
    recall >= 0.99 and fewer misses than without the sieve."""
    from parity import compare
    with open(SMALL) as f:
        gold = json.load(f)["series"]
    series = workloads.batched_workload(4096, seed=0, indices=[e["index"] for e in gold])
    params = [(q.m_min, q.m_max, q.k, q.excl) for q in series]
    got = pn.Context(precision=1, topk_mode=0).pmp_batch([q.x for q in series], params)
    off = pn.Context(precision=1, topk_mode=0, flags=pn.FLAG_NO_FOCUS_SIEVE).pmp_batch([q.x for q in series], params)
    misses = misses_off = total = 0
    for q, g, o, e in zip(series, got, off, gold):
        assert (len(q.x), q.m_min, q.m_max) == (e["n"], e["m_min"], e["m_max"])
        ref = [tuple(t) for t in e["global"]]
        r = compare(q.x.astype(np.float64), g, ref)
        assert r["bad_dist"] == 0
        misses += r["misses"]
        total += r["n"]
        if r["misses"]:
            print("short series misses:", e["index"], q.kind, len(q.x), q.m_min, q.m_max, r["miss_list"])
        ro = compare(q.x.astype(np.float64), o, ref)
        misses_off += ro["misses"]
        if ro["misses"]:
            print("  without the focused sieve:", e["index"], ro["misses"])
    print(f"short batched series: {misses} of {total} oracle cells missed ({misses_off} without the focused sieve)")
    assert misses <= 0.01 * total
    assert misses < misses_off
