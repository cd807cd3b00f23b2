"""The request server: continuous batching, admission by HBM footprint, live streams.

Results must not depend on which requests share a batch or run alongside
(each result the same alone and in the mix); the parity tolerance here is
zero: motifs are compared bit for bit.
"""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_17481_b300 as pkg
    from paper_2607_17481_b300 import build
    build.build()
    return pkg


def _series(count, seed, n_hi=30000):
    return workloads.batched_workload(count, seed=seed, n_hi=n_hi)


def test_alone_equals_mix(pn):
    reqs = _series(12, seed=11)
    alone = []
    with_one = pn.Server(slots=1)
    for q in reqs:
        t = with_one.submit(q.x, q.m_min, q.m_max, q.k, q.excl)
        alone.append(with_one.wait(t)[0])
    with_one.close()
    mix = pn.Server(slots=3)
    noise = _series(20, seed=12)
    tickets = []
    for a, b in zip(noise[:12], reqs):               # interleave with unrelated requests
        mix.submit(a.x, a.m_min, a.m_max, a.k, a.excl)
        tickets.append(mix.submit(b.x, b.m_min, b.m_max, b.k, b.excl))
    for t, ref in zip(tickets, alone):
        got, lat = mix.wait(t)
        assert np.array_equal(got, ref)
        assert lat > 0
    st = mix.stats()
    assert st["completed"] >= 24 and st["failed"] == 0
    mix.close()


def test_server_matches_context(pn):
    q = _series(1, seed=3)[0]
    ctx = pn.Context()
    ref = ctx.pmp(q.x, q.m_min, q.m_max, q.k, q.excl)
    sv = pn.Server(slots=2)
    got, _ = sv.wait(sv.submit(q.x, q.m_min, q.m_max, q.k, q.excl))
    assert np.array_equal(got, ref)
    sv.close()


def test_admission_budget(pn):
    reqs = _series(6, seed=21, n_hi=20000)
    ctx = pn.Context()
    ctx.pmp(reqs[0].x, reqs[0].m_min, reqs[0].m_max, reqs[0].k, reqs[0].excl)
    one = ctx.stats()["device_bytes"]
    # a budget below one request refuses it at submission
    tiny = pn.Server(slots=2, hbm_budget_bytes=max(1, one // 4))
    with pytest.raises(pn.PanacheError) as e:
        tiny.submit(reqs[0].x, reqs[0].m_min, reqs[0].m_max, reqs[0].k, reqs[0].excl)
    assert e.value.code == -3
    tiny.close()
    # a budget that fits about one request at a time serialises the slots; nothing is lost
    big = max(one, max(_footprint(pn, q) for q in reqs))
    tight = pn.Server(slots=4, hbm_budget_bytes=int(big * 1.3))
    ts = [tight.submit(q.x, q.m_min, q.m_max, q.k, q.excl) for q in reqs]
    for t in ts:
        tight.wait(t)
    st = tight.stats()
    assert st["completed"] == 6 and st["peak_reserved_bytes"] <= st["budget_bytes"]
    tight.close()


def _footprint(pn, q):
    ctx = pn.Context()
    ctx.pmp(q.x, q.m_min, q.m_max, q.k, q.excl)
    return ctx.stats()["device_bytes"]


def test_live_stream_topk_equals_offline(pn):
    s = workloads.planted_random_walk()
    sv = pn.Server(slots=2, topk_mode=1)
    sid = sv.stream_open(s.m_min, s.m_max, s.k, s.excl)
    rng = np.random.default_rng(7)
    pos = 0
    mid_ticket = None
    while pos < s.x.shape[0]:
        step = int(rng.integers(1, 2500))
        sv.append(sid, s.x[pos:pos + step])
        pos += step
        if mid_ticket is None and pos > 4000:
            mid_ticket, mid_len = sv.stream_topk(sid), pos   # snapshot while appends continue
    final, _ = sv.wait(sv.stream_topk(sid))
    ctx = pn.Context(topk_mode=1)
    assert np.array_equal(final, ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl))
    snap, _ = sv.wait(mid_ticket)
    assert np.array_equal(snap, ctx.pmp(s.x[:mid_len], s.m_min, s.m_max, s.k, s.excl))
    sv.close()


def test_request_that_cannot_fit_beside_streams_is_refused(pn):
    """Live streams hold their reservation; a request that no longer fits
    beside them while nothing else runs is refused, not left waiting."""
    s = workloads.planted_random_walk()
    big = _series(1, seed=31, n_hi=60000)[0]
    need = _footprint(pn, big)
    stream_probe = pn.Server(slots=1, hbm_budget_bytes=10 << 30)
    sid = stream_probe.stream_open(s.m_min, s.m_max, s.k, s.excl)
    stream_probe.append(sid, s.x)
    res = stream_probe.stats()["peak_reserved_bytes"]         # the stream's reservation
    stream_probe.close()
    assert 0 < res
    # a budget that holds the stream, and the request alone, but not both
    budget = max(need, res) + min(need, res) // 2
    sv = pn.Server(slots=2, hbm_budget_bytes=budget)
    sid = sv.stream_open(s.m_min, s.m_max, s.k, s.excl)
    sv.append(sid, s.x)
    t = sv.submit(big.x, big.m_min, big.m_max, big.k, big.excl)
    with pytest.raises(pn.PanacheError) as e:
        sv.wait(t, timeout_ms=60_000)
    assert e.value.code == -3
    # once the stream is closed the same request runs
    sv.stream_close(sid)
    got, _ = sv.wait(sv.submit(big.x, big.m_min, big.m_max, big.k, big.excl), timeout_ms=60_000)
    assert len(got) > 0
    sv.close()


def test_deadline_sheds_load(pn):
    """With a deadline, a submission whose predicted wait (queued work over the
    measured throughput) exceeds it is refused with EBUSY and counted; with
    the deadline off the same request is admitted and served."""
    reqs = _series(3, seed=41)
    sv = pn.Server(slots=1)
    q0, q1 = reqs[0], reqs[1]
    sv.wait(sv.submit(q0.x, q0.m_min, q0.m_max, q0.k, q0.excl))    # a throughput estimate exists
    sv.set_deadline(1e-6)
    with pytest.raises(pn.PanacheError) as e:
        sv.submit(q1.x, q1.m_min, q1.m_max, q1.k, q1.excl)
    assert e.value.code == pn.native.EBUSY
    assert sv.stats()["refused"] == 1
    sv.set_deadline(0.0)
    got, _ = sv.wait(sv.submit(q1.x, q1.m_min, q1.m_max, q1.k, q1.excl))
    assert np.array_equal(got, pn.Context().pmp(q1.x, q1.m_min, q1.m_max, q1.k, q1.excl))
    sv.close()


def test_many_small_appends_coalesce(pn):
    """Hundreds of small appends queued faster than they are applied: the
    stream workers apply runs of them as one append; snapshots taken in
    between see exactly the samples accepted before them."""
    s = workloads.planted_random_walk()
    sv = pn.Server(slots=1, topk_mode=0)
    sid = sv.stream_open(s.m_min, s.m_max, s.k, s.excl)
    snaps = []
    for pos in range(0, s.x.shape[0], 37):
        sv.append(sid, s.x[pos:pos + 37])
        if pos in (2997, 5994):
            snaps.append((sv.stream_topk(sid), min(pos + 37, s.x.shape[0])))
    snaps.append((sv.stream_topk(sid), s.x.shape[0]))
    ctx = pn.Context(topk_mode=0)
    for t, n in snaps:
        got, lat = sv.wait(t)
        assert np.array_equal(got, ctx.pmp(s.x[:n], s.m_min, s.m_max, s.k, s.excl)), n
    st = sv.stats()
    assert st["snap_p50_ms"] > 0
    sv.stream_close(sid)
    sv.close()
