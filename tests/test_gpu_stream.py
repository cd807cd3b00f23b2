"""Resident streams: incremental appends against the offline path and the oracle.

A stream keeps its index on the device and searches, at each append, only
the queries whose batch the append completes (Algorithm 1 in stream order).
Every step is a function of the samples, so a snapshot after any sequence of
appends must equal the offline request on the same samples bit for bit, and
the offline request is pinned to the oracle by test_gpu_parity.py.
"""
import numpy as np
import pytest

import workloads
from oracle import exact, topk

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


@pytest.fixture(scope="module")
def small():
    return workloads.planted_random_walk()


def chunks(n, seed, lo=1, hi=1500):
    rng = np.random.default_rng(seed)
    pos = 0
    while pos < n:
        step = int(rng.integers(lo, hi))
        yield pos, min(n, pos + step)
        pos += step


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_snapshots_equal_offline_prefixes(pn, small, precision, mode):
    s = small
    ctx = pn.Context(topk_mode=mode, precision=precision)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    marks = {2500, 5200}
    for a, b in chunks(s.x.shape[0], 11):
        st.append(s.x[a:b])
        for mk in sorted(marks):
            if a < mk <= b:
                marks.discard(mk)
                snap = st.topk()
                assert np.array_equal(snap, ctx.pmp(s.x[:b], s.m_min, s.m_max, s.k, s.excl)), b
    assert len(st) == s.x.shape[0]
    final = st.topk()
    assert np.array_equal(final, ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl))
    # a second snapshot with no append in between is the same
    assert np.array_equal(st.topk(), final)
    st.close()


def test_half_feature_rows_stream_equals_offline(pn, small):
    """Half-precision rows in a resident stream: the rows grow with the stream
    like the FP32 rows, and the snapshot equals the offline request."""
    s = small
    ctx = pn.Context(topk_mode=0, precision=1, flags=pn.FLAG_HALF_FEATURES)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    for a, b in chunks(s.x.shape[0], 15, 200, 1500):
        st.append(s.x[a:b])
    assert np.array_equal(st.topk(), ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl))
    st.close()


def test_stream_matches_oracle_global(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    for a, b in chunks(s.x.shape[0], 12, 1, 700):
        st.append(s.x[a:b])
    got = st.topk()
    P, I = exact.pmp(s.x, s.m_min, s.m_max, s.excl, tier="diag")
    ref = topk.select(P, I, s.m_min, s.k, topk.GLOBAL)
    assert [(int(r["m"]), int(r["i"]), int(r["j"])) for r in got] == [(m, i, j) for (m, i, j, _) in ref]
    for r, (_, _, _, d) in zip(got, ref):
        assert abs(float(r["d"]) - d) <= 1e-6 * d + 1e-12


def test_appends_search_only_new_queries(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    st.append(s.x[:6000])
    full = ctx.stats()["queries"]
    n_anchor = len(range(s.m_min, s.m_max + 1, 2)) + (0 if (s.m_max - s.m_min) % 2 == 0 else 1)
    assert full > 0.9 * n_anchor * (6000 - s.m_max - s.excl)
    delta = 128
    st.append(s.x[6000:6000 + delta])
    q = ctx.stats()["queries"]
    # the append completes at most delta + one batch of queries per anchor
    assert 0 < q <= n_anchor * (delta + s.excl)
    st.close()


def test_float32_and_device_chunks(pn, small):
    s = small
    x32 = s.x.astype(np.float32)
    ctx = pn.Context(topk_mode=0)
    ref = ctx.pmp(x32, s.m_min, s.m_max, s.k, s.excl)
    host = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    dev = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    xd = torch.from_numpy(x32).cuda()
    for a, b in chunks(s.x.shape[0], 13, 200, 2000):
        host.append(x32[a:b])
        dev.append(xd[a:b])
    assert np.array_equal(host.topk(), ref)
    assert np.array_equal(dev.topk(), ref)


def test_short_and_empty_streams(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    assert len(st.topk()) == 0                       # no samples yet
    st.append(s.x[:20])                              # shorter than every length
    assert len(st.topk()) == 0
    st.append(s.x[20:90])                            # windows, but no valid pair yet
    assert len(st.topk()) == 0
    st.append(s.x[90:400])
    assert np.array_equal(st.topk(), ctx.pmp(s.x[:400], s.m_min, s.m_max, s.k, s.excl))


def test_server_stream_budget_and_close(pn, small):
    s = small
    sv = pn.Server(slots=1, hbm_budget_bytes=64 << 20, topk_mode=0)
    sid = sv.stream_open(s.m_min, s.m_max, s.k, s.excl)
    sv.append(sid, s.x[:4000])                       # fits the budget
    with pytest.raises(pn.PanacheError) as e:
        sv.append(sid, np.tile(s.x, 40))             # would grow the state past it
    assert e.value.code == -3
    got, _ = sv.wait(sv.stream_topk(sid))            # the stream kept its samples
    ctx = pn.Context(topk_mode=0)
    assert np.array_equal(got, ctx.pmp(s.x[:4000], s.m_min, s.m_max, s.k, s.excl))
    sv.stream_close(sid)
    sid2 = sv.stream_open(s.m_min, s.m_max, s.k, s.excl)
    sv.append(sid2, s.x[:4000])                      # the closed stream's reservation was released
    sv.close()


def test_checkpoint_resume(pn, small):
    s = small
    ctx = pn.Context(topk_mode=1)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    st.append(s.x[:3333])
    ck = st.checkpoint()
    assert np.array_equal(ck, s.x[:3333])
    # resume on another context, then both continue with the same appends
    ctx2 = pn.Context(topk_mode=1)
    st2 = ctx2.stream(s.m_min, s.m_max, s.k, s.excl)
    st2.append(ck)
    for a, b in chunks(s.x.shape[0] - 3333, 14, 100, 900):
        st.append(s.x[3333 + a:3333 + b])
        st2.append(s.x[3333 + a:3333 + b])
    assert np.array_equal(st.topk(), st2.topk())
    assert np.array_equal(st2.topk(), ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl))


def test_stream_survives_context_destruction(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    st = pn.Stream(ctx, s.m_min, s.m_max, s.k, s.excl)
    st.append(s.x[:1000])
    ctx.close()
    with pytest.raises(pn.PanacheError) as e:
        st.append(s.x[1000:1100])
    assert e.value.code == -6                        # ESTATE: the context's device state is gone
    st.close()


def test_stream_checkpoint_and_calibration_argument_errors(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    st.append(s.x[:500])
    lib = pn.native.lib()
    import ctypes
    n = ctypes.c_int64()
    buf = np.zeros(10)
    # a checkpoint buffer smaller than the stream: ETRUNC with the length needed
    rc = lib.panache_stream_checkpoint(st._h, buf.ctypes.data_as(ctypes.c_void_p), 10, ctypes.byref(n))
    assert rc == -5 and n.value == 500
    K = ctypes.c_int32()
    x = np.ascontiguousarray(s.x)
    # eta outside (0, 1], lengths below 3, m_max < m_min
    for eta, lo, hi in ((1.5, 32, 64), (-0.1, 32, 64), (0.85, 2, 64), (0.85, 40, 32)):
        rc = lib.panache_calibrate_width(ctx._h, x.ctypes.data_as(ctypes.c_void_p), pn.F64, len(x), lo, hi, eta,
                                         ctypes.byref(K), None, None)
        assert rc == -1, (eta, lo, hi)
    # a series shorter than every length: every window set is empty, K falls back to 16
    K2, e, c = ctx.calibrate_width(s.x[:20], 32, 64)
    assert K2 == 16 and np.all(e == 0) and np.all(c == 0)
