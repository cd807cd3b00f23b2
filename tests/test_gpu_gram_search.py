"""The tensor-core Gram search (opt-in) against the per-query Parseval search.

Both searches admit the same pairs (each query's budgeted list) and
evaluate exactly, with the same FP32 arithmetic, every admitted pair that
can still lower one of its cells; the Gram search only decides differently
which pairs those are.  So the profile rows must be equal bit for bit, right
after the search (emit stages off) and after the whole emit stage, and the
motifs equal.  Covered: float64 and float32 series, FP32 and half feature
rows, global and per-length modes, strides 1 and 2, the wafer-like prefix,
the batched form and a live stream.
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


@pytest.fixture(scope="module")
def walk():
    return workloads.planted_random_walk()


@pytest.fixture(scope="module")
def wafer():
    return workloads.wafer_like(200_000, seed=0)


def _both(pn, x, m_min, m_max, k, excl, flags=0, **cfg):
    out = []
    for extra in (pn.FLAG_GRAM_SEARCH, 0):
        ctx = pn.Context(precision=1, flags=flags | extra, **cfg)
        mot = ctx.pmp(x, m_min, m_max, k, excl)
        rows = ctx.profile_rows(0, len(x), m_max - m_min + 1)
        out.append((mot, rows, ctx.stats()))
    return out


def _search_only(pn):
    return pn.FLAG_NO_SIEVE | pn.FLAG_NO_COMPLETION | pn.FLAG_NO_REFINE


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("stride", [1, 2])
def test_search_rows_equal(pn, walk, dtype, stride):
    s = walk
    x = s.x.astype(dtype)
    (mg, rg, sg), (mp, rp, sp) = _both(pn, x, s.m_min, s.m_max, s.k, s.excl, flags=_search_only(pn),
                                       topk_mode=1, stride=stride)
    assert np.array_equal(rg, rp)
    assert np.array_equal(mg, mp)
    assert sg["queries"] == sp["queries"] and sg["candidates"] == sp["candidates"]
    print(f"exact distances: gram {sg['exact_stream']} vs parseval {sp['exact_stream']}")


@pytest.mark.parametrize("mode", [0, 1])
def test_full_request_equal(pn, walk, mode):
    s = walk
    (mg, rg, _), (mp, rp, _) = _both(pn, s.x, s.m_min, s.m_max, s.k, s.excl, topk_mode=mode)
    assert np.array_equal(rg, rp)
    assert np.array_equal(mg, mp)


def test_half_rows_equal(pn, walk):
    s = walk
    (mg, rg, _), (mp, rp, _) = _both(pn, s.x, s.m_min, s.m_max, s.k, s.excl,
                                     flags=_search_only(pn) | pn.FLAG_HALF_FEATURES, topk_mode=1, stride=2)
    assert np.array_equal(rg, rp)
    assert np.array_equal(mg, mp)


def test_wafer_prefix_equal(pn, wafer):
    w = wafer
    x = w.x.astype(np.float32)
    (mg, rg, sg), (mp, rp, sp) = _both(pn, x, 100, 150, 20, 150, flags=_search_only(pn), topk_mode=0)
    assert np.array_equal(rg, rp)
    assert np.array_equal(mg, mp)
    print(f"wafer 200k exact distances: gram {sg['exact_stream']} vs parseval {sp['exact_stream']}")


def test_batched_equal(pn):
    b = workloads.batched_workload(12, seed=3, n_hi=20000)
    series = [s.x for s in b]
    params = [(s.m_min, s.m_max, s.k, s.excl) for s in b]
    res = []
    for extra in (pn.FLAG_GRAM_SEARCH, 0):
        ctx = pn.Context(precision=1, topk_mode=1, flags=extra)
        res.append(ctx.pmp_batch(series, params))
    for ra, rb in zip(*res):
        assert np.array_equal(ra, rb)


def test_stream_equal(pn, walk):
    s = walk
    tops = []
    for extra in (pn.FLAG_GRAM_SEARCH, 0):
        ctx = pn.Context(precision=1, topk_mode=0, flags=extra)
        st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
        for lo in range(0, len(s.x), 1500):
            st.append(s.x[lo:lo + 1500])
        tops.append(st.topk())
        st.close()
    assert np.array_equal(tops[0], tops[1])
