"""Failure paths, with every failure made on the host (no GPU is faulted).

* A device allocation of a request's state refused (ENOMEM), the upload of
  its samples refused (ECUDA), and the tensor-core anchor kernel's bounded
  waits run out (ETIMEOUT: the kernel issues no MMA, gives up after a few
  tries, records the timeout and frees its tensor memory): each call fails
  with its code, and the same context then serves the next request with the
  result of an untouched context.
* A request server's wait with a 1 ms limit on a request that takes far
  longer returns ETIMEOUT; the ticket stays valid and a later wait returns
  the result, equal to the single-context result.
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
    yield pkg
    pkg.inject_fault(pkg.native.FAULT_NONE)


@pytest.fixture(scope="module")
def walk():
    return workloads.planted_random_walk()


@pytest.fixture(scope="module")
def expected(pn, walk):
    s = walk
    return pn.Context(precision=1, topk_mode=0).pmp(s.x, s.m_min, s.m_max, s.k, s.excl)


def _same(a, b):
    assert np.array_equal(a[["m", "i", "j"]], b[["m", "i", "j"]])
    assert np.array_equal(a["d"], b["d"])


@pytest.mark.parametrize("kind,after,code", [("FAULT_ALLOC", 0, "ENOMEM"), ("FAULT_ALLOC", 7, "ENOMEM"),
                                             ("FAULT_COPY", 0, "ECUDA"), ("FAULT_TC_WAIT", 0, "ETIMEOUT")])
def test_failure_then_recovery(pn, walk, expected, kind, after, code):
    from paper_2607_17481_b300 import native
    s = walk
    ctx = pn.Context(precision=1, topk_mode=0)
    first = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)        # the context has served a request
    _same(first, expected)
    pn.inject_fault(getattr(native, kind), after)
    with pytest.raises(pn.PanacheError) as ei:
        ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    assert ei.value.code == getattr(native, code)
    again = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)        # the hook disarmed itself
    _same(again, expected)


def test_fault_hook_does_not_fire_for_other_kinds(pn, walk, expected):
    """An armed copy fault leaves device-resident input alone (no upload)."""
    from paper_2607_17481_b300 import native
    s = walk
    x = torch.from_numpy(s.x).cuda()
    ctx = pn.Context(precision=1, topk_mode=0)
    pn.inject_fault(native.FAULT_COPY, 0)
    try:
        _same(ctx.pmp(x, s.m_min, s.m_max, s.k, s.excl), expected)
    finally:
        pn.inject_fault(native.FAULT_NONE)


def test_server_wait_times_out_then_delivers(pn):
    from paper_2607_17481_b300 import native
    w = workloads.wafer_like(2_000_000, seed=4)
    sv = pn.Server(slots=1, precision=1, topk_mode=0)
    try:
        t = sv.submit(w.x, 100, 150, 20, 150)
        with pytest.raises(pn.PanacheError) as ei:
            sv.wait(t, timeout_ms=1)
        assert ei.value.code == native.ETIMEOUT
        got, lat = sv.wait(t)
        assert lat > 1.0
    finally:
        sv.close()
    ref = pn.Context(precision=1, topk_mode=0).pmp(w.x, 100, 150, 20, 150)
    _same(got, ref)
