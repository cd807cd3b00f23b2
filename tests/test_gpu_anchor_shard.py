"""Anchor sharding of one series (Sec. 3.5: anchors share no state), with the
ranks emulated one after another on one GPU: each "rank" indexes, searches
and sieves its share of the anchors, the rows merge by the elementwise
unsigned minimum, and the emit stage on the merged rows reports exactly the
motifs of the unsharded call."""
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


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision,mode", [(1, 0), (0, 0), (1, 1)])
def test_sharded_equals_single(pn, world, precision, mode):
    from paper_2607_17481_b300 import shard
    s = workloads.planted_random_walk()
    # the focused top-k sieve needs the request's own directories, which a
    # call on rows handed in from the ranks does not have: compared without it
    ctx = pn.Context(precision=precision, topk_mode=mode, flags=pn.FLAG_NO_FOCUS_SIEVE)
    want = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    stride = 1 if mode == 1 else 2
    parts = []
    for r in range(world):
        rows = ctx.pmp_anchor_shard(s.x, s.m_min, s.m_max, s.k, s.excl, r, world)
        mine = set(shard.anchor_positions(s.m_min, s.m_max, stride, r, world))
        for m in range(s.m_min, s.m_max + 1):
            if m not in mine:                           # only the rank's own anchor rows are written
                assert np.all(rows[m - s.m_min] == np.uint64(shard.EMPTY_KEY)), (r, m)
        parts.append(rows)
    merged = parts[0]
    for p in parts[1:]:
        merged = np.minimum(merged, p)
    got = ctx.pmp_from_rows(s.x, s.m_min, s.m_max, s.k, s.excl, merged)
    assert np.array_equal(got, want)


def test_shard_arguments(pn):
    s = workloads.planted_random_walk()
    ctx = pn.Context()
    for r, w in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(pn.PanacheError):
            ctx.pmp_anchor_shard(s.x, s.m_min, s.m_max, s.k, s.excl, r, w)
