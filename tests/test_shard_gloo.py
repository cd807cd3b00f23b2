"""Multi-rank batched form on CPU (gloo, world size 2): sharding, gathering, failure detection.

No GPU is used: the per-rank compute is a stand-in that returns a
deterministic summary of each series, so the test checks the host logic
(assignment, gather order) and that a failing rank is detected by the others
through the process group's timeout instead of hanging.
"""
import datetime
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2607_17481_b300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _series():
    rng = np.random.default_rng(0)
    xs = [rng.standard_normal(int(n)) for n in rng.integers(200, 3000, size=11)]
    params = [(16, 16 + int(L), 5, 16 + int(L)) for L in rng.integers(4, 30, size=11)]
    return xs, params


def _stand_in(xs, params):
    return [(len(x), round(float(np.sum(x)), 9), p) for x, p in zip(xs, params)]


def _worker(rank, world, port, mode, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=8))
    xs, params = _series()
    try:
        if mode == "fail" and rank == 1:
            raise RuntimeError("injected failure on rank 1")
        res = shard.run_sharded(xs, params, _stand_in)
        out.put((rank, "ok", res))
    except Exception as e:  # noqa: BLE001
        out.put((rank, "error", repr(e)))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:  # noqa: BLE001
            pass


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    return {r: (status, payload) for r, status, payload in got}


def test_assignment_is_balanced_and_deterministic():
    costs = [100, 90, 80, 10, 10, 10, 5]
    a = shard.assign(costs, 2)
    assert sorted(a[0] + a[1]) == list(range(7))
    loads = [sum(costs[i] for i in part) for part in a]
    assert max(loads) - min(loads) <= max(costs)
    assert a == shard.assign(costs, 2)
    assert shard.assign([], 3) == [[], [], []]


def test_two_ranks_gather_every_result_in_order():
    res = _run("ok")
    xs, params = _series()
    ref = _stand_in(xs, params)
    for r in (0, 1):
        status, payload = res[r]
        assert status == "ok"
        assert payload == ref


def test_failing_rank_is_detected():
    res = _run("fail")
    assert res[1][0] == "error" and "injected" in res[1][1]
    # rank 0 does not hang: its gather ends with an error when rank 1 never joins
    assert res[0][0] == "error"


# ---- anchor sharding of one series -------------------------------------------------

def _pack(d, j):
    """Packed profile key: the FP64 bits of d with the low 26 bits replaced by j."""
    b = np.asarray(d, dtype=np.float64).view(np.uint64) & ~np.uint64((1 << 26) - 1)
    return b | np.asarray(j, dtype=np.uint64)


def _anchor_stand_in(rank, world, m_min=20, m_max=31, stride=2, n=400):
    """Per-rank rows of a stand-in compute: rank r fills the rows of its own
    anchor lengths with seeded keys, every other row is empty."""
    L = m_max - m_min + 1
    rows = np.full((L, n), np.uint64(shard.EMPTY_KEY), dtype=np.uint64)
    for a in shard.anchor_positions(m_min, m_max, stride, rank, world):
        g = np.random.default_rng([7, a])
        d = g.uniform(0.0, 3.0, size=n)
        j = g.integers(0, n, size=n)
        keep = g.random(n) < 0.8                       # some cells stay empty
        rows[a - m_min][keep] = _pack(d[keep], j[keep])
    return rows


def _anchor_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=30))
    try:
        merged = shard.run_anchor_sharded(lambda r, w: _anchor_stand_in(r, w), lambda rows: rows)
        out.put((rank, "ok", merged))
    except Exception as e:  # noqa: BLE001
        out.put((rank, "error", repr(e)))
    finally:
        dist.destroy_process_group()


def test_anchor_positions_partition_the_anchor_set():
    for (m_min, m_max, s) in ((100, 150, 2), (32, 64, 2), (20, 31, 3), (16, 16, 2)):
        full = shard.anchor_positions(m_min, m_max, s, 0, 1)
        assert full[0] == m_min and full[-1] == m_max
        for world in (1, 2, 3, 5):
            parts = [shard.anchor_positions(m_min, m_max, s, r, world) for r in range(world)]
            assert sorted(a for p in parts for a in p) == full


def test_merge_rows_is_the_unsigned_minimum():
    """Single process (no group): unchanged.  The reduction's key mapping keeps
    the unsigned order, with the empty key largest."""
    a = np.array([shard.EMPTY_KEY, 5, _pack(0.5, 3), _pack(0.0, 7)], dtype=np.uint64)
    assert np.array_equal(shard.merge_rows(a), a)
    s = a.view(np.int64).copy()
    s[a == np.uint64(shard.EMPTY_KEY)] = np.iinfo(np.int64).max
    assert list(np.argsort(s, kind="stable")) == list(np.argsort(a, kind="stable"))


def test_two_ranks_merge_anchor_rows():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_anchor_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {r: (st, payload) for r, st, payload in [q.get(timeout=120) for _ in procs]}
    for p in procs:
        p.join(timeout=60)
    want = np.minimum(_anchor_stand_in(0, 2), _anchor_stand_in(1, 2))
    single = _anchor_stand_in(0, 1)                       # one rank owning every anchor
    assert np.array_equal(want, single)
    for r in (0, 1):
        assert got[r][0] == "ok", got[r]
        assert np.array_equal(got[r][1], want)
