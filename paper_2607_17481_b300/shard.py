"""Sharding across ranks (one process per GPU).

Batched requests: the series of a batch are independent problems, so they
split across ranks with no data-path collective: each rank runs its own
shard through the library (one pmp_batch), and only the finished motif lists
are gathered.  The assignment balances the estimated work n * L greedily
(largest first), deterministically, so every rank derives the same plan on
its own.

One series: its anchors are independent (Sec. 3.5), so rank r indexes,
searches and sieves the anchors at positions p = r mod world of the anchor
set (panache_pmp_anchor_shard); the ranks' profile rows merge by the
elementwise minimum of their packed keys (the one exchange), and every rank
runs the emit stage on the merged rows with the whole series present
(panache_pmp_from_rows).
"""
from __future__ import annotations

import heapq


def work(n: int, m_min: int, m_max: int) -> int:
    """Windows x lengths of one series: the unit the work scales with."""
    return sum(max(0, n - m + 1) for m in range(m_min, m_max + 1))


def assign(costs: list[int], world: int) -> list[list[int]]:
    """Indices of the series each rank runs (largest first onto the least loaded rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda t: (-costs[t], t)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + costs[i], r))
    for r in range(world):
        out[r].sort()
    return out


def run_sharded(series: list, params: list[tuple[int, int, int, int]], run_fn, group=None):
    """Runs this rank's shard with run_fn(series_subset, params_subset) -> results, then gathers.

    Returns every series' result in the original order (on every rank).
    Without an initialised process group it runs everything locally.
    """
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return list(run_fn(series, params))
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    costs = [work(len(x), mn, mx) for x, (mn, mx, _, _) in zip(series, params)]
    mine = assign(costs, world)[rank]
    local = list(run_fn([series[i] for i in mine], [params[i] for i in mine])) if mine else []
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, local), group=group)
    out = [None] * len(series)
    for idx, res in gathered:
        for i, r in zip(idx, res):
            out[i] = r
    return out


EMPTY_KEY = 0xFFFFFFFFFFFFFFFF


def anchor_positions(m_min: int, m_max: int, stride: int, rank: int, world: int) -> list[int]:
    """Anchor lengths rank `rank` of `world` owns: positions p of
    A = (m_min, m_min + s, ..., m_max) with p mod world == rank."""
    a = list(range(m_min, m_max + 1, stride))
    if a[-1] != m_max:
        a.append(m_max)
    return [x for p, x in enumerate(a) if p % world == rank]


def merge_rows(rows, group=None):
    """Elementwise minimum of the ranks' packed profile keys (unsigned 64-bit).

    Keys of non-negative distances have a clear top bit, so as signed 64-bit
    integers they keep their order; the empty key (all ones) is mapped to
    the largest signed value for the reduction and back afterwards.  Without
    an initialised process group the rows are returned unchanged.
    """
    import numpy as np
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(rows, dtype=np.uint64)
    if not (dist.is_available() and dist.is_initialized()):
        return a.copy()
    signed = a.view(np.int64).copy()
    empty = a == np.uint64(EMPTY_KEY)
    signed[empty] = np.iinfo(np.int64).max
    t = torch.from_numpy(signed)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    out = t.numpy().copy()
    back = out == np.iinfo(np.int64).max
    res = out.view(np.uint64)
    res[back] = np.uint64(EMPTY_KEY)
    return res


def run_anchor_sharded(shard_fn, emit_fn, group=None):
    """shard_fn(rank, world) -> this rank's rows; the merged rows go to emit_fn(rows) -> motifs."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        world, rank = dist.get_world_size(group), dist.get_rank(group)
    else:
        world, rank = 1, 0
    mine = shard_fn(rank, world)
    return emit_fn(merge_rows(mine, group))
