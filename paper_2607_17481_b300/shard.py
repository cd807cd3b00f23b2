"""Sharding of a batched request across ranks (one process per GPU).

The series of a batch are independent problems, so they split across ranks
with no data-path collective: each rank runs its own shard through the
library (one pmp_batch), and only the finished motif lists are gathered.
The assignment balances the estimated work n * L greedily (largest first),
deterministically, so every rank derives the same plan on its own.
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
