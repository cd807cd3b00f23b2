"""Writes the oracle's top-10 lists for a seeded subset of the batched
workload (batched_workload(4096, seed=0)): eight series covering the three
generators, series of 10k-58k samples, length intervals from 18..42 up to
122..172, one series with n >= 50,000 and several with m_min >= 100.  Each
list is the global top-10 (the workload's top-k, exclusion m_max) and the
top-10 of every length.  The oracle's wall time per series (tier ii, FP64,
all host cores) is recorded as the timed CPU baseline on this subset.

Calls only the oracle (tier ii exact PMP, FP64) and the seeded generator:
  python tests/golden/make_batched_subset.py    (a few minutes on 8 cores)
Output: tests/golden/batched_subset_top10.json, entries [m, i, j, d].
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import exact, topk  # noqa: E402

INDICES = [12, 21, 6, 17, 5, 24, 200, 356]


def main():
    out = {"workload": "batched_workload(4096, seed=0)", "oracle": "tier ii exact PMP, FP64",
           "cores": exact.max_threads(), "series": []}
    for s, q in zip(INDICES, workloads.batched_workload(4096, seed=0, indices=INDICES)):
        x = np.asarray(q.x, dtype=np.float64)
        t0 = time.perf_counter()
        P, I = exact.pmp(x, q.m_min, q.m_max, q.excl, tier="diag")
        dt = time.perf_counter() - t0
        out["series"].append({
            "index": s, "kind": q.kind, "n": int(x.shape[0]), "m_min": q.m_min, "m_max": q.m_max, "k": q.k,
            "excl": q.excl, "oracle_seconds": round(dt, 2),
            "windows_lengths": workloads.windows_lengths(x.shape[0], q.m_min, q.m_max),
            "global": [list(t) for t in topk.select(P, I, q.m_min, q.k, topk.GLOBAL)],
            "per_length": [list(t) for t in topk.select(P, I, q.m_min, q.k, topk.PER_LENGTH)]})
        print(s, q.kind, x.shape[0], q.m_min, q.m_max, f"{dt:.1f} s", flush=True)
    with open(os.path.join(HERE, "batched_subset_top10.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
