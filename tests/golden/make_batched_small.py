"""Writes the oracle's global top-10 for every series of the batched
workload (batched_workload(4096, seed=0)) with at most 12,000 samples and
m_min <= 24: short series at the workload's shortest lengths, where the
directory's hot classes hold many near-copy windows and the band of sieve
neighbours alone can leave the closest pairs of a class unevaluated.

Calls only the oracle (tier ii exact PMP, FP64) and the seeded generator:
  python tests/golden/make_batched_small.py    (a few minutes on 8 cores)
Output: tests/golden/batched_small_top10.json, entries [m, i, j, d].
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import exact, topk  # noqa: E402

N_MAX, M_MIN_MAX = 12000, 24


def main():
    series = workloads.batched_workload(4096, seed=0)
    picked = [i for i, q in enumerate(series) if len(q.x) <= N_MAX and q.m_min <= M_MIN_MAX]
    out = {"workload": "batched_workload(4096, seed=0)", "rule": f"every series with n <= {N_MAX} and m_min <= {M_MIN_MAX}",
           "oracle": "tier ii exact PMP, FP64", "series": []}
    for i in picked:
        q = series[i]
        x = np.asarray(q.x, dtype=np.float64)
        P, I = exact.pmp(x, q.m_min, q.m_max, q.excl, tier="diag")
        out["series"].append({"index": i, "kind": q.kind, "n": int(x.shape[0]), "m_min": q.m_min, "m_max": q.m_max,
                              "k": q.k, "excl": q.excl,
                              "global": [list(t) for t in topk.select(P, I, q.m_min, q.k, topk.GLOBAL)]})
    with open(os.path.join(HERE, "batched_small_top10.json"), "w") as f:
        json.dump(out, f)
    print(len(picked), "series")


if __name__ == "__main__":
    main()
