"""Writes the oracle's top-20 lists for the 200,000-sample prefix of the
1,000,000-sample wafer-like series (seed 0), lengths 100..150, exclusion 150.

Calls only the oracle (tier ii exact PMP, FP64) and the seeded generator:
  python tests/golden/make_wafer_prefix.py      (about 10 minutes on 8 cores)
Output: tests/golden/wafer200k_top20.json with the global top-20 and the
top-20 of every length, each entry [m, i, j, d].
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import workloads  # noqa: E402
from oracle import exact, topk  # noqa: E402

N_PREFIX, M_MIN, M_MAX, EXCL, K = 200_000, 100, 150, 150, 20


def main():
    s = workloads.wafer_like(1_000_000, seed=0)
    x = np.asarray(s.x[:N_PREFIX], dtype=np.float64)
    P, I = exact.pmp(x, M_MIN, M_MAX, EXCL, tier="diag")
    out = {"series": "wafer_like(1_000_000, seed=0)[:200_000]", "m_min": M_MIN, "m_max": M_MAX,
           "excl": EXCL, "k": K, "oracle": "tier ii exact PMP, FP64",
           "global": [list(t) for t in topk.select(P, I, M_MIN, K, topk.GLOBAL)],
           "per_length": [list(t) for t in topk.select(P, I, M_MIN, K, topk.PER_LENGTH)]}
    with open(os.path.join(HERE, "wafer200k_top20.json"), "w") as f:
        json.dump(out, f)


if __name__ == "__main__":
    main()
