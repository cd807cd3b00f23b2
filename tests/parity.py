"""Comparison of reported motifs with the oracle's top-k, aware of exact ties.

The oracle ranks cells by (d, m, i) and takes the lowest neighbour index
among equal distances (Sec. 2).  Where two results are equally correct --
a neighbour whose distance equals the oracle's to 1e-12 relative, or a
boundary cell whose distance ties the oracle's cell -- the comparison
accepts either, re-checks the reported distance against the oracle's FP64
definition, and counts it separately.
"""
from __future__ import annotations

from oracle import exact

TIE_RTOL = 1e-12


def compare(x, got, ref, dist_rtol=1e-6):
    """Returns dict(hits, ties, misses, bad_dist, n)."""
    gset = {(int(r["m"]), int(r["i"]), int(r["j"])): float(r["d"]) for r in got}
    gcell = {(int(r["m"]), int(r["i"])): (int(r["j"]), float(r["d"])) for r in got}
    ref_cells = {(m, i) for (m, i, _, _) in ref}
    extra = [(m, i, j, d) for (m, i), (j, d) in gcell.items() if (m, i) not in ref_cells]
    hits = ties = misses = bad = 0
    miss_list = []
    for (m, i, j, d) in ref:
        if (m, i, j) in gset:
            hits += 1
            if abs(gset[(m, i, j)] - d) > dist_rtol * d + 1e-12:
                bad += 1
            continue
        if (m, i) in gcell:
            j2, d2 = gcell[(m, i)]
            dj2 = exact.dist(x, m, i, j2)
            if abs(dj2 - d) <= TIE_RTOL * max(d, 1e-300) and abs(i - j2) >= 1:
                ties += 1
                continue
        if any(em == m and abs(exact.dist(x, em, ei, ej) - d) <= TIE_RTOL * max(d, 1e-300)
               for (em, ei, ej, _) in extra):
            ties += 1
            continue
        misses += 1
        miss_list.append((m, i, j, d))
    return dict(hits=hits, ties=ties, misses=misses, bad_dist=bad, n=len(ref), miss_list=miss_list)
