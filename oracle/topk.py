"""Zero-snap and top-k pan-motif selection (test infrastructure only).

Sec. 2: a pan-motif is a low cell of the profile stack with its neighbour;
the top-k list sorts cells by distance and skips any cell within m/2 of an
already accepted cell of the same length.  Sec. 3.6 / Algorithm 2: distances
below eps0 = 1e-6 are reported as exactly zero before the selection.

Readings (where the paper is silent):
* "within m/2" is the integer test 2*|i - i'| <= m;
* equal distances are ordered by (m, i) ascending;
* GLOBAL mode ranks all cells of the stack together; PER_LENGTH mode applies
  the same rule to each length separately and concatenates the lists in
  ascending m.
"""
from __future__ import annotations

import numpy as np

EPS0 = 1e-6
GLOBAL = 0
PER_LENGTH = 1


def zero_snap(P: np.ndarray, eps0: float = EPS0) -> np.ndarray:
    out = np.array(P, dtype=np.float64, copy=True)
    out[out < eps0] = 0.0
    return out


def _greedy(cells_d, cells_m, cells_i, k):
    order = np.lexsort((cells_i, cells_m, cells_d))
    accepted: dict[int, list[int]] = {}
    picked = []
    for t in order:
        m = int(cells_m[t])
        i = int(cells_i[t])
        if any(2 * abs(i - a) <= m for a in accepted.get(m, ())):
            continue
        accepted.setdefault(m, []).append(i)
        picked.append(t)
        if len(picked) == k:
            break
    return picked


def select(P: np.ndarray, I: np.ndarray, m_min: int, k: int, mode: int = GLOBAL,
           eps0: float = EPS0):
    """Top-k motifs from profile rows P[L][n], I[L][n].

    Returns a list of (m, i, j, d) tuples in selection order.
    """
    Ps = zero_snap(P, eps0)
    L = Ps.shape[0]
    out = []
    if mode == GLOBAL:
        ms, iis = np.nonzero(np.isfinite(Ps))
        d = Ps[ms, iis]
        for t in _greedy(d, ms + m_min, iis, k):
            out.append((int(ms[t] + m_min), int(iis[t]), int(I[ms[t], iis[t]]), float(d[t])))
    else:
        for r in range(L):
            iis = np.nonzero(np.isfinite(Ps[r]))[0]
            d = Ps[r, iis]
            mm = np.full(iis.shape, r + m_min)
            for t in _greedy(d, mm, iis, k):
                out.append((int(r + m_min), int(iis[t]), int(I[r, iis[t]]), float(d[t])))
    return out
