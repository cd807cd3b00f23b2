"""Pins of the exact-PMP oracle against things other than itself.

Definitions: Sec. 2 (z-normalised distance, validity, profile rows, top-k
rule); zero-snap from Sec. 3.6.
"""
import math

import numpy as np
import pytest

from oracle import exact, topk


def naive_dist(x, m, i, j):
    """Pure-Python z-normalised distance (Sec. 2), written independently."""
    a = [float(v) for v in x[i:i + m]]
    b = [float(v) for v in x[j:j + m]]
    ma, mb = sum(a) / m, sum(b) / m
    sa = math.sqrt(sum((v - ma) ** 2 for v in a) / m)
    sb = math.sqrt(sum((v - mb) ** 2 for v in b) / m)
    if max(a) == min(a) or max(b) == min(b):
        return math.inf
    return math.sqrt(sum(((u - ma) / sa - (v - mb) / sb) ** 2 for u, v in zip(a, b)))


def naive_pmp(x, m_min, m_max, excl):
    n = len(x)
    out = {}
    for m in range(m_min, m_max + 1):
        for i in range(n - m + 1):
            best, arg = math.inf, -1
            for j in range(n - m + 1):
                if abs(i - j) < excl:
                    continue
                d = naive_dist(x, m, i, j)
                if d < best:
                    best, arg = d, j
            out[(m, i)] = (best, arg)
    return out


@pytest.mark.parametrize("tier", ["direct", "diag"])
def test_brute_force_tiny(tier):
    rng = np.random.default_rng(7)
    x = np.cumsum(rng.standard_normal(64))
    P, I = exact.pmp(x, 5, 9, 4, tier=tier)
    ref = naive_pmp(x, 5, 9, 4)
    for (m, i), (d, j) in ref.items():
        assert I[m - 5, i] == j
        assert P[m - 5, i] == pytest.approx(d, rel=1e-9, abs=1e-12)
    # cells past the last window are empty
    assert np.all(np.isinf(P[4, 64 - 9 + 1:])) and np.all(I[4, 64 - 9 + 1:] == -1)


def test_closed_form_pearson():
    """d^2 = 2m(1 - rho) with rho from numpy's Pearson correlation (Sec. 2)."""
    rng = np.random.default_rng(3)
    x = np.cumsum(rng.standard_normal(500)) + 40.0
    for (m, i, j) in [(16, 0, 100), (50, 17, 300), (77, 200, 401), (5, 3, 9)]:
        rho = np.corrcoef(x[i:i + m], x[j:j + m])[0, 1]
        assert exact.dist(x, m, i, j) == pytest.approx(math.sqrt(max(0.0, 2 * m * (1 - rho))),
                                                       rel=1e-9)


def test_tiers_agree_small_cfg(cfg_small, cfg_small_exact):
    s = cfg_small
    P2, I2 = cfg_small_exact
    # tier i on a sub-range of lengths of the same series
    P1, I1 = exact.pmp(s.x[:3000], 40, 44, s.excl, tier="direct")
    P3, I3 = exact.pmp(s.x[:3000], 40, 44, s.excl, tier="diag")
    f = np.isfinite(P1)
    assert np.array_equal(f, np.isfinite(P3))
    assert np.max(np.abs(P1[f] - P3[f])) < 1e-8
    assert np.array_equal(I1, I3)
    assert P2.shape == (33, 8192)


def test_affine_invariance():
    rng = np.random.default_rng(11)
    x = np.cumsum(rng.standard_normal(400))
    P, I = exact.pmp(x, 10, 14, 8, tier="direct")
    Pa, Ia = exact.pmp(3.5 * x - 17.0, 10, 14, 8, tier="direct")
    f = np.isfinite(P)
    assert np.max(np.abs(P[f] - Pa[f])) < 1e-9
    assert np.mean(I == Ia) > 0.999


def test_time_reversal():
    """Reversing the series maps window i of length m to n - m - i."""
    rng = np.random.default_rng(5)
    x = np.cumsum(rng.standard_normal(300))
    n = x.shape[0]
    for (m, i, j) in [(12, 0, 50), (20, 100, 170), (31, 7, 260)]:
        assert exact.dist(x, m, i, j) == pytest.approx(
            exact.dist(x[::-1].copy(), m, n - m - i, n - m - j), rel=1e-10)


def test_zero_snap_and_lowest_index_ties():
    """Exact repeats (a tiled period) give d = 0; the neighbour is the lowest valid repeat."""
    rng = np.random.default_rng(2)
    p = 37
    base = rng.standard_normal(p)
    x = np.tile(base, 12)
    excl = 40
    P, I = exact.pmp(x, 20, 22, excl, tier="direct")
    n = x.shape[0]
    for r, m in enumerate(range(20, 23)):
        for i in range(n - m + 1):
            js = [j for j in range(i % p, n - m + 1, p) if abs(i - j) >= excl]
            assert I[r, i] == js[0]
            assert P[r, i] < 1e-6
    sel = topk.select(P, I, 20, 5, topk.GLOBAL)
    assert all(d == 0.0 for (_, _, _, d) in sel)
    # all distances tie at 0: the order is (m, i), with i at least m/2 apart
    assert [(m, i) for (m, i, _, _) in sel] == [(20, 0), (20, 11), (20, 22), (20, 33), (20, 44)]


def test_constant_windows_ignored():
    rng = np.random.default_rng(9)
    x = np.cumsum(rng.standard_normal(300))
    x[100:130] = 5.0
    P, I = exact.pmp(x, 8, 10, 6, tier="direct")
    Pd, Id = exact.pmp(x, 8, 10, 6, tier="diag")
    for r, m in enumerate(range(8, 11)):
        const = [i for i in range(300 - m + 1) if x[i:i + m].max() == x[i:i + m].min()]
        assert const and all(np.isinf(P[r, i]) and I[r, i] == -1 for i in const)
        assert not set(const) & set(I[r][I[r] >= 0].tolist())
    f = np.isfinite(P)
    assert np.array_equal(I, Id) and np.max(np.abs(P[f] - Pd[f])) < 1e-8


def test_cells_match_rows(cfg_small, cfg_small_exact):
    s = cfg_small
    P, I = cfg_small_exact
    rows = np.array([0, 5, 789, 1283, 4000, 8192 - 48])
    Pc, Ic = exact.pmp_cells(s.x, 48, s.excl, rows)
    assert np.allclose(Pc, P[48 - 32, rows], rtol=1e-9)
    assert np.array_equal(Ic, I[48 - 32, rows])


def test_planted_motifs_recovered(cfg_small, cfg_small_exact):
    """The planted pairs are the lowest cells at the planted length (Sec. 4 recovery rule)."""
    s = cfg_small
    P, I = cfg_small_exact
    sel = topk.select(P[48 - 32:48 - 32 + 1], I[48 - 32:48 - 32 + 1], 48, 6, topk.GLOBAL)
    found = {(min(i, j), max(i, j)) for (_, i, j, _) in sel}
    for pl in s.planted:
        a, b = pl.starts
        assert any(abs(i - a) <= 24 and abs(j - b) <= 24 for (i, j) in found), pl
    # planted distances are of the order of the planted noise, random-walk cells far above
    assert max(d for (_, _, _, d) in sel) < 1.5


def test_topk_rule_hand_cases():
    inf = math.inf
    # one length, m = 10: cells at i = 0..7
    P = np.array([[0.5, 0.4, 0.9, 0.3, 0.31, 0.2, inf, 0.25]])
    I = np.arange(8)[None, :] + 100
    # sorted: 5(0.2) 7(0.25) 3(0.3) 4(0.31) 1(0.4) 0(0.5) 2(0.9)
    # accept 5; 7: 2*2=4<=10 skip; 3: 4<=10 skip; ... everything within 5 of 5 -> only 5
    assert [(i, d) for (_, i, _, d) in topk.select(P, I, 10, 3)] == [(5, 0.2)]
    # m = 4: skip when 2|i-i'| <= 4, i.e. |i-i'| <= 2
    sel = topk.select(P, I, 4, 4)
    # 5 accepted; 7, 3, 4 within 2 of 5; 1 accepted; 0 and 2 within 1 of 1
    assert [i for (_, i, _, _) in sel] == [5, 1]
    # zero-snap makes tiny values exactly 0 and orders them by (m, i)
    P2 = np.array([[5e-7, 1e-7, 0.3], [2e-7, 0.1, 0.2]])
    I2 = np.zeros((2, 3), dtype=np.int64)
    sel = topk.select(P2, I2, 2, 10)
    # sorted: (0,m2,i0) (0,m2,i1) (0,m3,i0) (.1,m3,i1) (.2,m3,i2) (.3,m2,i2);
    # (2,1) and (3,1) lie within m/2 of an accepted cell of their length
    assert [(m, i, d) for (m, i, _, d) in sel] == [(2, 0, 0.0), (3, 0, 0.0), (3, 2, 0.2),
                                                   (2, 2, 0.3)]
    # per-length mode ranks each length separately
    sel = topk.select(P2, I2, 2, 1, topk.PER_LENGTH)
    assert [(m, i) for (m, i, _, _) in sel] == [(2, 0), (3, 0)]
