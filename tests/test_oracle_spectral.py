"""Pins of the spectral component oracles (Sec. 3.2-3.6, Appendix A)."""
import math
import os

import numpy as np
import pytest

from oracle import exact, spectral as sp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.strip() and not line.startswith("#"):
            rows.append([int(v, 16) for v in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = sp.philox4x32_10(r[0:4], r[4:6])[0]
        assert [int(v) for v in out] == r[6:10]


def test_paper_constants():
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_constants.txt")):
        if line.strip() and not line.startswith("#"):
            name, value = line.split()[:2]
            vals[name] = float(value)
    assert round(1.0 / (2 * sp.F32_EPS / 1e-4)) == vals["inv_two_eps_over_lambda"]
    # sqrt(2m)/600 is the lemma's threshold up to rounding (exactly 593.2)
    f = math.sqrt(250) / sp.lb_safe_threshold(125)
    assert abs(f - vals["inv_threshold_factor"]) / vals["inv_threshold_factor"] < 0.02
    assert sp.lb_inflation_bound(80) < vals["inflation_max_m80"]
    assert sp.lb_inflation_bound(80) > 0.9 * vals["inflation_max_m80"]
    assert 8 * 16 == vals["budget_R"]


def test_kprime_cap():
    """K' = min(K-1, ceil(m/2)-1) keeps 2K' < m, so no bin is counted with its alias."""
    for m in range(3, 40):
        for K in (2, 4, 8, 16):
            kp = sp.kprime(m, K)
            assert 2 * kp < m
            assert kp == min(K - 1, math.ceil(m / 2) - 1)
    assert sp.kprime(31) == 15 and sp.kprime(32) == 15 and sp.kprime(30) == 14 and sp.kprime(125) == 15


def test_features_match_fft_and_ac_invariance():
    """F equals bins 1..K' of the FFT of the z-normalised window (Lemma 1)."""
    rng = np.random.default_rng(1)
    x = np.cumsum(rng.standard_normal(600)) + 100.0
    for m in (7, 32, 33, 64, 125):
        F = sp.dft_features(x, m, 16, rows=[0, 13, 600 - m])
        kp = sp.kprime(m)
        for t, i in enumerate([0, 13, 600 - m]):
            Xz = sp.full_dft_znorm(x[i:i + m])
            assert abs(Xz[0]) < 1e-9                       # DC of a z-normalised window vanishes
            assert np.allclose(F[t, 0:2 * kp:2], Xz[1:kp + 1].real, atol=1e-9)
            assert np.allclose(F[t, 1:2 * kp:2], Xz[1:kp + 1].imag, atol=1e-9)
            assert np.all(F[t, 2 * kp:] == 0.0)
            # Parseval: the z-normalised spectrum carries m^2; stored bins at most m^2/2
            assert np.sum(np.abs(Xz) ** 2) == pytest.approx(m * m, rel=1e-10)
            assert np.sum(F[t] ** 2) <= m * m / 2 + 1e-9


def test_sliding_recurrence_sign_convention():
    """Direct features obey X_{i+1,k} = e^{2 pi i k/m} (X_{i,k} - t_i + t_{i+m}) (Sec. 3.2)."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal(300)
    m = 40
    kp = sp.kprime(m)
    mu, sg, _ = exact.moments(x, m)
    F = sp.dft_features(x, m)
    X = (F[:, 0:2 * kp:2] + 1j * F[:, 1:2 * kp:2]) * sg[:, None]
    k = np.arange(1, kp + 1)
    rot = np.exp(2j * np.pi * k / m)
    for i in (0, 10, 200):
        pred = rot * (X[i] - x[i] + x[i + m])
        assert np.allclose(pred, X[i + 1], atol=1e-9)


def test_lower_bound_exhaustive():
    """LB <= d for every equal-length pair, non-decreasing in K (Lemma 2, Prop. 3)."""
    rng = np.random.default_rng(8)
    x = np.cumsum(rng.standard_normal(160))
    for m in (9, 16, 31, 40):
        nw = 160 - m + 1
        D = np.array([[exact.dist(x, m, i, j) for j in range(nw)] for i in range(nw)])
        prev = np.zeros_like(D)
        for K in (2, 3, 5, 8, 16):
            F = sp.dft_features(x, m, K)
            LB = sp.lower_bound(F[:, None, :], F[None, :, :], m)
            assert np.all(LB <= D + 1e-9)
            assert np.all(LB >= prev - 1e-12)
            prev = LB
        if m % 2 == 1 and sp.kprime(m) == (m - 1) // 2:
            # all conjugate pairs retained: the bound is the distance itself
            assert np.allclose(LB, D, atol=1e-9)


def test_projections_are_standard_gaussian():
    g = np.concatenate([sp.projections(a, 12345).ravel() for a in range(30, 130)])
    assert g.shape[0] == 100 * 25 * 30
    assert abs(g.mean()) < 0.02 and abs(g.std() - 1.0) < 0.02
    # Kolmogorov-Smirnov distance to N(0,1)
    gs = np.sort(g)
    cdf = 0.5 * (1 + np.vectorize(math.erf)(gs / math.sqrt(2)))
    ks = np.max(np.abs(cdf - np.arange(1, gs.shape[0] + 1) / gs.shape[0]))
    assert ks < 1.63 / math.sqrt(gs.shape[0])          # 1% level
    # independent per anchor and per seed
    assert not np.allclose(sp.projections(40, 1), sp.projections(42, 1))
    assert not np.allclose(sp.projections(40, 1), sp.projections(40, 2))
    assert np.array_equal(sp.projections(40, 1), sp.projections(40, 1))


def test_simhash_collision_rate():
    """Pr[bit differs] = theta/pi (Fact 1), over many seeded projections."""
    rng = np.random.default_rng(0)
    u = rng.standard_normal(30)
    v = u + 0.8 * rng.standard_normal(30)
    theta = math.acos(u @ v / np.linalg.norm(u) / np.linalg.norm(v))
    diffs = 0
    total = 0
    for seed in range(200):
        g = sp.projections(64, seed)
        su = sp.margins(u, g) >= 0
        sv = sp.margins(v, g) >= 0
        diffs += int(np.sum(su != sv))
        total += su.shape[0]
    p = theta / math.pi
    sd = math.sqrt(p * (1 - p) / total)
    assert abs(diffs / total - p) < 4 * sd


def test_signature_bit_order():
    g = np.zeros((25, 30))
    g[0, 0] = 1.0          # bit 1 looks at dim 0
    g[23, 1] = 1.0         # bit 24 looks at dim 1
    F = np.zeros((3, 30))
    F[0, 0] = 1.0
    F[1, 1] = 1.0
    F[2, :2] = -1.0
    sig = sp.signature(F, g)
    # zero margins count as set bits (>= 0)
    assert sig[0] == (1 << 24) - 1
    assert sig[1] == (1 << 24) - 1
    assert sig[2] == (1 << 24) - 1 - (1 << 23) - 1
    assert sp.prefix(sig, 1)[2] == 0 and sp.prefix(sig, 2)[2] == 1


def test_depth_rule_occupancy():
    """Literal insertion with global doubling keeps P <= alpha 2^d (Prop. 4)."""
    alpha, B = 16, 24
    d, moves = 0, 0
    for P in range(1, 200001):
        while P > alpha * (1 << d) and d < B:
            d += 1
            moves += P            # a doubling rehomes every stored entry
        assert P <= alpha * (1 << d)
        assert sp.depth(P, alpha, B) == d
        if d > 0:
            assert alpha * (1 << (d - 1)) < P          # mean occupancy in (alpha/2, alpha]
    assert moves < 4 * 200000 + d
    assert sp.depth(10 ** 12, 16, 24) == 24


def test_probe_order():
    rng = np.random.default_rng(3)
    for d in (0, 1, 5, 12, 13, 16, 20, 24):
        marg = rng.standard_normal(24)
        sig = int(rng.integers(0, 1 << 24))
        pb = sp.probe_buckets(sig, marg, d)
        h = sp.probe_count(d)
        assert len(pb) == 1 + h
        assert h == (0 if d == 0 else min(d, 8, 1 + max(0, d - 12)))
        pre = sig >> (24 - d) if d else 0
        assert pb[0] == pre
        flipped = [(b ^ pre).bit_length() for b in pb[1:]]
        assert all(bin(b ^ pre).count("1") == 1 for b in pb[1:])
        bits = [d - f for f in flipped]                 # 0-based signature bit
        mags = [abs(marg[b]) for b in bits]
        assert mags == sorted(mags)
        assert set(bits) == set(sorted(range(d), key=lambda l: abs(marg[l]))[:h])


def test_budget_select():
    for s in range(0, 70):
        for r in range(0, 40):
            sel = sp.budget_select(s, r)
            assert len(sel) == min(s, r)
            assert len(set(sel)) == len(sel)
            assert all(0 <= p < s for p in sel)
            if s > r > 0:
                h1 = (r + 1) // 2
                assert sel[-h1:] == list(range(s - h1, s))           # most recent half
                even = sel[:r // 2]
                assert even == sorted(even) and (not even or even[0] == 0)
                assert all(p < s - h1 for p in even)
                if len(even) > 1:
                    gaps = np.diff(even)
                    assert gaps.max() - gaps.min() <= 1              # even intervals


def test_sieve_pairs_bruteforce():
    rng = np.random.default_rng(6)
    members = rng.choice(5000, size=40, replace=False)
    proj = rng.standard_normal(40)
    pairs = set(sp.sieve_pairs(members, proj, excl=100, w=8))
    order = sorted(range(40), key=lambda t: (proj[t], members[t]))
    ref = set()
    for u in range(40):
        for v in range(40):
            if 0 < abs(u - v) <= 8:
                a, b = members[order[u]], members[order[v]]
                if abs(int(a) - int(b)) >= 100:
                    ref.add((min(int(a), int(b)), max(int(a), int(b))))
    assert pairs == ref


def test_completion_box():
    tr = sp.completion_triples(40, 500, 900, 2000, 32, 64, 64)
    assert len(tr) == 13 * 9 * 9 == 1053
    tr = sp.completion_triples(33, 2, 60, 200, 32, 64, 64)
    assert all(32 <= m <= 39 and 0 <= i <= 200 - m and 0 <= j <= 200 - m and abs(i - j) >= 64
               for (m, i, j) in tr)
    assert len(tr) < 1053


def test_anchor_set():
    assert sp.anchors(32, 64) == list(range(32, 65, 2))
    assert len(sp.anchors(32, 64)) == 17
    assert len(sp.anchors(100, 150)) == 26
    assert sp.anchors(100, 151) == list(range(100, 151, 2)) + [151]


def test_half_precision_inflation_bound():
    """Proof of Lemma 5 at half precision (eps = 2^-11): rounding every stored
    feature of exact FP64 rows to float16 moves the computed bound by at most
    the absolute inflation bound 4 sqrt(m) eps (plus 2^-24 per component for
    subnormal halves); the triangle inequality gives half of it, the slack the
    half-row search keeps.  The stored bins of a z-normalised window hold at
    most m^2 / 2 of energy (Parseval), and above the lemma's threshold the
    (1 - lambda) shrink alone covers the rounding."""
    eps, lam = 2.0 ** -11, 0.02
    rng = np.random.default_rng(11)
    n = 1200
    series = {
        "walk": np.cumsum(rng.standard_normal(n)),
        "noise": rng.standard_normal(n),
        "tone": np.sin(2 * np.pi * np.arange(n) / 37.0) + 0.05 * rng.standard_normal(n),
    }
    for name, x in series.items():
        for m in (32, 100, 150):
            F = sp.dft_features(x, m)
            assert np.all((F ** 2).sum(axis=1) <= 0.5 * m * m * (1 + 1e-12)), (name, m)
            Fh = F.astype(np.float16).astype(np.float64)
            nw = F.shape[0]
            i, j = rng.integers(0, nw, 4000), rng.integers(0, nw, 4000)
            lb = sp.lower_bound(F[i], F[j], m)
            lbh = sp.lower_bound(Fh[i], Fh[j], m)
            sub = math.sqrt(2.0 * F.shape[1] / m) * 2.0 ** -24
            gap = np.abs(lbh - lb)
            assert np.all(gap <= sp.lb_inflation_bound(m, eps) + sub), (name, m, float(gap.max()))
            assert np.all(gap <= 0.5 * sp.lb_inflation_bound(m, eps) + sub), (name, m, float(gap.max()))
            big = lb >= sp.lb_safe_threshold(m, eps, lam)
            assert np.all((1 - lam) * lbh[big] <= lb[big] + 1e-12), (name, m)


def _stream_simulation(n: int, a: int, beta: int, nonconst) -> dict:
    """Algorithm 1's schedule, literally: samples arrive beta at a time; after
    each arrival every window whose last sample has arrived is inserted (if
    non-constant), then the windows completed by this arrival are searched
    and see the directory as it stands."""
    seen = {}
    inserted = 0
    next_window = 0
    arrived = 0
    while arrived < n:
        arrived = min(n, arrived + beta)                   # samples [0, arrived) are here
        done = []
        while next_window + a <= arrived:                  # window fully arrived
            if nonconst[next_window]:
                inserted += 1
            done.append(next_window)
            next_window += 1
        for q in done:
            seen[q] = inserted
    return seen


def test_stream_population_hand_cases():
    # n = 20, a = 4, beta = 5, no constant window: window w ends at sample w + 3
    pre = np.arange(0, 18)                                 # nonconst_prefix[t] = t (17 windows)
    # q = 0 ends at 3, batch [0, 5): windows ending at <= 4 are 0 and 1
    assert sp.stream_population(0, 4, 20, 5, pre) == 2
    assert sp.stream_population(1, 4, 20, 5, pre) == 2
    # q = 2 ends at 5, batch [5, 10): windows 0..6
    assert sp.stream_population(2, 4, 20, 5, pre) == 7
    assert sp.stream_population(6, 4, 20, 5, pre) == 7
    assert sp.stream_population(7, 4, 20, 5, pre) == 12
    # last batch [15, 20): every one of the 17 windows
    assert sp.stream_population(16, 4, 20, 5, pre) == 17
    # a last partial batch: beta = 6, batches [0,6) [6,12) [12,18) [18,20)
    assert sp.stream_population(14, 4, 20, 6, pre) == 15     # ends at 17, batch [12, 18)
    assert sp.stream_population(15, 4, 20, 6, pre) == 17     # ends at 18, batch [18, 20) clipped
    # beta = 1 (every sample its own batch): a query sees itself and all earlier windows
    for q in range(17):
        assert sp.stream_population(q, 4, 20, 1, pre) == q + 1
    # constant windows 3..5 are never inserted
    nc = np.ones(17, bool)
    nc[3:6] = False
    pre_c = np.concatenate([[0], np.cumsum(nc)])
    assert sp.stream_population(2, 4, 20, 5, pre_c) == 4     # windows 0..6 less 3, 4, 5
    assert sp.stream_population(16, 4, 20, 5, pre_c) == 14


@pytest.mark.parametrize("seed", range(6))
def test_stream_population_matches_simulation(seed):
    rng = np.random.default_rng(seed)
    for _ in range(25):
        a = int(rng.integers(3, 40))
        n = int(rng.integers(a, 400))
        beta = int(rng.integers(1, 90))
        nw = n - a + 1
        nonconst = rng.random(nw) < rng.uniform(0.3, 1.0)
        pre = np.concatenate([[0], np.cumsum(nonconst)])
        sim = _stream_simulation(n, a, beta, nonconst)
        assert sorted(sim) == list(range(nw))
        for q in range(nw):
            assert sp.stream_population(q, a, n, beta, pre) == sim[q], (n, a, beta, q)
