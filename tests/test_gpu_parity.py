"""GPU parity of the CUDA path against the CPU oracle, step by step and end to end.

Tolerances and where they come from:
* features: FP32 rows of FP64 sliding-DFT state (plain) differ from the
  oracle's direct FP64 DFT by the rounding of the FP64 state to FP32 (half
  an FP32 ulp, 2^-24 |F|) plus the FP64 recurrence's drift over at most C
  slides, far below it; the test allows 2^-22 (|F| + 1).  The mixed form's
  FP32 recurrence accumulates one rounding per slide and bin, at most about
  sqrt(C) 2^-24 |X| / sigma for C = 256 slides (about 1e-6 relative), with
  the anchor's own 3xTF32 error (about 1e-6 |F|) on top; the drift measured
  at C = 256 is 0.8e-6 to 4.2e-6 relative, and 2e-4 (|F| + 1) leaves a
  factor of about 50 above it.
* signature bits: equal wherever the oracle's margin exceeds the feature
  error times the projection norm (the decision is taken in FP32 on the GPU).
* in-stream distances: 1e-9 relative (plain, FP64) or 2e-5 relative + 2e-5
  absolute (mixed, FP32 sums of float-float centred samples).
* reported motifs: the oracle's top-k (m, i, j) exactly, distances within
  1e-6 relative (FP64 recomputation of the reported cells).
"""
import numpy as np
import pytest

import workloads
from oracle import exact, spectral, topk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pn():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_17481_b300 as pkg
    from paper_2607_17481_b300 import build
    build.build()
    return pkg


@pytest.fixture(scope="module")
def small():
    return workloads.planted_random_walk()


@pytest.fixture(scope="module")
def small_exact(small):
    return exact.pmp(small.x, small.m_min, small.m_max, small.excl, tier="diag")


def run(pn, s, **cfg):
    ctx = pn.Context(**cfg)
    mot = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    return ctx, mot


@pytest.mark.parametrize("precision", [0, 1])
def test_features_and_signatures(pn, small, precision):
    s = small
    ctx, _ = run(pn, s, precision=precision, topk_mode=1, stride=2)
    for ai in (0, 5, 16):
        a = spectral.anchors(s.m_min, s.m_max)[ai]
        nw = s.x.shape[0] - a + 1
        a_got, F, sig = ctx.anchor_state(0, ai, nw)
        assert a_got == a
        ref = spectral.dft_features(s.x, a)
        err = np.abs(F[:, :30].astype(np.float64) - ref)
        tol = (2.0 ** -22 if precision == 0 else 2e-4) * (np.abs(ref) + 1.0)
        assert np.all(err <= tol), (a, float(err.max()))
        assert np.all(F[:, 30:] == 0.0)
        g = ctx.projections(a).astype(np.float64)[:, :30]
        marg = ref @ g[:24].T
        bits = ((sig[:, None] >> np.arange(23, -1, -1)[None, :]) & 1).astype(bool)
        decided = np.abs(marg) > 1e-3 * (np.linalg.norm(ref, axis=1, keepdims=True) + 1.0)
        assert np.array_equal(bits[decided], (marg >= 0)[decided])
        assert decided.mean() > 0.99


@pytest.mark.parametrize("beta", [0, 7])
def test_query_levels_match_stream_population(pn, small, beta):
    """The directory population and depth every query is searched with equal
    the oracle's batched schedule (Sec. 3.5; depth rule of Prop. 4), read
    back from the device through panache_query_levels, which evaluates the
    search kernel's own rule.  A planted constant run checks the skipped
    windows; beta = 7 checks batches shorter than the exclusion zone."""
    x = small.x.copy()
    x[3000:3100] = x[3000]
    ctx = pn.Context(beta=beta, topk_mode=0)
    ctx.pmp(x, small.m_min, small.m_max, small.k, small.excl)
    b = beta if 0 < beta < small.excl else small.excl
    n = x.shape[0]
    cfg = ctx.config
    for ai, a in enumerate(spectral.anchors(small.m_min, small.m_max)):
        nw = n - a + 1
        pop, dep = ctx.query_levels(0, ai, nw)
        W = np.lib.stride_tricks.sliding_window_view(x, a)
        nonconst = W.max(axis=1) != W.min(axis=1)
        pre = np.concatenate([[0], np.cumsum(nonconst)])
        searched = nonconst & (np.arange(nw) >= small.excl)
        assert not nonconst[3000:3100 - a + 1].any()       # windows inside the constant run
        assert np.all(pop[~searched] == -1) and np.all(dep[~searched] == -1)
        want_p = np.array([spectral.stream_population(q, a, n, b, pre) for q in np.nonzero(searched)[0]])
        want_d = np.array([spectral.depth(int(P), cfg.alpha, cfg.B) for P in want_p])
        assert np.array_equal(pop[searched], want_p), a
        assert np.array_equal(dep[searched], want_d), a


@pytest.mark.parametrize("alpha", [16, 4])
def test_candidate_lists_match_oracle(pn, small, alpha):
    """Every sampled query's candidate list -- probe order, valid prefixes,
    budget split (Sec. 3.4) -- read back through panache_query_candidates,
    equals the list the oracle's probe_buckets and budget_select build over
    the directory level the query sees (the first alpha 2^d non-constant
    windows in stream order, bucketed by the d-bit prefix of their keys, in
    ascending start).  The keys and rows are the device's (their own parity
    is tested above); queries whose margin ranking is within rounding of a
    tie are skipped.  alpha = 4 (R = 32) makes most lists overflow a bucket."""
    s = small
    ctx = pn.Context(precision=1, topk_mode=0, stride=2, alpha=alpha)
    ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    cfg = ctx.config
    R = cfg.gamma * cfg.alpha
    n = s.x.shape[0]
    rng = np.random.default_rng(11)
    checked = 0
    for ai in (0, 8, 16):
        a = spectral.anchors(s.m_min, s.m_max)[ai]
        nw = n - a + 1
        _, F, sig = ctx.anchor_state(0, ai, nw)
        g = ctx.projections(a).astype(np.float64)
        W = np.lib.stride_tricks.sliding_window_view(s.x, a)
        nonconst = W.max(axis=1) != W.min(axis=1)
        pre = np.concatenate([[0], np.cumsum(nonconst)])
        order = np.nonzero(nonconst)[0]                     # stream order of the non-constant windows
        qs = rng.choice(np.arange(s.excl, nw), size=150, replace=False)
        got = ctx.query_candidates(0, ai, qs, cap=512)
        for q, lst in zip(qs, got):
            assert lst is not None
            P = spectral.stream_population(int(q), a, n, s.excl, pre)
            d = spectral.depth(P, cfg.alpha, cfg.B)
            marg = F[q, :30].astype(np.float64) @ g[:cfg.B, :30].T
            mag = np.sort(np.abs(marg[:d]))
            if d > 1 and np.any(np.diff(mag) <= 1e-4 * (mag[1:] + 1e-12)):
                continue                                    # a near-tie of margins: either order is right
            members = order[:min(len(order), cfg.alpha << d)]
            pref = (sig[members].astype(np.int64) >> (cfg.B - d)) if d > 0 else np.zeros(len(members), np.int64)
            want, taken = [], 0
            for b in spectral.probe_buckets(int(sig[q]), marg, d, cfg.B, cfg.d0, cfg.probe_cap):
                if taken >= R:
                    break
                valid = np.sort(members[(pref == b) & (members <= q - s.excl)])
                pos = spectral.budget_select(len(valid), R - taken)
                want.extend(int(valid[p]) for p in pos)
                taken += len(pos)
            assert list(lst) == want, (ai, int(q), d)
            checked += 1
    assert checked >= 300


@pytest.mark.parametrize("precision", [0, 1])
def test_profile_rows_are_sound(pn, small, small_exact, precision):
    """Every finite cell is the exact distance of a valid neighbour and never below the exact profile (Prop. 1)."""
    s = small
    P, I = small_exact
    ctx, _ = run(pn, s, precision=precision, topk_mode=1)
    L = s.m_max - s.m_min + 1
    d, j = pn.unpack_keys(ctx.profile_rows(0, s.x.shape[0], L))
    # stored keys keep 26 mantissa bits (truncation 2^-26 relative) on top of the in-stream error
    rtol, atol = (2.0 ** -25, 1e-12) if precision == 0 else (2e-5, 2e-5)
    fin = np.isfinite(d)
    assert fin[::2].mean() > 0.9           # anchor rows are filled by the streaming pass
    ms, iis = np.nonzero(fin)
    assert np.all(np.abs(iis - j[ms, iis]) >= s.excl)
    rng = np.random.default_rng(0)
    pick = rng.choice(ms.shape[0], size=min(3000, ms.shape[0]), replace=False)
    for t in pick:
        m = s.m_min + ms[t]
        ref = exact.dist(s.x, m, iis[t], j[ms[t], iis[t]])
        assert abs(d[ms[t], iis[t]] - ref) <= rtol * ref + atol, (m, iis[t])
    assert np.all(d[fin] >= P[fin] * (1 - rtol) - atol)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_topk_matches_oracle(pn, small, small_exact, mode, precision):
    """Recall 1.0 of the oracle's top-20 (global) and top-20 per length (660
    cells), distances within 1e-6, at the library's defaults (anchor stride
    2 for the global list, 1 for the per-length lists)."""
    from parity import compare
    s = small
    P, I = small_exact
    ref = topk.select(P, I, s.m_min, s.k, mode)
    ctx, got = run(pn, s, precision=precision, topk_mode=mode)
    assert len(got) == len(ref)
    r = compare(s.x, got, ref)
    assert r["misses"] == 0, r["miss_list"]
    assert r["bad_dist"] == 0
    # the per-length default builds one anchor per length
    L = s.m_max - s.m_min + 1
    n_anchor = L if mode == 1 else len(spectral.anchors(s.m_min, s.m_max))
    assert ctx.query_levels(0, n_anchor - 1, s.x.shape[0] - s.m_max + 1)[0].shape[0] > 0
    with pytest.raises(pn.PanacheError):
        ctx.query_levels(0, n_anchor, 1)


@pytest.mark.parametrize("mode", [0, 1])
def test_topk_sieve_matches_oracle(pn, small, small_exact, mode):
    """With the top-k sieve (float64 walk: the (hi, lo) sample staging, tile
    tables pruned by pivot distances) the lists are still the oracle's."""
    from parity import compare
    s = small
    P, I = small_exact
    ref = topk.select(P, I, s.m_min, s.k, mode)
    ctx, got = run(pn, s, precision=1, topk_mode=mode, flags=pn.FLAG_TOPK_SIEVE)
    assert len(got) == len(ref)
    r = compare(s.x, got, ref)
    assert r["misses"] == 0, r["miss_list"]
    assert r["bad_dist"] == 0


def test_recall_at_paper_stride(pn, small, small_exact):
    """The paper's stride 2 in per-length mode: reported.  Two cells of one
    pair at length 60 are missed: the anchor's search finds the pair shifted
    by one sample, and the cell is not among the completion seeds of its
    length (a better-valued neighbour within m/2 takes its place)."""
    from parity import compare
    s = small
    P, I = small_exact
    ref = topk.select(P, I, s.m_min, s.k, 1)
    _, got = run(pn, s, precision=1, topk_mode=1, stride=2)
    r = compare(s.x, got, ref)
    print("recall at stride 2 (per-length top-20):", (r["hits"] + r["ties"]) / r["n"], r["miss_list"])
    assert r["misses"] <= 0.01 * r["n"]
    assert r["bad_dist"] == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_warm_start_keeps_profile(pn, small, precision):
    """The search's warm start evaluates admitted pairs only, so the profile
    rows (the minimum over the admitted pairs) are bit-identical with and
    without it, through the whole emit stage."""
    s = small
    a, ma = run(pn, s, precision=precision, topk_mode=1, stride=2, flags=pn.FLAG_WARM_START)
    b, mb = run(pn, s, precision=precision, topk_mode=1, stride=2)
    L = s.m_max - s.m_min + 1
    assert np.array_equal(a.profile_rows(0, s.x.shape[0], L), b.profile_rows(0, s.x.shape[0], L))
    assert np.array_equal(ma, mb)
    print("exact distances in the stream with / without warm start:",
          a.stats()["exact_stream"], b.stats()["exact_stream"])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("precision", [0, 1])
def test_reported_cells_hold_exact_profile(pn, small, small_exact, mode, precision):
    """After the row refinement, every reported motif's distance is its
    cell's exact profile value (the oracle's nearest valid neighbour), at
    the paper's stride in both modes; without the refinement the rows are
    only an upper bound (Prop. 1)."""
    s = small
    P, I = small_exact
    ctx, got = run(pn, s, precision=precision, topk_mode=mode, stride=2)
    assert ctx.stats()["refine_passes"] >= 1 and ctx.stats()["exact_refine"] > 0
    for r in got:
        m, i, d = int(r["m"]), int(r["i"]), float(r["d"])
        ref = P[m - s.m_min, i]
        assert abs(d - ref) <= 1e-6 * ref + 1e-12, (m, i, int(r["j"]), d, ref)
    off, _ = run(pn, s, precision=precision, topk_mode=mode, stride=2, flags=pn.FLAG_NO_REFINE)
    assert off.stats()["exact_refine"] == 0


def test_exhaustive_sieve_gram_matches_dense(pn, small):
    """The exhaustive sieve's tensor-core Gram filter skips only pairs whose
    Parseval bound (with its rounding margin) cannot lower either cell: the
    rows equal those of evaluating every pair, within the FP32 rounding of the
    in-stream distances, with fewer exact evaluations."""
    s = small
    off = pn.FLAG_NO_COMPLETION | pn.FLAG_NO_REFINE | pn.FLAG_EXHAUSTIVE_SIEVE
    L = s.m_max - s.m_min + 1
    g, _ = run(pn, s, precision=1, topk_mode=1, stride=2, flags=off | pn.FLAG_SIEVE_GRAM)
    d, _ = run(pn, s, precision=1, topk_mode=1, stride=2, flags=off)
    dg, _ = pn.unpack_keys(g.profile_rows(0, s.x.shape[0], L))
    dd, _ = pn.unpack_keys(d.profile_rows(0, s.x.shape[0], L))
    assert np.array_equal(np.isfinite(dg), np.isfinite(dd))
    fin = np.isfinite(dd)
    assert np.all(np.abs(dg[fin] - dd[fin]) <= 2e-5 * dd[fin] + 2e-5)
    assert g.stats()["exact_sieve"] <= d.stats()["exact_sieve"]
    print("exact sieve evaluations, Gram filter / dense:", g.stats()["exact_sieve"], d.stats()["exact_sieve"])


def test_deterministic(pn, small):
    s = small
    ctx, a = run(pn, s, topk_mode=1, precision=1)
    rows_a = ctx.profile_rows(0, s.x.shape[0], s.m_max - s.m_min + 1)
    ctx2, b = run(pn, s, topk_mode=1, precision=1)
    rows_b = ctx2.profile_rows(0, s.x.shape[0], s.m_max - s.m_min + 1)
    assert np.array_equal(a, b)
    assert np.array_equal(rows_a, rows_b)


def test_batch_equals_single(pn):
    series = workloads.batched_workload(5, seed=3, n_hi=12000)
    ctx = pn.Context(precision=1)
    params = [(q.m_min, q.m_max, q.k, q.excl) for q in series]
    batch = ctx.pmp_batch([q.x for q in series], params)
    for q, got in zip(series, batch):
        one = ctx.pmp(q.x, q.m_min, q.m_max, q.k, q.excl)
        assert np.array_equal(one, got)


def test_batched_series_match_oracle(pn):
    """Batched form: every series' top-10 equals the oracle's (seeded subset of the batched workload)."""
    from parity import compare
    series = workloads.batched_workload(6, seed=5, n_hi=6000)
    ctx = pn.Context(precision=1, topk_mode=0)
    got = ctx.pmp_batch([q.x for q in series], [(q.m_min, q.m_max, q.k, q.excl) for q in series])
    for q, g in zip(series, got):
        P, I = exact.pmp(q.x, q.m_min, q.m_max, q.excl, tier="diag")
        ref = topk.select(P, I, q.m_min, q.k, topk.GLOBAL)
        r = compare(q.x.astype(np.float64), g, ref)
        assert r["misses"] == 0 and r["bad_dist"] == 0, (q.kind, len(q.x), r["miss_list"])


def test_batch_waves_do_not_change_results(pn):
    """A small HBM budget splits the batch into several waves; results are unchanged."""
    series = workloads.batched_workload(8, seed=2, n_hi=20000)
    params = [(q.m_min, q.m_max, q.k, q.excl) for q in series]
    ctx = pn.Context(precision=1)
    one = ctx.pmp_batch([q.x for q in series], params)
    assert ctx.stats()["waves"] == 1
    small = pn.Context(precision=1, hbm_budget_bytes=max(ctx.stats()["device_bytes"] // 3, 200_000_000))
    many = small.pmp_batch([q.x for q in series], params)
    assert small.stats()["waves"] > 1
    for a, b in zip(one, many):
        assert np.array_equal(a, b)


def test_stream_equals_offline(pn, small):
    s = small
    ctx = pn.Context(topk_mode=1)
    st = ctx.stream(s.m_min, s.m_max, s.k, s.excl)
    rng = np.random.default_rng(1)
    pos = 0
    while pos < s.x.shape[0]:
        step = int(rng.integers(1, 3000))
        st.append(s.x[pos:pos + step])
        pos += step
    assert len(st) == s.x.shape[0]
    got = st.topk()
    ref = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    assert np.array_equal(got, ref)


def test_device_input_equals_host(pn, small):
    s = small
    ctx = pn.Context(topk_mode=0)
    host = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    dev = ctx.pmp(torch.from_numpy(s.x).cuda(), s.m_min, s.m_max, s.k, s.excl)
    assert np.array_equal(host, dev)


def test_edge_cases(pn):
    ctx = pn.Context(topk_mode=0)
    rng = np.random.default_rng(4)
    x = np.cumsum(rng.standard_normal(700))
    # series shorter than every length: no windows, no motifs
    assert len(ctx.pmp(x[:20], 32, 40, 5, 8)) == 0
    # windows exist but no valid pair (n < m + excl)
    assert len(ctx.pmp(x[:60], 32, 40, 5, 40)) == 0
    # a single length, ragged chunk tail, planted exactly constant run
    y = x.copy()
    y[300:360] = 1.5
    got = ctx.pmp(y, 16, 16, 4, 16)
    P, I = exact.pmp(y, 16, 16, 16, tier="direct")
    ref = topk.select(P, I, 16, 4, topk.GLOBAL)
    assert [(int(r["m"]), int(r["i"]), int(r["j"])) for r in got] == [(m, i, j) for (m, i, j, _) in ref]
    # constant windows never appear as cells or neighbours
    L = 1
    d, j = pn.unpack_keys(ctx.profile_rows(0, y.shape[0], L))
    const = [i for i in range(700 - 16 + 1) if y[i:i + 16].max() == y[i:i + 16].min()]
    assert np.all(np.isinf(d[0, const]))
    assert not set(const) & set(j[0][j[0] >= 0].tolist())
    # invalid arguments are rejected
    with pytest.raises(pn.PanacheError):
        ctx.pmp(x, 2, 10, 5, 8)
    with pytest.raises(pn.PanacheError):
        ctx.pmp(x, 20, 10, 5, 8)


def test_mixed_drift_within_lambda_over_ten(pn):
    """Mixed form: FP32 sliding state from FP64 anchors drifts at most lambda/10 at the default chunk.

    This keeps Lemma 5's (1 - lambda) shrink valid at the paper's margin.
    Measured on the planted walk (large offsets) and the wafer-like series.
    """
    from paper_2607_17481_b300 import autotune
    for x, (m1, m2) in ((workloads.planted_random_walk().x, (32, 64)),
                        (workloads.wafer_like(100_000, seed=0).x, (100, 150))):
        for a in (m1, m2):
            d, curve = autotune.feature_drift(x, a, 256)
            assert d <= 1e-5, (a, d)
            # windows at an anchor carry the anchor's own error only: 3xTF32
            # tensor-core products (about 2^-21 relative) plus FP32 rounding
            assert curve[0] <= 2e-6


def test_autotune_picks_a_valid_chunk(pn):
    """The tuner takes the longest tested chunk within lambda/10, else the shortest one."""
    from paper_2607_17481_b300 import autotune
    x = workloads.wafer_like(60_000, seed=1).x
    r = autotune.tune(x, 100, 150, sample=60_000, grid_mults=(4, 8))
    ok = [c for c, d in r["drift"].items() if d <= 1e-5]
    assert r["chunk"] == (max(ok) if ok else 64)
    tested = sorted(r["drift"], reverse=True)
    assert all(r["drift"][c] > 1e-5 for c in tested if c > r["chunk"])
    assert r["grid_mult"] in (4, 8)


def test_graph_replay_equals_eager(pn, small):
    """Requests of one shape replay a captured graph of the index and search
    steps; each replay reads the new samples and matches the eager path."""
    s = small
    eager = pn.Context(topk_mode=1)
    graph = pn.Context(topk_mode=1, flags=pn.FLAG_GRAPH)
    rng = np.random.default_rng(21)
    x2 = np.cumsum(rng.standard_normal(s.x.shape[0]))
    x3 = np.cumsum(rng.standard_normal(5000))
    for x in (s.x, x2, s.x, x3, x2[:5000], torch.from_numpy(x2).cuda()):
        n = x.shape[0]
        want = eager.pmp(x, s.m_min, s.m_max, s.k, s.excl)
        got = graph.pmp(x, s.m_min, s.m_max, s.k, s.excl)
        assert np.array_equal(got, want), n
    assert graph.stats()["kernel_launches"] > 0


@pytest.mark.parametrize("kind", ["wafer", "walk", "noise"])
def test_width_calibration_matches_oracle(pn, kind):
    """Spectral-width calibration (Sec. 3.2): the device statistics equal the
    oracle's sample means to FP64 rounding, and the chosen width is the same."""
    from oracle import calibrate
    rng = np.random.default_rng(8)
    if kind == "wafer":
        x, lo, hi = workloads.wafer_like(30_000, seed=3).x, 100, 150
    elif kind == "walk":
        x, lo, hi = np.cumsum(rng.standard_normal(20_000)), 32, 64
    else:
        x, lo, hi = rng.standard_normal(20_000), 40, 80
    ctx = pn.Context()
    K, e, c = ctx.calibrate_width(x, lo, hi)
    eo, co, _ = calibrate.statistics(np.asarray(x, dtype=np.float64), lo, hi)
    assert np.allclose(e, eo, rtol=1e-9, atol=1e-12)
    assert np.allclose(c, co, rtol=1e-9, atol=1e-15)
    assert K == calibrate.select_width(eo, co, len(x))
    # the device path reads device series too
    K2, e2, _ = ctx.calibrate_width(torch.from_numpy(np.ascontiguousarray(x)).cuda(), lo, hi)
    assert K2 == K and np.array_equal(e2, e)


@pytest.mark.parametrize("precision", [0, 1])
def test_exhaustive_sieve(pn, small, small_exact, precision):
    """The exhaustive sieve evaluates every valid pair of every hot class (the
    mixed form as 64 x 64 tiles): with completion and row refinement off
    (their seeds depend on the rows), every cell is at most the default sieve's up to the in-stream
    rounding, the rows stay sound, and with completion the global top-k
    equals the oracle's."""
    s = small
    P, I = small_exact
    off = pn.FLAG_NO_COMPLETION | pn.FLAG_NO_REFINE
    base, _ = run(pn, s, precision=precision, topk_mode=1, flags=off)
    L = s.m_max - s.m_min + 1
    d0, _ = pn.unpack_keys(base.profile_rows(0, s.x.shape[0], L))
    ctx, _ = run(pn, s, precision=precision, topk_mode=1, flags=pn.FLAG_EXHAUSTIVE_SIEVE | off)
    d1, j1 = pn.unpack_keys(ctx.profile_rows(0, s.x.shape[0], L))
    rtol, atol = (2.0 ** -25, 1e-12) if precision == 0 else (2e-5, 2e-5)
    fin0 = np.isfinite(d0)
    assert np.all(np.isfinite(d1[fin0]))
    assert np.all(d1[fin0] <= d0[fin0] * (1 + 2 * rtol) + atol)
    fin = np.isfinite(d1)
    assert np.all(d1[fin] >= P[fin] * (1 - rtol) - atol)
    ms, iis = np.nonzero(fin)
    assert np.all(np.abs(iis - j1[ms, iis]) >= s.excl)
    # global top-k: exact at the paper's defaults (per length, stride 2 misses
    # up to 1% of cells with or without the exhaustive sieve; see the recall test)
    _, got = run(pn, s, precision=precision, topk_mode=0, flags=pn.FLAG_EXHAUSTIVE_SIEVE)
    ref = topk.select(P, I, s.m_min, s.k, topk.GLOBAL)
    from parity import compare
    r = compare(s.x, got, ref)
    assert r["misses"] == 0 and r["bad_dist"] == 0, r


@pytest.mark.parametrize("mode", [0, 1])
def test_half_feature_rows(pn, small, small_exact, mode):
    """Half-precision feature rows (the row cache of Sec. 3.2 at half the
    bytes): the rows are the FP32 rows rounded to nearest, the keys come from
    the FP32 rows, and every bound read from half rows carries the absolute
    inflation margin of Lemma 5's proof.  The margin's premises are checked on
    the rows, the motifs equal the FP32-row form's (global mode: the
    oracle's), and the device footprint shrinks."""
    s = small
    full, got_full = run(pn, s, precision=1, topk_mode=mode, stride=2)
    half, got_half = run(pn, s, precision=1, topk_mode=mode, stride=2, flags=pn.FLAG_HALF_FEATURES)
    assert np.array_equal(got_half[["m", "i", "j"]], got_full[["m", "i", "j"]])
    assert np.allclose(got_half["d"], got_full["d"], rtol=1e-12, atol=0)
    assert half.stats()["device_bytes"] < full.stats()["device_bytes"]
    for ai in (0, 5, 16):
        a = spectral.anchors(s.m_min, s.m_max)[ai]
        nw = s.x.shape[0] - a + 1
        a0, F0, k0 = full.anchor_state(0, ai, nw)
        a1, F1, k1 = half.anchor_state(0, ai, nw)
        assert a0 == a1 == a and np.array_equal(k0, k1)          # keys from the FP32 rows
        # round to nearest even, as numpy's float16 conversion
        assert np.array_equal(F1, F0.astype(np.float16).astype(np.float32))
        # the margin's premises: the stored bins of a z-normalised window hold
        # at most a^2 / 2 of energy (Parseval), and a bound read from half rows
        # is within 4 sqrt(a) 2^-11 of the FP32 rows' bound
        E = (F0.astype(np.float64) ** 2).sum(axis=1)
        assert E.max() <= 0.5 * a * a * (1 + 1e-3)
        rng = np.random.default_rng(ai)
        i, j = rng.integers(0, nw, 8192), rng.integers(0, nw, 8192)
        lb0 = np.sqrt(2.0 / a * ((F0[i].astype(np.float64) - F0[j]) ** 2).sum(axis=1))
        lb1 = np.sqrt(2.0 / a * ((F1[i].astype(np.float64) - F1[j]) ** 2).sum(axis=1))
        assert np.all(np.abs(lb1 - lb0) <= spectral.lb_inflation_bound(a, 2.0 ** -11))
    if mode == 0:
        from parity import compare
        P, I = small_exact
        r = compare(s.x, got_half, topk.select(P, I, s.m_min, s.k, topk.GLOBAL))
        assert r["misses"] == 0 and r["bad_dist"] == 0, r
    with pytest.raises(pn.PanacheError) as e:
        pn.Context(precision=0, flags=pn.FLAG_HALF_FEATURES)      # the plain form keeps FP32 rows
    assert e.value.code == -1
