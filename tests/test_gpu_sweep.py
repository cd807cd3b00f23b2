"""Soundness across configurations (Prop. 1), through the C ABI.

The method is a heuristic selection of the pairs it evaluates, so recall
depends on the knobs; soundness does not.  For every configuration below,
in both precision forms and for float32 input, the profile rows and the
reported motifs must satisfy what holds whatever pairs were admitted:
every finite cell is at least the exact profile, its neighbour is valid
(outside the exclusion zone, not a constant window), sampled cells equal
the oracle's direct distance of their stored pair, and every reported
motif carries the FP64 direct distance of its pair.  The sweep reaches code
paths the default configuration does not (narrow widths, short keys, wide
sieve bands that run the per-member sieve in the mixed form, small and
large chunks, exhaustive sieve, half-precision rows with each of them).
"""
import numpy as np
import pytest

import workloads
from oracle import exact

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
def exact64(small):
    return exact.pmp(small.x, small.m_min, small.m_max, small.excl, tier="diag")


@pytest.fixture(scope="module")
def exact32(small):
    x32 = small.x.astype(np.float32).astype(np.float64)
    return x32, exact.pmp(x32, small.m_min, small.m_max, small.excl, tier="diag")


HALF, EXH, NOS, NOC, FP64A = 0x80, 0x1, 0x2, 0x4, 0x20

CONFIGS = [
    dict(K=4),
    dict(K=9, B=12),
    dict(B=16, d0=6),
    dict(stride=1),
    dict(stride=5),
    dict(alpha=4),
    dict(alpha=64, gamma=2),
    dict(probe_cap=1),
    dict(sieve_w=4),
    dict(sieve_w=32),
    dict(chunk=64),
    dict(chunk=4096),
    dict(beta=16),
    dict(rounds=1, dm=2, dp=1),
    dict(seed=12345),
    dict(flags=EXH),
    dict(flags=NOS | NOC),
    # mixed form only
    dict(flags=HALF, mixed_only=True),
    dict(flags=HALF, sieve_w=32, mixed_only=True),
    dict(flags=HALF | EXH, mixed_only=True),
    dict(flags=HALF, chunk=64, K=6, mixed_only=True),
    dict(flags=FP64A, mixed_only=True),
]


def _ids(c):
    return "-".join(f"{k}{v}" for k, v in c.items() if k != "mixed_only") or "default"


def check_sound(pn, ctx, got, x, P, s, precision, tag):
    L = s.m_max - s.m_min + 1
    d, j = pn.unpack_keys(ctx.profile_rows(0, x.shape[0], L))
    # stored keys keep 26 mantissa bits on top of the in-stream arithmetic
    rtol, atol = (2.0 ** -25, 1e-12) if precision == 0 else (2e-5, 2e-5)
    fin = np.isfinite(d)
    assert fin.any(), tag
    assert np.all(d[fin] >= P[fin] * (1 - rtol) - atol), tag
    ms, iis = np.nonzero(fin)
    jj = j[ms, iis]
    assert np.all(np.abs(iis - jj) >= s.excl), tag
    assert np.all(np.isfinite(P[ms, jj])), tag                 # the neighbour is not constant
    rng = np.random.default_rng(1)
    for t in rng.choice(ms.shape[0], size=min(300, ms.shape[0]), replace=False):
        m = s.m_min + ms[t]
        ref = exact.dist(x, m, iis[t], jj[t])
        assert abs(d[ms[t], iis[t]] - ref) <= rtol * ref + atol, (tag, m, iis[t])
    assert len(got) > 0, tag
    for r in got:
        ref = exact.dist(x, int(r["m"]), int(r["i"]), int(r["j"]))
        ref = 0.0 if ref < 1e-6 else ref                        # zero-snap (Sec. 3.6)
        assert abs(float(r["d"]) - ref) <= 1e-9 * ref + 1e-12, (tag, r)
        assert abs(int(r["i"]) - int(r["j"])) >= s.excl, (tag, r)
        # the oracle's per-diagonal recurrences round differently from a direct evaluation
        assert float(r["d"]) >= P[int(r["m"]) - s.m_min, int(r["i"])] * (1 - 1e-9) - 1e-9, (tag, r)


@pytest.mark.parametrize("cfg", CONFIGS, ids=_ids)
@pytest.mark.parametrize("precision", [0, 1])
def test_sound_across_configurations(pn, small, exact64, cfg, precision):
    cfg = dict(cfg)
    if cfg.pop("mixed_only", False) and precision == 0:
        pytest.skip("half rows and tensor-core anchors exist in the mixed form only")
    s = small
    P, _ = exact64
    ctx = pn.Context(precision=precision, topk_mode=0, **cfg)
    got = ctx.pmp(s.x, s.m_min, s.m_max, s.k, s.excl)
    check_sound(pn, ctx, got, s.x, P, s, precision, (precision, _ids(cfg)))


@pytest.mark.parametrize("cfg", [c for c in CONFIGS if c.get("flags", 0) & HALF or "sieve_w" in c or "K" in c],
                         ids=_ids)
def test_sound_across_configurations_float32_input(pn, small, exact32, cfg):
    """Float32 input runs the packed single-float distance path of the mixed form."""
    cfg = {k: v for k, v in cfg.items() if k != "mixed_only"}
    s = small
    x32, (P, _) = exact32
    ctx = pn.Context(precision=1, topk_mode=0, **cfg)
    got = ctx.pmp(s.x.astype(np.float32), s.m_min, s.m_max, s.k, s.excl)
    check_sound(pn, ctx, got, x32, P, s, 1, ("f32", _ids(cfg)))
