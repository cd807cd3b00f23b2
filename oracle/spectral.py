"""Component oracles for the spectral index -- TEST INFRASTRUCTURE ONLY.

Each function is the plain FP64 statement of one step of the method, in the
paper's notation, with no blocking or fusion.

* ``kprime`` / ``dft_features``: X_{i,m,k} = sum_r t_{i+r} e^{-2 pi i k r/m},
  F_{i,m} = (X_{i,m,1..K'}) / sigma_{i,m}, K' = min(K-1, ceil(m/2)-1),
  zero-padded to K-1 bins (Sec. 3.2).  Layout of a feature row: 2(K-1) reals
  [Re X_1, Im X_1, Re X_2, Im X_2, ...] / sigma.
* ``lower_bound``: LB^2 = (2/m) sum_{k<=K'} |F_i,k - F_j,k|^2 (Lemma 2).
* ``philox4x32_10`` / ``projections``: seeded Gaussian projections g_{a,l}
  (Sec. 3.4).  Philox-4x32-10 follows its published definition (Salmon et
  al., SC'11); Box-Muller maps pairs of uniforms to Gaussians.
* ``signature``: bit l = 1{<g_{a,l}, F> >= 0}, l = 1..B, bit 1 the most
  significant of the B-bit key (Sec. 3.4).
* ``depth``: global depth after P insertions, split while P > alpha 2^d and
  d < B (Sec. 3.4, Prop. 4).
* ``probe_buckets``: exact prefix bucket, then 1 + max(0, d - d0) Hamming-1
  buckets in increasing projection margin, capped by d and an implementation
  limit (Sec. 3.4).
* ``budget_select``: when a bucket has more valid entries than the remaining
  budget r, half of r takes the most recent entries and half takes entries
  at even intervals (Sec. 3.4).
* ``sieve_pairs``: pairs within w positions in the projected sort order of a
  hot class (Sec. 3.6).
* ``completion_triples``: the re-cut box of one seed (Sec. 3.6).
* ``stream_population``: the directory population a query sees under the
  batched schedule of Algorithm 1 (Sec. 3.5).

Readings of points the paper leaves open:
the prefix is bits 1..d of the signature, read as an integer with bit 1 most
significant; the initial depth is 0; the Hamming-1 cap is 8; margin ties go
to the lower bit index; the even-interval half of the budget spreads over the
entries not already taken as most recent,
v[floor(t * (s - ceil(r/2)) / floor(r/2))], t = 0..floor(r/2)-1; the Philox
counter for projection l of anchor a, dimensions 4c..4c+3, is
(c, l, a, 0x50414E43) under key (seed mod 2^32, seed div 2^32); the sieve
direction is l = B + 1.
"""
from __future__ import annotations

import math

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
PROJ_TAG = 0x50414E43


def kprime(m: int, K: int = 16) -> int:
    """Number of retained non-DC bins at length m (Sec. 3.2)."""
    return max(0, min(K - 1, (m + 1) // 2 - 1))


def anchors(m_min: int, m_max: int, s: int = 2) -> list[int]:
    """A = {m_min + r s <= m_max} U {m_max} (Sec. 3.3)."""
    a = list(range(m_min, m_max + 1, s))
    if a[-1] != m_max:
        a.append(m_max)
    return a


def dft_features(x, m: int, K: int = 16, rows=None) -> np.ndarray:
    """F_{i,m} for every window (or the listed starts), shape [nw, 2(K-1)], FP64."""
    x = np.asarray(x, dtype=np.float64)
    nw = x.shape[0] - m + 1
    idx = np.arange(nw) if rows is None else np.asarray(rows)
    kp = kprime(m, K)
    r = np.arange(m)
    k = np.arange(1, kp + 1)
    tw = np.exp(-2j * np.pi * np.outer(r, k) / m)            # [m, K']
    out = np.zeros((idx.shape[0], 2 * (K - 1)))
    step = 65536
    for s0 in range(0, idx.shape[0], step):
        ii = idx[s0:s0 + step]
        W = x[ii[:, None] + r[None, :]]                       # windows [b, m]
        mu = W.mean(axis=1)
        sg = np.sqrt(((W - mu[:, None]) ** 2).mean(axis=1))
        X = W @ tw                                            # [b, K']
        with np.errstate(divide="ignore", invalid="ignore"):
            Fz = X / sg[:, None]
        out[s0:s0 + ii.shape[0], 0:2 * kp:2] = Fz.real
        out[s0:s0 + ii.shape[0], 1:2 * kp:2] = Fz.imag
    return out


def full_dft_znorm(w) -> np.ndarray:
    """All m DFT bins of the z-normalised window w (used by the pins)."""
    w = np.asarray(w, dtype=np.float64)
    z = (w - w.mean()) / w.std()
    return np.fft.fft(z)


def lower_bound(Fi, Fj, m: int) -> np.ndarray:
    """Parseval lower bound LB_{K,m}(i,j) (Lemma 2); broadcasts over rows."""
    Fi = np.asarray(Fi, dtype=np.float64)
    Fj = np.asarray(Fj, dtype=np.float64)
    return np.sqrt((2.0 / m) * np.sum((Fi - Fj) ** 2, axis=-1))


def _mulhilo(a: int, b: np.ndarray):
    p = np.uint64(a) * b.astype(np.uint64)
    return (p >> np.uint64(32)).astype(np.uint32), (p & np.uint64(0xFFFFFFFF)).astype(np.uint32)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox-4x32 with 10 rounds.  ctr: [N,4] uint32, key: [N,2] or [2] uint32."""
    c = np.array(ctr, dtype=np.uint32).reshape(-1, 4).copy()
    k = np.broadcast_to(np.array(key, dtype=np.uint32).reshape(-1, 2), (c.shape[0], 2)).copy()
    for rnd in range(10):
        hi0, lo0 = _mulhilo(PHILOX_M0, c[:, 0])
        hi1, lo1 = _mulhilo(PHILOX_M1, c[:, 2])
        c = np.stack([hi1 ^ c[:, 1] ^ k[:, 0], lo1, hi0 ^ c[:, 3] ^ k[:, 1], lo0], axis=1)
        if rnd < 9:
            k[:, 0] = (k[:, 0].astype(np.uint64) + PHILOX_W0).astype(np.uint32)
            k[:, 1] = (k[:, 1].astype(np.uint64) + PHILOX_W1).astype(np.uint32)
    return c


def box_muller(u0: np.ndarray, u1: np.ndarray):
    """Two standard normals from two uint32 draws: u0 -> (0,1], u1 -> [0,1)."""
    a = (u0.astype(np.float64) + 1.0) * 2.0 ** -32
    b = u1.astype(np.float64) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(a))
    return r * np.cos(2.0 * np.pi * b), r * np.sin(2.0 * np.pi * b)


def projections(a: int, seed: int, B: int = 24, K: int = 16) -> np.ndarray:
    """Gaussian projections g_{a,l}, l = 1..B+1, shape [B+1, 2(K-1)], FP64.

    Row l-1 holds g_{a,l}; row B is the sieve direction.
    """
    dims = 2 * (K - 1)
    groups = (dims + 3) // 4
    ls = np.repeat(np.arange(1, B + 2), groups)
    cs = np.tile(np.arange(groups), B + 1)
    ctr = np.stack([cs, ls, np.full_like(ls, a), np.full_like(ls, PROJ_TAG)], axis=1).astype(np.uint32)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    o = philox4x32_10(ctr, key)
    g0, g1 = box_muller(o[:, 0], o[:, 1])
    g2, g3 = box_muller(o[:, 2], o[:, 3])
    g = np.stack([g0, g1, g2, g3], axis=1).reshape(B + 1, groups * 4)
    return g[:, :dims]


def margins(F, g, B: int = 24) -> np.ndarray:
    """Projections <g_{a,l}, F> for l = 1..B, shape [..., B]."""
    return np.asarray(F, dtype=np.float64) @ np.asarray(g[:B], dtype=np.float64).T


def signature(F, g, B: int = 24) -> np.ndarray:
    """B-bit SimHash key, bit l = 1{<g_l, F> >= 0}, bit 1 most significant."""
    bits = (margins(F, g, B) >= 0.0).astype(np.uint64)
    w = (np.uint64(1) << np.arange(B - 1, -1, -1, dtype=np.uint64))
    return (bits * w).sum(axis=-1).astype(np.uint32)


def depth(P: int, alpha: int = 16, B: int = 24, d_init: int = 0) -> int:
    """Global depth after P insertions (split while P > alpha 2^d and d < B)."""
    d = d_init
    while P > alpha * (1 << d) and d < B:
        d += 1
    return d


def prefix(sig, d: int, B: int = 24):
    """The d-bit bucket address of a B-bit key."""
    return np.asarray(sig, dtype=np.uint32) >> np.uint32(B - d) if d > 0 else np.zeros_like(
        np.asarray(sig, dtype=np.uint32))


def probe_count(d: int, d0: int = 12, cap: int = 8) -> int:
    """Hamming-1 probes at depth d: 1 + max(0, d - d0), capped by d and cap."""
    if d <= 0:
        return 0
    return min(d, cap, 1 + max(0, d - d0))


def probe_buckets(sig_q: int, marg_q, d: int, B: int = 24, d0: int = 12, cap: int = 8) -> list[int]:
    """Bucket addresses a query probes, in order (exact prefix first)."""
    pre = int(sig_q) >> (B - d) if d > 0 else 0
    out = [pre]
    h = probe_count(d, d0, cap)
    if h:
        mag = np.abs(np.asarray(marg_q, dtype=np.float64)[:d])
        order = sorted(range(d), key=lambda l: (mag[l], l))[:h]
        for l in order:                      # l is 0-based: bit l+1 of the key
            out.append(pre ^ (1 << (d - 1 - l)))
    return out


def budget_select(s: int, r: int) -> list[int]:
    """Positions taken from a bucket of s valid entries (ascending start) under budget r."""
    if s <= r:
        return list(range(s))
    if r <= 0:
        return []
    h1 = (r + 1) // 2
    h2 = r // 2
    rest = s - h1
    even = [(t * rest) // h2 for t in range(h2)]
    return even + list(range(s - h1, s))


def sieve_pairs(members, proj, excl: int, w: int = 8) -> list[tuple[int, int]]:
    """S_hot(C): members sorted by projection (ties by start); pairs within w positions, valid only."""
    members = np.asarray(members)
    proj = np.asarray(proj)
    order = np.lexsort((members, proj))
    pi = members[order]
    out = []
    for u in range(pi.shape[0]):
        for v in range(u + 1, min(pi.shape[0], u + w + 1)):
            if abs(int(pi[u]) - int(pi[v])) >= excl:
                out.append((min(int(pi[u]), int(pi[v])), max(int(pi[u]), int(pi[v]))))
    return out


def completion_triples(m0: int, i0: int, j0: int, n: int, m_min: int, m_max: int, excl: int,
                       dm: int = 6, dp: int = 4):
    """Admissible (m, i, j) of one seed's re-cut box (Sec. 3.6), clipped to valid ranges."""
    out = []
    for m in range(max(m_min, m0 - dm), min(m_max, m0 + dm) + 1):
        hi = n - m
        for i in range(max(0, i0 - dp), min(hi, i0 + dp) + 1):
            for j in range(max(0, j0 - dp), min(hi, j0 + dp) + 1):
                if abs(i - j) >= excl:
                    out.append((m, i, j))
    return out


def stream_population(q: int, a: int, n: int, beta: int, nonconst_prefix) -> int:
    """Directory population seen by query q of anchor a (Sec. 3.5).

    The batch holding sample tau = q + a - 1 (batches of beta samples from
    tau = 0) is inserted in full before its searches; the population counts
    the non-constant windows inserted so far.  ``nonconst_prefix[t]`` is the
    number of non-constant windows with start < t.
    """
    tau = q + a - 1
    tau_end = min(n - 1, (tau // beta + 1) * beta - 1)
    last = tau_end - a + 1
    return int(nonconst_prefix[last + 1])


F32_EPS = 2.0 ** -24


def lb_safe_threshold(m: int, eps: float = F32_EPS, lam: float = 1e-4) -> float:
    """Lemma 5: the (1 - lambda) shrink keeps the bound valid above sqrt(2m) 2 sqrt(2) eps / lambda."""
    return math.sqrt(2.0 * m) * 2.0 * math.sqrt(2.0) * eps / lam


def lb_inflation_bound(m: int, eps: float = F32_EPS) -> float:
    """Proof of Lemma 5: absolute inflation of the computed bound is at most 4 sqrt(m) eps."""
    return 4.0 * math.sqrt(m) * eps
