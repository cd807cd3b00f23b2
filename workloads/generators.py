"""Seeded synthetic series shaped like the workloads of the Panache paper.

This module holds input generators only: no step of the motif method lives
here.  Both the CPU oracle tests and the CUDA path read the arrays it
produces, so the two sides always see the same bytes.

Every generator takes an explicit ``seed`` and draws from numpy's PCG64
(``default_rng``) in a fixed order, so a (generator, seed, size) triple names
one array forever.

Workloads (the paper evaluates on UCR data, which is not available here; these
synthetic stand-ins take its place, see Sec. 4 "Evaluation"):

* ``planted_random_walk``  -- random walk with planted motif pairs
  (the small exact single-series case, lengths 32..64).
* ``wafer_like``           -- concatenated 152-sample step/plateau segments
  drawn from two templates, shaped like the Wafer trace of Sec. 4 that the
  paper tiles up to 5M samples.
* ``ecg_like``, ``sine_mix`` and ``random_walk`` -- the per-series
  generators of the batched workload.
* ``batched_workload``     -- many independent series with their own
  length intervals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PLANT_LEN = 48


def plant_shape(f: float, phi: float, length: int = PLANT_LEN) -> np.ndarray:
    """Gaussian-windowed sine of amplitude 3 used for planted motifs."""
    r = np.arange(length, dtype=np.float64)
    c = 0.5 * (length - 1)
    w = 8.0 * length / PLANT_LEN
    return 3.0 * np.exp(-0.5 * ((r - c) / w) ** 2) * np.sin(2.0 * np.pi * f * r / length + phi)


def _pick_starts(rng: np.random.Generator, n: int, count: int, length: int, gap: int) -> list[int]:
    """Rejection-sample ``count`` starts in [1, n-length) at least ``gap`` apart."""
    starts: list[int] = []
    tries = 0
    while len(starts) < count:
        tries += 1
        if tries > 100000:
            raise ValueError("series too short for the requested planted motifs")
        p = int(rng.integers(1, n - length))
        if all(abs(p - s) >= gap for s in starts):
            starts.append(p)
    return starts


def _walk_with_plants(inc: np.ndarray, plants: list[tuple[int, np.ndarray]]) -> np.ndarray:
    """Random walk from increments, with segments replaced by planted shapes.

    A planted segment starting at p replaces x[p .. p+len) by
    x[p-1] + shape (the caller adds the noise into ``shape``); the walk then
    continues from the last planted sample.
    """
    n = inc.shape[0]
    x = np.empty(n, dtype=np.float64)
    pos = 0
    last = 0.0
    for p, seg in sorted(plants, key=lambda t: t[0]):
        if p > pos:
            x[pos:p] = last + np.cumsum(inc[pos:p])
            last = x[p - 1]
        x[p:p + seg.shape[0]] = last + seg
        pos = p + seg.shape[0]
        last = x[pos - 1]
    if pos < n:
        x[pos:] = last + np.cumsum(inc[pos:])
    return x


@dataclass
class Planted:
    """A planted motif pair: both starts and the shape length."""
    starts: tuple[int, int]
    length: int


@dataclass
class Series:
    x: np.ndarray
    m_min: int
    m_max: int
    excl: int
    k: int
    planted: list[Planted] = field(default_factory=list)
    kind: str = ""


def planted_random_walk(n: int = 8192, seed: int = 0, pairs: int = 3) -> Series:
    """n-sample float64 random walk (cumsum of N(0,1)) with planted pairs.

    Draw order: increments N(0,1)[n]; per pair its phase U(0, 2*pi);
    2*pairs starts at least 48+64 apart; N(0, 0.05) noise per planted sample.
    Pair p uses frequency 2+p cycles per 48 samples; a motif is inserted by
    replacement (the walk resumes from the last planted sample).
    """
    rng = np.random.default_rng(seed)
    inc = rng.standard_normal(n)
    phis = rng.uniform(0.0, 2.0 * np.pi, size=pairs)
    starts = _pick_starts(rng, n, 2 * pairs, PLANT_LEN, PLANT_LEN + 64)
    plants = []
    planted = []
    for p in range(pairs):
        shape = plant_shape(2.0 + p, float(phis[p]))
        a, b = starts[2 * p], starts[2 * p + 1]
        for s in (a, b):
            plants.append((s, shape + rng.normal(0.0, 0.05, PLANT_LEN)))
        planted.append(Planted((min(a, b), max(a, b)), PLANT_LEN))
    x = _walk_with_plants(inc, plants)
    return Series(x=x, m_min=32, m_max=64, excl=64, k=20, planted=planted, kind="planted_random_walk")


def wafer_templates(rng: np.random.Generator, count: int = 2, length: int = 152) -> np.ndarray:
    """Step/plateau templates: S~U{3..8} plateaus, sorted change points, levels U(-2,2)."""
    out = np.empty((count, length), dtype=np.float64)
    for t in range(count):
        s = int(rng.integers(3, 9))
        cps = np.sort(rng.choice(np.arange(1, length), size=s - 1, replace=False))
        levels = rng.uniform(-2.0, 2.0, size=s)
        bounds = np.concatenate(([0], cps, [length]))
        for q in range(s):
            out[t, bounds[q]:bounds[q + 1]] = levels[q]
    return out


def wafer_like(n: int = 1_000_000, seed: int = 0, dtype=np.float32) -> Series:
    """Wafer-like sensor trace: concatenated 152-sample template segments.

    Draw order: the two templates; per segment its template U{0,1};
    scale U(0.8,1.2)[segments]; offset N(0,0.1)[segments]; noise
    N(0,0.05)[segments*152].  Lengths 100..150, exclusion 150, top-20.
    """
    rng = np.random.default_rng(seed)
    tpl = wafer_templates(rng)
    L = tpl.shape[1]
    segs = (n + L - 1) // L
    which = rng.integers(0, tpl.shape[0], size=segs)
    scale = rng.uniform(0.8, 1.2, size=segs)
    offset = rng.normal(0.0, 0.1, size=segs)
    noise = rng.normal(0.0, 0.05, size=(segs, L))
    x = tpl[which] * scale[:, None] + offset[:, None] + noise
    x = x.reshape(-1)[:n].astype(dtype)
    return Series(x=x, m_min=100, m_max=150, excl=150, k=20, kind="wafer_like")


# Per-beat (amplitude, centre, width) of the P, QRS and T waves, as fractions
# of the beat period (centre, width) and in signal units (amplitude).
_ECG_WAVES = ((0.15, 0.20, 0.035), (1.20, 0.40, 0.012), (0.35, 0.68, 0.060))


def random_walk(rng: np.random.Generator, n: int) -> np.ndarray:
    return np.cumsum(rng.standard_normal(n))


def ecg_like(rng: np.random.Generator, n: int) -> np.ndarray:
    """Beats as sums of three Gaussians; period U(150,300) with 5% jitter per beat."""
    period = rng.uniform(150.0, 300.0)
    x = np.zeros(n, dtype=np.float64)
    t = 0.0
    while t < n:
        p = period * (1.0 + rng.uniform(-0.05, 0.05))
        lo = int(t)
        hi = min(n, int(t + p) + 1)
        r = np.arange(lo, hi, dtype=np.float64) - t
        for amp, c, w in _ECG_WAVES:
            x[lo:hi] += amp * np.exp(-0.5 * ((r - c * p) / (w * p)) ** 2)
        t += p
    return x + rng.normal(0.0, 0.02, n)


def sine_mix(rng: np.random.Generator, n: int) -> np.ndarray:
    """Three sines with periods U(20,500) plus N(0, 0.2) noise."""
    r = np.arange(n, dtype=np.float64)
    x = np.zeros(n)
    for _ in range(3):
        per = rng.uniform(20.0, 500.0)
        x += rng.uniform(0.5, 1.5) * np.sin(2.0 * np.pi * r / per + rng.uniform(0, 2 * np.pi))
    return x + rng.normal(0.0, 0.2, n)


_KINDS = ("random_walk", "ecg_like", "sine_mix")


def batched_series(rng: np.random.Generator, n: int) -> Series:
    """One series of the batched workload (generator, interval, plants)."""
    kind = _KINDS[int(rng.integers(0, 3))]
    x = {"random_walk": random_walk, "ecg_like": ecg_like, "sine_mix": sine_mix}[kind](rng, n)
    m_min = int(rng.integers(16, 129))
    span = int(rng.integers(20, 65))
    m_max = m_min + span - 1
    n_plant = int(rng.integers(0, 6))
    planted = []
    for _ in range(n_plant):
        length = int(rng.integers(m_min, m_max + 1))
        try:
            a, b = _pick_starts(rng, n, 2, length, length + m_max)
        except ValueError:
            break
        shape = plant_shape(float(rng.integers(2, 5)), float(rng.uniform(0, 2 * np.pi)), length)
        scale = float(np.std(x)) + 1e-3
        for s in (a, b):
            x[s:s + length] = x[s - 1] + scale * shape / 3.0 + rng.normal(0.0, 0.05 * scale, length)
        planted.append(Planted((min(a, b), max(a, b)), length))
    return Series(x=x.astype(np.float32), m_min=m_min, m_max=m_max, excl=m_max, k=10,
                  planted=planted, kind=kind)


def batched_workload(count: int = 4096, seed: int = 0, n_lo: int = 2000, n_hi: int = 200_000,
                     indices=None) -> list[Series]:
    """``count`` independent series with log-uniform lengths in [n_lo, n_hi].

    Series s is drawn from its own child generator (seed, s), so any subset
    (``indices``) is generated without drawing the others.
    """
    out = []
    idx = range(count) if indices is None else indices
    for s in idx:
        rng = np.random.default_rng([seed, int(s)])
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        out.append(batched_series(rng, n))
    return out


def windows_lengths(n: int, m_min: int, m_max: int) -> int:
    """W = sum over m in [m_min, m_max] of (n - m + 1): the metric's unit count."""
    return sum(max(0, n - m + 1) for m in range(m_min, m_max + 1))
