"""Autotuning of the mixed form: re-anchoring period (drift) and search grid (time).

Chunk length C: the mixed form slides FP32 spectral state up to C - 1 times
from each FP64 direct-DFT anchor (Sec. 3.2 recomputes every 4096 slides).
Its features drift from the plain form's FP64 state; Lemma 5's (1 - lambda)
shrink stays valid at the paper's margin only while the drift stays near
FP32 rounding.  tune() picks the longest C whose worst relative row drift
(features at m_min and m_max of a sample of the series) stays at or below
lambda / 10, then the search grid multiple with the shortest measured
search step.  Everything runs through the C ABI on the device.
"""
from __future__ import annotations

import numpy as np

from . import native


def feature_drift(x, a: int, chunk: int, context_kw: dict | None = None):
    """(max relative row drift, drift per slide offset q mod C) at anchor length a."""
    kw = dict(context_kw or {})
    rows = {}
    for prec in (0, 1):
        ctx = native.Context(precision=prec, chunk=chunk, flags=native.FLAG_INDEX_ONLY, **kw)
        ctx.pmp(x, a, a, 1, a)
        nw = len(x) - a + 1
        _, F, _ = ctx.anchor_state(0, 0, nw)
        rows[prec] = F.astype(np.float64)
        ctx.close()
    ref = rows[0]
    norm = np.linalg.norm(ref, axis=1)
    ok = norm > 0
    rel = np.zeros(len(ref))
    rel[ok] = np.linalg.norm(rows[1][ok] - ref[ok], axis=1) / norm[ok]
    off = np.arange(len(ref)) % chunk
    curve = np.zeros(chunk)
    np.maximum.at(curve, off, rel)
    return float(rel.max()), curve


def tune(x, m_min: int, m_max: int, lam: float = 1e-4, chunks=(4096, 2048, 1024, 512, 256, 128, 64),
         grid_mults=(4, 8, 16), sample: int = 200_000, time_k: int = 20, time_excl: int | None = None) -> dict:
    x = np.ascontiguousarray(np.asarray(x)[:sample])
    drift = {}
    chosen = None
    for c in chunks:
        d = max(feature_drift(x, m_min, c)[0], feature_drift(x, m_max, c)[0])
        drift[c] = d
        if d <= lam / 10:
            chosen = c
            break
    if chosen is None:
        chosen = min(chunks)
    excl = time_excl or m_max
    times = {}
    for g in grid_mults:
        ctx = native.Context(precision=1, chunk=chosen, grid_mult=g, flags=native.FLAG_TIMING)
        ctx.pmp(x, m_min, m_max, time_k, excl)
        ctx.pmp(x, m_min, m_max, time_k, excl)
        times[g] = ctx.stats()["step_ms"]["search"]
        ctx.close()
    best_g = min(times, key=times.get)
    return {"chunk": chosen, "grid_mult": best_g, "drift": drift, "search_ms": times, "lambda": lam}


_CACHE: dict = {}


def shape_key(n: int, m_min: int, m_max: int, dtype) -> tuple:
    """Requests of one shape class share a tuned configuration: the series
    length to the nearest power of two, the length interval and the sample type."""
    return (int(np.round(np.log2(max(2, n)))), int(m_min), int(m_max), np.dtype(dtype).name)


def tuned(x, m_min: int, m_max: int, **kw) -> dict:
    """tune() once per shape class (cached for the process)."""
    x = np.asarray(x)
    key = shape_key(x.shape[0], m_min, m_max, x.dtype)
    if key not in _CACHE:
        _CACHE[key] = tune(x, m_min, m_max, **kw)
    return _CACHE[key]


def config_for_batch(series: list, params: list, sample: int = 64, **kw) -> dict:
    """The configuration one batched request runs with: the tuned chunk and
    grid multiple of the batch's largest series among the first `sample`
    (by windows x lengths), from the per-shape cache."""
    best, best_w = None, -1
    for x, (m_min, m_max, _, _) in list(zip(series, params))[:sample]:
        w = sum(max(0, len(x) - m + 1) for m in range(m_min, m_max + 1))
        if w > best_w:
            best, best_w = (x, m_min, m_max), w
    x, m_min, m_max = best
    x = x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    return tuned(x, m_min, m_max, **kw)
