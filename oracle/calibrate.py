"""Spectral-width calibration oracle -- TEST INFRASTRUCTURE ONLY.

The width K (bins 1..K-1 retained) is fixed before insertion by a
calibration on sampled windows (Sec. 3.2, "Spectral width selection"): the
smallest K with

    E[ (2/m^2) sum_{k<=K'(m)} |X^_{i,m,k}|^2 ] >= eta          (energy)
    n E[ (1 - theta_K / pi)^B ] <= 2 gamma alpha               (collisions)

where X^ is the DFT of the z-normalised window, theta_K the angle between the
K-width features of two sampled windows, n the series length and
R = gamma alpha the verification budget.  Near-duplicate pairs do not enter
the collision estimate.  Plain FP64 numpy; each step in the paper's order.

Readings of what the paper leaves open:
* sample: at each of m_min, floor((m_min + m_max) / 2) and m_max (each length
  once), the starts floor(t (n - m) / (S - 1)), t = 0..S-1, S = min(256,
  n - m + 1), duplicates removed, constant windows (max == min) dropped;
* both expectations pool the three lengths; angles are taken between windows
  of the same length only;
* a pair is a near-duplicate when its full-width bound (K = K_max) is below
  0.1 sqrt(2m);
* a zero feature vector makes an angle of pi/2;
* when no K in [2, K_max] meets both conditions, K = K_max.
"""
from __future__ import annotations

import math

import numpy as np

from . import spectral

ETA = 0.85
SAMPLE = 256
DUP_FRAC = 0.1


def calibration_lengths(m_min: int, m_max: int) -> list[int]:
    out = []
    for m in (m_min, (m_min + m_max) // 2, m_max):
        if m not in out:
            out.append(m)
    return out


def sample_starts(x, m: int, per_length: int = SAMPLE) -> np.ndarray:
    """Evenly spaced starts of non-constant windows of length m."""
    x = np.asarray(x, dtype=np.float64)
    nw = x.shape[0] - m + 1
    if nw <= 0:
        return np.zeros(0, dtype=np.int64)
    S = min(per_length, nw)
    if S == 1:
        starts = np.zeros(1, dtype=np.int64)
    else:
        starts = np.unique((np.arange(S, dtype=np.int64) * (nw - 1)) // (S - 1))
    keep = [s for s in starts if x[s:s + m].max() != x[s:s + m].min()]
    return np.asarray(keep, dtype=np.int64)


def statistics(x, m_min: int, m_max: int, B: int = 24, K_max: int = 16, per_length: int = SAMPLE,
               dup_frac: float = DUP_FRAC):
    """(energy[K], collision_prob[K], pairs) for K = 2..K_max: the sample means of
    the two calibration conditions (collision_prob is E[(1 - theta_K/pi)^B])."""
    x = np.asarray(x, dtype=np.float64)
    Ks = list(range(2, K_max + 1))
    e_sum = np.zeros(len(Ks))
    e_cnt = 0
    c_sum = np.zeros(len(Ks))
    c_cnt = 0
    for m in calibration_lengths(m_min, m_max):
        starts = sample_starts(x, m, per_length)
        if starts.shape[0] == 0:
            continue
        F = spectral.dft_features(x, m, K_max, rows=starts)          # [S, 2(K_max-1)], = X^_{1..K'}
        for t, K in enumerate(Ks):
            kp = spectral.kprime(m, K)
            e_sum[t] += np.sum((2.0 / m ** 2) * np.sum(F[:, :2 * kp] ** 2, axis=1))
        e_cnt += starts.shape[0]
        S = starts.shape[0]
        ii, jj = np.triu_indices(S, k=1)
        lb = spectral.lower_bound(F[ii], F[jj], m)
        keep = lb >= dup_frac * math.sqrt(2.0 * m)
        ii, jj = ii[keep], jj[keep]
        c_cnt += ii.shape[0]
        for t, K in enumerate(Ks):
            kp = spectral.kprime(m, K)
            A = F[ii, :2 * kp]
            Bv = F[jj, :2 * kp]
            na = np.sqrt(np.sum(A * A, axis=1))
            nb = np.sqrt(np.sum(Bv * Bv, axis=1))
            dot = np.sum(A * Bv, axis=1)
            with np.errstate(divide="ignore", invalid="ignore"):
                cos = np.where((na > 0) & (nb > 0), dot / (na * nb), 0.0)
            theta = np.arccos(np.clip(cos, -1.0, 1.0))
            c_sum[t] += np.sum((1.0 - theta / math.pi) ** B)
    energy = e_sum / max(1, e_cnt)
    coll = c_sum / max(1, c_cnt)
    return energy, coll, c_cnt


def select_width(energy, coll, n: int, alpha: int = 16, gamma: int = 8, eta: float = ETA, K_max: int = 16) -> int:
    """Smallest K in [2, K_max] meeting both conditions, else K_max."""
    for t, K in enumerate(range(2, K_max + 1)):
        if energy[t] >= eta and n * coll[t] <= 2 * gamma * alpha:
            return K
    return K_max


def calibrate(x, m_min: int, m_max: int, B: int = 24, alpha: int = 16, gamma: int = 8, eta: float = ETA,
              K_max: int = 16):
    """(K, energy, collision_prob) for series x."""
    energy, coll, _ = statistics(x, m_min, m_max, B, K_max)
    return select_width(energy, coll, np.asarray(x).shape[0], alpha, gamma, eta, K_max), energy, coll
