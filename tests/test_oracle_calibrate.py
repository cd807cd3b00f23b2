"""Pins of the spectral-width calibration oracle (Sec. 3.2, "Spectral width
selection") against closed forms, not against a retyping of its formulas."""
import math

import numpy as np

from oracle import calibrate, spectral


def test_white_noise_energy_closed_form():
    # z-normalised i.i.d. noise spreads its energy m^2 evenly over the m - 1
    # non-DC bins, so E[(2/m^2) sum_{k<=K'} |X^_k|^2] = 2 K' / (m - 1)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(60_000)
    m = 100
    energy, _, _ = calibrate.statistics(x, m, m, K_max=16)
    for t, K in enumerate(range(2, 17)):
        want = 2.0 * spectral.kprime(m, K) / (m - 1)
        # 256 windows: the sample mean is within ~4 standard errors of the expectation
        assert abs(energy[t] - want) <= 4.0 * want * math.sqrt(2.0 / (256 * 2 * spectral.kprime(m, K))) + 1e-12


def test_pure_tone_energy_is_a_step():
    # a sinusoid of period 20: a window of length m holds it entirely in bin m / 20
    n = 4000
    x = np.sin(2 * np.pi * np.arange(n) / 20.0 + 0.3)
    energy, _, _ = calibrate.statistics(x, 40, 80, K_max=16)   # lengths 40, 60, 80: bins 2, 3, 4
    want = {2: 0.0, 3: 1 / 3, 4: 2 / 3, 5: 1.0}
    for K, w in want.items():
        assert abs(energy[K - 2] - w) < 1e-9, (K, energy[K - 2])
    assert np.all(np.abs(energy[3:] - 1.0) < 1e-9)


def test_pure_tone_collision_closed_form():
    # one bin carries the whole feature: the angle between the windows at s1, s2
    # is the phase difference 2 pi k (s2 - s1) / m folded into [0, pi]; pairs
    # a whole number of periods apart are identical and are near-duplicates
    n, P, m, B = 5000, 25, 50, 24
    x = np.cos(2 * np.pi * np.arange(n) / P)
    starts = calibrate.sample_starts(x, m)
    tot, cnt = 0.0, 0
    for a in range(len(starts)):
        for b in range(a + 1, len(starts)):
            ph = (2 * np.pi * (starts[b] - starts[a]) / P) % (2 * np.pi)
            th = min(ph, 2 * np.pi - ph)
            lb = math.sqrt((2.0 / m) * 2 * (m / 2) ** 2 * (2 - 2 * math.cos(th)))   # |F_i - F_j| at |X^_k| = m/2
            if lb < 0.1 * math.sqrt(2 * m):
                continue
            tot += (1 - th / math.pi) ** B
            cnt += 1
    _, coll, pairs = calibrate.statistics(x, m, m, B=B, K_max=16)
    assert pairs == cnt
    for K in range(3, 17):                       # bin 2 = m / P is retained from K = 3
        assert abs(coll[K - 2] - tot / cnt) < 1e-9 * max(1.0, tot / cnt)


def test_selection_rule():
    energy = np.array([0.5, 0.8, 0.86, 0.9, 0.95] + [0.99] * 10)
    coll = np.array([1e-2, 1e-3, 1e-3, 1e-6, 1e-7] + [1e-8] * 10)
    # K = 4 meets the energy condition but not the collision one at n = 1e6 (1000 > 256)
    assert calibrate.select_width(energy, coll, 1_000_000) == 5
    assert calibrate.select_width(energy, coll, 100_000) == 4
    assert calibrate.select_width(energy, coll, 100, eta=0.999) == 16          # nothing qualifies
    assert calibrate.select_width(energy, coll, 100, eta=0.5) == 2


def test_sampling_rule():
    x = np.arange(1000, dtype=float)
    s = calibrate.sample_starts(x, 100)
    assert s[0] == 0 and s[-1] == 900 and len(s) == 256 and np.all(np.diff(s) > 0)
    y = x.copy()
    y[0:150] = 1.0                               # windows inside the constant run are dropped
    s2 = calibrate.sample_starts(y, 100)
    assert np.all(s2 > 50) and len(s2) == len(s) - np.sum(s <= 50)
    assert calibrate.calibration_lengths(32, 32) == [32]
    assert calibrate.calibration_lengths(32, 64) == [32, 48, 64]
