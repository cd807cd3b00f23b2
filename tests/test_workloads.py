"""The seeded generators are deterministic and shaped as documented."""
import numpy as np

import workloads


def test_planted_walk_deterministic():
    a = workloads.planted_random_walk()
    b = workloads.planted_random_walk()
    assert a.x.dtype == np.float64 and a.x.shape == (8192,)
    assert np.array_equal(a.x, b.x)
    assert len(a.planted) == 3
    starts = sorted(s for p in a.planted for s in p.starts)
    assert min(np.diff(starts)) >= 48 + 64
    assert workloads.windows_lengths(8192, 32, 64) == 268785


def test_wafer_like_shape():
    s = workloads.wafer_like(100_000, seed=3)
    assert s.x.dtype == np.float32 and s.x.shape == (100_000,)
    assert np.array_equal(s.x, workloads.wafer_like(100_000, seed=3).x)
    assert (s.m_min, s.m_max, s.excl, s.k) == (100, 150, 150, 20)
    assert abs(float(s.x.mean())) < 2.0
    assert workloads.windows_lengths(1_000_000, 100, 150) == 50_993_676
    assert workloads.windows_lengths(5_000_000, 100, 150) == 254_993_676


def test_batched_subset_matches_full():
    full = workloads.batched_workload(6, seed=1, n_hi=20000)
    sub = workloads.batched_workload(6, seed=1, n_hi=20000, indices=[4])
    assert np.array_equal(full[4].x, sub[0].x)
    for s in full:
        assert 2000 <= s.x.shape[0] <= 20000
        assert 16 <= s.m_min <= 128 and 20 <= s.m_max - s.m_min + 1 <= 64
        assert s.excl == s.m_max and s.k == 10


def test_autotune_shape_key_classes():
    """Requests of one shape class (length to the nearest power of two, the
    length interval, the sample type) share one tuned configuration."""
    import numpy as np
    from paper_2607_17481_b300 import autotune
    k = autotune.shape_key
    assert k(40_000, 100, 150, np.float32) == k(45_000, 100, 150, np.float32)
    assert k(40_000, 100, 150, np.float32) != k(80_000, 100, 150, np.float32)
    assert k(40_000, 100, 150, np.float32) != k(40_000, 100, 151, np.float32)
    assert k(40_000, 100, 150, np.float32) != k(40_000, 100, 150, np.float64)
