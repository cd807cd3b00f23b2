import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")


@pytest.fixture(scope="session")
def cfg_small():
    """The small exact case: planted random walk, n=8192, m=32..64, excl=64."""
    import workloads
    return workloads.planted_random_walk()


@pytest.fixture(scope="session")
def cfg_small_exact(cfg_small):
    from oracle import exact
    return exact.pmp(cfg_small.x, cfg_small.m_min, cfg_small.m_max, cfg_small.excl, tier="diag")
