"""The C-ABI library loads and exports every entry point include/panache.h declares.

No compute call is made here: this runs on machines without a GPU.
"""
import ctypes
import os
import re

import pytest

from paper_2607_17481_b300 import build, native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "panache.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(panache_[a-z_]+)\s*\(", hdr)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return native.lib()


def test_every_declared_symbol_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 16
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(native.EXPORTED)


def test_default_config_is_the_papers(lib):
    c = native.default_config()
    assert (c.alpha, c.gamma, c.stride, c.K, c.B, c.d0, c.probe_cap, c.sieve_w) == (16, 8, 0, 16, 24, 12, 8, 8)
    # stride 0: resolved by the context from the top-k mode (2 global, 1 per length)
    assert (c.dm, c.dp, c.rounds) == (6, 4, 8)
    assert c.lambda_ == 1e-4 and c.eps0 == 1e-6


def test_strerror_and_argument_errors(lib):
    assert lib.panache_strerror(0) == b"ok"
    assert b"budget" in lib.panache_strerror(native.EBUDGET)
    # null output handle / config values out of range are rejected before any device work
    assert lib.panache_create(None, None) == native.EINVAL
    bad = native.default_config(K=17)
    h = ctypes.c_void_p()
    assert lib.panache_create(ctypes.byref(bad), ctypes.byref(h)) == native.EINVAL
    bad = native.default_config(chunk=100)
    assert lib.panache_create(ctypes.byref(bad), ctypes.byref(h)) == native.EINVAL
    bad = native.default_config(alpha=64, gamma=16)        # R = 1024 > 512
    assert lib.panache_create(ctypes.byref(bad), ctypes.byref(h)) == native.EINVAL
    assert lib.panache_pmp(None, None, 2, 0, 3, 4, 1, 1, None, 0, None) == native.EINVAL
    assert lib.panache_last_stats(None, None) == native.EINVAL


def test_projection_table_matches_oracle(lib):
    """The library's host-side Philox/Box-Muller draw equals the oracle's to FP32 rounding (Sec. 3.4)."""
    import numpy as np
    from oracle import spectral
    for a, seed, K in [(48, 0, 16), (125, 12345, 16), (33, 2 ** 40 + 7, 9), (64, 1, 4)]:
        g = native.projections(a, native.default_config(seed=seed, K=K))
        ref = spectral.projections(a, seed, 24, K)
        dims = 2 * (K - 1)
        assert np.allclose(g[:, :dims], ref, rtol=2e-7, atol=1e-6)
        assert np.all(g[:, dims:] == 0.0)

def test_no_cpu_fallback_when_library_missing(tmp_path, monkeypatch):
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(native, "_lib", None)
    with pytest.raises(ImportError):
        native.lib()


def test_inject_fault_arguments():
    """The fault hook validates its arguments and disarms (no device needed)."""
    from paper_2607_17481_b300 import native
    assert native.lib().panache_inject_fault(99, 0) == native.EINVAL
    assert native.lib().panache_inject_fault(native.FAULT_ALLOC, -1) == native.EINVAL
    assert native.lib().panache_inject_fault(native.FAULT_NONE, 0) == native.OK
