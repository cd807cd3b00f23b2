"""CPU oracle for the Panache hot path -- TEST INFRASTRUCTURE ONLY.

Nothing in the product path may import this package: only ``tests/``, the
smoke check and the benchmark's CPU-baseline leg use it.  It shares no code
with the CUDA library (no headers, kernels, tables or helpers); the two meet
only through the seeded generators in ``workloads``.

Contents
  exact     -- ctypes wrappers over ``pmp_exact.c``: the exact pan matrix
               profile by definition (tier i) and by per-diagonal sliding dot
               products with the closed form (tier ii), Sec. 2.
  topk      -- zero-snap and the greedy top-k rule with the m/2 overlap skip
               (Sec. 2, Sec. 3.6).
  spectral  -- direct-DFT features, the Parseval bound, Philox-drawn SimHash
               projections and signatures, the depth rule, probe order and
               budget selection (Sec. 3.2, 3.4).
  calibrate -- the spectral-width calibration: energy and accidental-
               collision conditions on sampled windows (Sec. 3.2).

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, brute force on tiny inputs, invariants or published
known-answer vectors; none is "parity unpinned".
"""
from . import calibrate, exact, spectral, topk  # noqa: F401
