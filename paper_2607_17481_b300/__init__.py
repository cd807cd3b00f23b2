"""B300-native Panache pan-motif engine (one-pass z-normalised PMP motif search).

The compute path is the CUDA library ``libpanache.so`` (sources in
``csrc/``, C ABI in ``include/panache.h``); ``native`` is its thin ctypes
binding.  Importing the package does not load the library; the first call
that needs it does, and fails loudly if it has not been built.
"""
from .native import (DEVICE, F32, F64, FLAG_EXHAUSTIVE_SIEVE, FLAG_FP64_ANCHORS, FLAG_GRAPH,  # noqa: F401
                     FLAG_HALF_FEATURES, FLAG_INDEX_ONLY, FLAG_NO_COMPLETION, FLAG_NO_REFINE, FLAG_NO_SIEVE, FLAG_GRAM_SEARCH,
                     FLAG_SIEVE_GRAM, FLAG_TIMING, FLAG_TOPK_SIEVE, FLAG_NO_FOCUS_SIEVE, FLAG_WARM_START, MIXED, PLAIN_FP64, STEP_NAMES, TOPK_GLOBAL,
                     TOPK_PER_LENGTH, Context, PanacheError, Server, Stream, alu_peak, default_config,
                     inject_fault, unpack_keys)
