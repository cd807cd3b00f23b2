"""Seeded synthetic workloads (input generation only, no method arithmetic)."""
from .generators import (Planted, Series, batched_series, batched_workload, ecg_like,  # noqa: F401
                         plant_shape, planted_random_walk, random_walk, sine_mix,
                         wafer_like, windows_lengths)
