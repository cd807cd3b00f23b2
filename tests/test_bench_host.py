"""Host-side arithmetic of the benchmark line (no GPU).

The roofline object divides the search's algorithmic bytes -- a 128-byte
feature row per query and per inspected candidate -- by its mean launch time,
against the HBM copy peak; the DRAM traffic figure comes from the committed
ncu record only while the kernel's sources still hash to the captured ones.
"""
import hashlib
import json
import os

import pytest

import bench


def _stats(queries, candidates, search_ms, features_ms=1.0):
    return {"queries": queries, "candidates": candidates,
            "step_ms": {"search": search_ms, "features": features_ms}}


def test_roofline_arithmetic():
    steps = [_stats(1_000_000, 99_000_000, 2.0), _stats(1_000_000, 99_000_000, 4.0)]
    r = bench.roofline(steps, {"hbm_gbs": 8000.0}, "measured", None)
    # 128 B x (1e6 + 99e6) per launch over a 3 ms mean launch: 4266.7 GB/s
    assert r["bytes_per_launch"] == 128.0 * 100_000_000
    assert r["achieved"] == pytest.approx(128.0 * 1e8 / 3e-3 / 1e9, rel=1e-4)
    assert r["frac"] == pytest.approx(4266.67 / 8000.0, rel=1e-3)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None
    assert r["peak_source"].startswith("measured")


def test_peaks_fall_back_when_unmeasured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peaks, src = bench.measured_peaks()
    assert src == "fallback" and peaks["hbm_gbs"] == 6400.0
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6469.6, "bf16_tflops": 1839.8}))
    peaks, src = bench.measured_peaks()
    assert src == "measured" and peaks["hbm_gbs"] == 6469.6


def test_traffic_record_follows_kernel_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_traffic(10) is None                       # no record
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel v1")
    os.makedirs(tmp_path / "profiles")
    rec = {"k_search": {"dram_bytes_per_query": 352.0,
                        "sources_sha256_16": {"k.cu": hashlib.sha256(b"kernel v1").hexdigest()[:16]}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.measured_traffic(1000) == pytest.approx(352000.0)
    src.write_bytes(b"kernel v2")                                   # source changed since the capture
    assert bench.measured_traffic(1000) is None


def test_kernel_table_arithmetic():
    """Per-kernel fractions: algorithmic flops and bytes per request over the
    kernel's event time, against the measured FP32 / TF32 and HBM ceilings."""
    st = {"queries": 1000, "candidates": 100_000, "exact_stream": 40_000, "exact_sieve": 8000,
          "exact_completion": 10_530, "completion_rounds": 3}
    kt = {"anchor_tc": (0.5, 1), "features": (1.0, 1), "search": (10.0, 1), "sieve": (2.0, 1),
          "complete": (1.0, 3), "select": (0.5, 4)}
    anchors = [100, 150]
    n = 10_000
    rows = {r["kernel"]: r for r in bench.kernel_table(st, kt, n, anchors, {"hbm_gbs": 8000.0},
                                                       {"fp32": 100.0, "tf32_cublas": 500.0})}
    s = rows["search"]
    assert s["flops"] == 90.0 * 100_000 + 5.0 * 125.0 * 40_000
    assert s["bytes"] == 128.0 * 101_000
    assert s["fp32_frac"] == pytest.approx(s["flops"] / 10e-3 / 1e12 / 100.0, rel=1e-3)
    assert s["hbm_frac"] == pytest.approx(s["bytes"] / 10e-3 / 1e9 / 8000.0, rel=1e-3)
    f = rows["features"]
    nwa = (n - 99) + (n - 149)
    assert f["flops"] == 1650.0 * nwa and f["bytes"] == 164.0 * nwa
    assert "tf32_frac" in rows["anchor_tc"] and "fp32_frac" not in rows["anchor_tc"]
    assert rows["select"]["bytes"] == 24.0 * 51 * n * 4


def test_paper_recovery_rule():
    """Sec. 4's recovery: position match within m/2 at the same length, else
    value match of the length's best reported distance (5% or 0.05), else missed."""
    import numpy as np
    dt = [("m", "i4"), ("i", "i8"), ("j", "i8"), ("d", "f8")]
    ref = np.array([(100, 1000, 5000, 0.30),     # reported 50 samples away: position (2*50 <= 100)
                    (100, 2000, 6000, 0.31),     # reported 51 away only: not a position match, value 0.30 vs 0.31
                    (120, 3000, 7000, 0.40),     # no cell at 120: missed
                    (101, 4000, 8000, 0.20)],    # best at 101 is 0.26: |0.06| > 0.05 and > 5%: missed
                   dtype=dt)
    got = np.array([(100, 1050, 5050, 0.30), (100, 2051, 6051, 0.35), (101, 9000, 9900, 0.26)], dtype=dt)
    r = bench.paper_recovery(ref, got)
    assert r == {"position": 1, "value": 1, "missed": 2, "of": 4}
    # the rule is per length: a cell at the right start but another length does not count
    r2 = bench.paper_recovery(ref[:1], np.array([(101, 1000, 5000, 0.30)], dtype=dt))
    assert r2 == {"position": 0, "value": 0, "missed": 1, "of": 1}
    assert bench.paper_recovery(ref, ref)["position"] == 4
