"""Host-side pieces of the benchmark that need no GPU: the algorithmic byte
and flop counts, the workload names the JSON line carries, the measured HBM
peak (and its fallback), the traffic table's keys, and the CPU baseline
(the oracle timed on whole steps) for both storage types."""
from __future__ import annotations

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_counts():
    # read + write of the upper triangle with its diagonal, one read of V
    assert bench.alg_bytes(5000, 16) == 8 * 5000 * 5001 + 8 * 5000 * 16
    assert bench.alg_bytes(8192, 16, 4) == 4 * 8192 * 8193 + 4 * 8192 * 16
    # 4 flops per element and vector for the rotation, 6 per row and vector for Compute
    assert bench.alg_flops(3, 2) == 2 * (2 * 3 * 2 + 6 * 3)


def test_workload_names():
    assert bench.workload_name(bench.N, bench.K, "f64").endswith("(paper headline shape)")
    assert "headline" not in bench.workload_name(32768, 16, "f64")
    assert "float32 storage + float64 Compute" in bench.workload_name(16384, 16, "f32")


def test_measured_peak_and_fallback(tmp_path, monkeypatch):
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6000.5}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.measured_hbm_gbs()
    assert peak == 6000.5 and src.startswith("measured")
    (tmp_path / "MEASURED_PEAKS.json").unlink()
    peak, src = bench.measured_hbm_gbs()
    assert peak == 6800.0 and src.startswith("fallback")


def test_traffic_table_keys():
    for key, traffic in bench.NCU_TRAFFIC.items():
        kernel, source_hash, n, k = key
        assert kernel in ("wave_kernel<double>", "wave_kernel<float>")
        assert len(source_hash) == 16 and int(source_hash, 16) >= 0
        elt = 8 if kernel == "wave_kernel<double>" else 4
        # a launch moves at least the algorithmic bytes, and not many times more
        assert bench.alg_bytes(n, k, elt) <= traffic <= 4 * bench.alg_bytes(n, k, elt)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_cpu_baseline_runs_whole_steps(dtype):
    import oracle
    oracle.build()
    cb, per_step = bench.cpu_baseline(96, 3, max_steps=2, dtype=dtype)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == bench.UNIT
    assert per_step > 0
    elt = 4 if dtype == "f32" else 8
    assert cb["value"] == pytest.approx(2 * bench.alg_bytes(96, 3, elt) / per_step / 1e9)
    assert ("float32 storage" in cb["sample"]) == (dtype == "f32")


def test_launches_per_modification_follow_the_settings():
    """The launch count the JSON line claims: the wave kernel once per 64
    vectors; a fused pass two launches per block of vectors (8 in float, 4 in
    float64 by default), a six-kernel pass six."""
    from paper_1011_1173_gb300 import chm
    assert bench.launches_per_modification(chm.PATH_WAVE, 16) == 1
    assert bench.launches_per_modification(chm.PATH_WAVE, 65) == 2
    assert bench.launches_per_modification(chm.PATH_PASS, 1, "f32") == 2
    assert bench.launches_per_modification(chm.PATH_PASS, 16, "f32") == 4
    assert bench.launches_per_modification(chm.PATH_PASS, 16, "f64") == 8
    chm.config_set("pass_fused", 0)
    try:
        assert bench.launches_per_modification(chm.PATH_PASS, 16, "f32") == 12
    finally:
        chm.config_set("pass_fused", 1)
    chm.config_set("pass_kb", 16)
    try:
        assert bench.launches_per_modification(chm.PATH_PASS, 16, "f32") == 6
    finally:
        chm.config_set("pass_kb", 0)
