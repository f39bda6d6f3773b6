"""Host logic of bench.py that needs no GPU: the per-launch DRAM traffic of a
kernel class is reported only while the sources recorded with it are
unchanged, the roofline peaks come from the measured file (sustained BF16
where present, TF32 and FP64 by the nominal ratios), and the clock sampler's
summary flags the throttle reasons it saw."""
import hashlib
import json
import os

import bench


def _tree(tmp_path, src_text):
    csrc = tmp_path / "paper_1612_03804_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_record_follows_its_sources(tmp_path, monkeypatch):
    csrc = _tree(tmp_path, "kernel v1\n")
    sha = hashlib.sha256(b"kernel v1\n").hexdigest()[:16]
    rec = {"gemm_tc": {"sources": ["k.cu"], "sha": sha, "launches": 3, "bytes_per_launch": 1.5e6}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.traffic_record("gemm_tc")
    assert got is not None and got["bytes_per_launch"] == 1.5e6
    assert bench.traffic_record("gemm_oz") is None
    (csrc / "k.cu").write_text("kernel v2\n")
    assert bench.traffic_record("gemm_tc") is None
    os.remove(csrc / "k.cu")
    assert bench.traffic_record("gemm_tc") is None


def test_traffic_record_without_a_file(tmp_path, monkeypatch):
    _tree(tmp_path, "x")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_record("gemm_tc") is None


def test_peaks_prefer_sustained_and_derive_other_types(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps(
        {"hbm_gbs": 6000.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}))
    p = bench.peaks()
    assert p["source"] == "measured (sustained)"
    assert p["bf16_tflops"] == 1700.0 and p["hbm_gbs"] == 6000.0
    assert abs(p["tf32_tflops"] - 1700.0 * 1100 / 2250) < 1e-9
    assert abs(p["fp64_tflops"] - 1700.0 * 1.25 / 2250) < 1e-12
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"nested": {"bf16_tflops": 1800.0}}))
    p = bench.peaks()
    assert p["source"] == "measured (burst)" and p["bf16_tflops"] == 1800.0
    os.remove(tmp_path / "MEASURED_PEAKS.json")
    assert bench.peaks()["source"] == "fallback"


def test_clock_summary_flags_throttle_reasons():
    cs = bench.ClockSampler(0)
    cs.lines = [
        "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbled line",
        "0, [N/A], 2070, 0, 0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = cs.stop()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_weak_scaling_value_counts_all_ranks():
    assert bench.weak_scaling_value(256, 4, 2.0) == 512.0
    assert bench.max_over_ranks(3.5) == 3.5
