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
    rec = {"chains16": {"gemm_tc": {"sources": ["k.cu"], "sha": sha, "launches": 3, "bytes_per_launch": 1.5e6}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    got = bench.traffic_record("gemm_tc")
    assert got is not None and got["bytes_per_launch"] == 1.5e6
    assert bench.traffic_record("gemm_oz") is None
    # a record holds for the workload it was captured on only
    assert bench.traffic_record("gemm_tc", "large") is None
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


def test_roofline_entry_uses_the_operand_type_peak():
    """The dominant class's fraction is taken against the peak of its own operand type;
    the issue efficiency (peak over the MMAs of one product) is a separate field."""
    pk = {"bf16_tflops": 1700.0, "tf32_tflops": 1700.0 * 1100 / 2250, "fp64_tflops": 1700.0 * 1.25 / 2250,
          "source": "measured (sustained)"}
    prof = {"gemm_tc": {"launches": 10, "ms": 100.0, "flops": 8.31e12},
            "gemm_oz": {"launches": 5, "ms": 50.0, "flops": 1e11},
            "panel_f64": {"launches": 5, "ms": 10.0, "flops": 1e9}}
    r = bench.roofline_entry(prof, "3xtf32", pk, "nowhere")
    assert r["kernel"] == "gemm_tc" and r["bound"] == "tensor" and r["dtype"] == "tf32"
    assert abs(r["achieved"] - 83.1) < 1e-9
    assert abs(r["frac"] - 83.1 / pk["tf32_tflops"]) < 1e-12
    assert abs(r["issue_efficiency"] - 5 * r["frac"]) < 1e-12
    assert r["traffic"] is None
    prof["gemm_oz"]["ms"] = 500.0
    r = bench.roofline_entry(prof, "bf16x3", pk, "nowhere")
    assert r["kernel"] == "gemm_oz" and r["dtype"] == "bf16"
    assert abs(r["frac"] - (1e11 / 0.5 / 1e12) / 1700.0) < 1e-12
    assert abs(r["issue_efficiency"] - 36 * r["frac"]) < 1e-12


def test_uneven_buckets_and_fill_fraction():
    b = bench.uneven_buckets()
    assert sum(b.values()) == 64 and len(b) == 10
    assert b[(12, 4.0)] == 7 and b[(32, 8.0)] == 6
    assert bench.fill_fraction(10.0, 2.0, 20.0, 2.0) == 0.5


def test_closed_forms_and_extrapolation():
    import numpy as np
    # G of the uniform field is the Fermi function in momentum space: its trace is the filling
    L, beta, mu = 6, 3.0, -0.7
    g = bench.closed_form_green_row(L, beta, 1.0, mu)
    k = 2 * np.pi * np.arange(L) / L
    eps = -2 * (np.cos(k)[None, :] + np.cos(k)[:, None]) - mu
    assert abs(g[0, 0] * L * L - np.sum(1.0 / (1.0 + np.exp(-beta * eps)))) < 1e-12
    ld = bench.closed_form_logdet(L, beta, 1.0, mu)
    assert abs(ld - np.sum(np.log1p(np.exp(-beta * eps)))) < 1e-12
    r = bench.extrapolate_oracle(1.0, dict(L=32, beta=20.0, dtau=0.1))
    assert abs(r - (256 / 1024) ** 3 * (100 / 200)) < 1e-15


def test_roofline_reports_the_dominant_launch_site():
    """The class with the most time can be several kernels; the roofline names the single
    launch site (one kernel instantiation) with the most time and takes its class's peak."""
    pk = {"bf16_tflops": 1700.0, "tf32_tflops": 1700.0 * 1100 / 2250, "fp64_tflops": 1700.0 * 1.25 / 2250,
          "fp32_tflops": 80.0, "source": "measured (sustained)"}
    sites = {"tc_gemm": {"cls": "gemm_tc", "launches": 10, "ms": 100.0, "flops": 1e13},
             "oz_gram": {"cls": "gemm_oz", "launches": 2, "ms": 60.0, "flops": 1e12},
             "oz_update_V": {"cls": "gemm_oz", "launches": 2, "ms": 60.0, "flops": 1e12}}
    prof = {"gemm_tc": {"launches": 10, "ms": 100.0, "flops": 1e13},
            "gemm_oz": {"launches": 4, "ms": 120.0, "flops": 2e12}}
    r = bench.roofline_entry(prof, "3xtf32", pk, "nowhere", sites)
    assert r["kernel"] == "tc_gemm" and r["class"] == "gemm_tc" and r["dtype"] == "tf32"
    assert abs(r["achieved"] - 100.0) < 1e-9
    assert abs(r["share"] - 100.0 / 220.0) < 1e-12 and abs(r["class_share"] - 100.0 / 220.0) < 1e-12
    assert bench.roofline_entry(prof, "3xtf32", pk, "nowhere")["kernel"] == "gemm_oz"
