"""Host-side arithmetic of the benchmark line, on the CPU: the roofline of a
decode (algorithmic bytes over its time against the measured peak), the DRAM
traffic record (accepted only for the kernel sources it was captured on, and
scaled by the code count) and the peak taken from the measured file."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_roofline_of_is_bytes_over_time_against_the_peak():
    r = bench.roofline_of(431_671_949, 0.33, 6763.3, "measured")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak_kind"] == "measured"
    assert r["achieved"] == pytest.approx(431_671_949 / 0.33e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6763.3)
    assert r["algorithmic_bytes"] == 431_671_949 and r["kernel_ms"] == 0.33


def test_traffic_record_matches_the_current_sources_and_scales_by_codes():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for kernel, e in rec.items():
        assert kernel in bench.KERNEL_SOURCES
        if e["source_hash"] != bench.kernel_source_hash(kernel):
            # the benchmark reports no traffic until the kernel is profiled again
            assert bench.recorded_traffic(kernel, e["n_codes"], {}) is None
            pytest.skip(f"{kernel}: traffic record predates the kernel sources")
        full = bench.recorded_traffic(kernel, e["n_codes"], {})
        assert full == pytest.approx(e["dram_bytes_per_launch"])
        half = bench.recorded_traffic(kernel, e["n_codes"] // 2, {})
        assert half == pytest.approx(e["dram_bytes_per_launch"] / 2)


def test_traffic_record_is_refused_once_a_source_changes(monkeypatch):
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kernel="decode_gap": "0" * 16)
    assert bench.recorded_traffic("decode_gap_one_pass", 134217728, {}) is None
    assert bench.recorded_traffic("no_such_kernel", 134217728, {}) is None


def test_peak_is_the_measured_copy_bandwidth():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if not os.path.exists(p):
        assert bench.measured_peak() == (bench.FALLBACK_HBM_GBS, "fallback")
        return
    with open(p) as f:
        d = json.load(f)
    assert bench.measured_peak() == (float(d["hbm_gbs"]), "measured")
