"""Host logic of bench.py (no GPU): the roofline arithmetic, the algorithmic
bytes of a scored slice, the parsing of the clock samples the timing rules
depend on (throttle reasons, median SM clock), and the reference arm's JSON
line (the FP64 oracle timed on the host)."""

import math
import os

import pytest

import bench


def test_slice_bytes_per_pose_point():
    # (2 + 2) rows x (c + 2) pixels x 8 bytes for 2 x c poses
    assert math.isclose(bench.slice_bytes_per_pp(10, "fp32"), 4 * 12 * 8 / 20)
    assert math.isclose(bench.slice_bytes_per_pp(6, "fp32"), 4 * 8 * 8 / 12)
    assert math.isclose(bench.slice_bytes_per_pp(6, "bf16"), bench.slice_bytes_per_pp(6, "fp32") / 2)


def test_roofline_arithmetic():
    r = bench.dense_roofline(pp_per_launch=3e9, ms_per_launch=2.0, sm_count=152, sm_mhz_peak=2070.0, traffic=123)
    peak = 128 * 152 * 2070e6 / 1e12
    achieved = 3e9 * (640.0 / 48.0) / 2e-3 / 1e12
    assert math.isclose(r["peak"], round(peak, 3))
    assert math.isclose(r["achieved"], round(achieved, 3))
    assert math.isclose(r["frac"], round(achieved / peak, 4))
    assert r["bound"] == "smem" and r["traffic"] == 123


def _sampler(tmp_path, lines):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clk.csv")
    with open(s.path, "w") as f:
        f.write("\n".join(lines) + "\n")
    s.proc = object()   # summary() only checks that sampling ran
    return s


def test_clock_summary_median_and_reasons(tmp_path):
    ok = "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1900, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1000.0, 0x0000000000000040, Not Active, Active, Not Active, Not Active"
    s = _sampler(tmp_path, [ok, ok, cap])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0 and out["samples"] == 3
    assert out["reasons"] == ["sw_power_cap"]
    out = _sampler(tmp_path, [ok, hot, hot]).summary()
    assert out["sm_mhz"] == 1500.0 and "hw_thermal_slowdown" in out["reasons"]


def test_clock_summary_without_samples(tmp_path):
    s = _sampler(tmp_path, ["garbage"])
    assert s.summary()["reasons"] == ["unsampled"]
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["unsampled"]


def test_reference_arm_line():
    """`bench.py --impl reference` times the FP64 oracle on the host and
    prints one JSON line in the benchmark's format, with the oracle's own
    host-only e2e figure (no copies)."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=root, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
