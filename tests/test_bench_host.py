"""Host logic of bench.py that needs no GPU: the summary of the sampled clocks and throttle
reasons that accompanies every measured number, and the choice of the HBM peak used as the
roofline denominator (the measured figure when present, else the stated fallback)."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _row(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(mx), "900.0", "0x0", hw, hwt, swt, cap]


def test_clock_summary_median_max_and_reasons():
    c = bench.ClockSampler(0)
    c.rows = [_row(1965, 2070), _row(1980, 2070, cap="Active"), _row(2010, 2070), _row("[N/A]", 2070)]
    s = c.summary()
    assert s["sm_mhz"] == 1980.0            # median of the readable samples
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 4


def test_clock_summary_reports_every_slowdown_once():
    c = bench.ClockSampler(0)
    c.rows = [_row(1200, 2070, hw="Active"), _row(1100, 2070, hwt="Active", swt="Active"),
              _row(1150, 2070, hw="Active")]
    assert c.summary()["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_samples():
    s = bench.ClockSampler(0).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["unavailable"]


def test_peak_measured_else_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._peaks() == (6800.0, "fallback")
    with open(tmp_path / "MEASURED_PEAKS.json", "w") as f:
        json.dump({"hbm_gbs": 6761.5, "bf16_tflops": 2000.0}, f)
    assert bench._peaks() == (6761.5, "measured")
