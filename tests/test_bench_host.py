"""Host logic of the benchmark that needs no GPU: the clock-sample summary
that decides whether a timed region is kept (throttle reasons, median clock)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_median_max_and_reasons():
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1965, 2070, 1391.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = bench.summarise_clocks(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_reports_thermal_and_hardware_slowdown():
    lines = ["0, 1500, 2070, 1300, 0x48, Active, Not Active, Active, Not Active"] * 4
    out = bench.summarise_clocks(lines)
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1500.0


def test_clock_summary_of_nothing():
    out = bench.summarise_clocks([])
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
