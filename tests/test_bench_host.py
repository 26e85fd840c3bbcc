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


def _fake_line():
    form = {"glups": 27.0, "roofline_frac": 0.9, "rel_linf_vs_f64": {"rho": 1e-3, "E": 2e-3}}
    case = lambda grid, tau, bad: {  # noqa: E731
        "grid": grid, "mach": 2.0, "beta": 1.0, "tau": tau,
        "nonphysical_at": {"f64": bad, "f32": bad, "f16dev": bad, "bf16dev": bad},
        "linf_worst": {f: ({"10": 1e-3, "100": 2e-3} if bad != 10 else {}) for f in ("f32", "f16dev", "bf16dev")},
        "l2_worst": {}}
    return {
        "value": 15.2, "roofline": {"frac": 1.01},
        "forms": {"f64": {"glups": 1.86, "roofline": {"frac": 0.79}}, "f16dev": form},
        "error_growth": {"steps": 1000, "cases": [case("256^3", 0.51, 1000), case("256^3", 0.6, None),
                                                  case("128^3", 0.51, 10), case("128^3", 0.6, None)]},
        "other_paths": {"resistive_channel": {"glups": 20.5, "roofline_frac": 0.98},
                        "batched_2d": {"glups_batched": 20.4, "roofline_frac_batched": 0.97, "speedup": 1.27},
                        "ideal_2d_128sq_f64": {"glups": 1.5},
                        "learned_closure": {"tests": [
                            {"fine_ms": 8800.0, "coarse_closure": [160.0, 0.02, 0.01, 0], "coarse_plain": [45.0, 0.03,
                                                                                                0.02, 0],
                             "plain": {"64": [10.0, 0.06, 0], "128": [45.0, 0.03, 0],
                                       "256": [550.0, 0.015, 0]},
                             "closure_over_curve": 1.01}] * 4,
                            "tensor_frac": 0.26}},
        "fp64_tflops": 1.057,
    }


def test_compact_summary_keeps_every_path_in_a_short_tail():
    import json
    out = bench.compact_summary(_fake_line())
    text = json.dumps(out)
    assert len(text) < 1400, len(text)
    assert out["headline"] == [15.2, 1.01]
    assert out["form_f64"] == [1.86, 0.79, None] and out["form_f16dev"] == [27.0, 0.9, 0.002]
    rows = out["growth_[f64bad,f32,f16,bf16:[step,linf]]"]
    assert rows["256^3 M2 b1 t0.51"] == [1000, [100, 0.002], [100, 0.002], [100, 0.002]]
    sweep = out["growth_sweep_M2,3xb.1,1,10"]
    assert sweep["128^3 t0.51"] == {"f64bad": [10], "bf16_linf_last": 0.0}
    assert out["batched"] == [20.4, 0.97, 1.27] and out["cfg1_f64[glups,flop_frac,pipe_frac]"] == [1.5, None, None]
    assert out["closure_[fine_ms,cl_ms,cl_err,plain_err,cl/curve]"][0] == [8800.0, 160.0, 0.02, 0.03, 1.01]
    assert out["closure_curve_ms_err_64,128,256"] == [[[10.0, 0.06], [45.0, 0.03], [550.0, 0.015]]]
