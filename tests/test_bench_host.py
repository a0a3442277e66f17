"""CPU tests of bench.py's host logic: the clock-sample summary that decides whether a timing run
is valid (throttle reasons, SM clock), the measured-peak lookup, and the workload recipes."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _sampler(lines):
    c = bench.ClockSampler(0)
    c.lines = list(lines)
    return c


def test_clock_summary_median_and_reasons():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1900, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1200.0, 0x20, Not Active, Not Active, Active, Not Active"
    s = _sampler([ok, ok, cap]).summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    s = _sampler([ok, hot, "garbage line"]).summary()
    assert s["reasons"] == ["sw_thermal_slowdown"] and s["samples"] == 2
    s = _sampler([]).summary()
    assert s["sm_mhz"] is None and s["reasons"] == ["unavailable"]


def test_peak_lookup_prefers_the_measured_file():
    peak, kind = bench.peaks()
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        assert kind == "measured" and peak > 1000
    else:
        assert (peak, kind) == (6800.0, "fallback")


def test_workload_recipes_are_seeded_and_in_range():
    W = bench.workload()
    assert (W["n"], W["k"], W["rhs"], W["steps"]) == (32, 2, 1, 2000)
    assert W["eps"].shape == (6 * 32 ** 3,) and 1.0 <= W["eps"].min() and W["eps"].max() < 4.0
    assert np.all((W["x0"] >= 0.2) & (W["x0"] < 0.8)) and np.allclose(W["d"], [0, 0, 1])
    B = bench.workload(rhs=64, leapfrog_steps=1000)
    assert B["xs"].shape == (64, 3) and np.allclose(np.linalg.norm(B["ds"], axis=1), 1.0)
    assert np.array_equal(bench.workload()["eps"], W["eps"])            # deterministic
    src = bench.source_for(B, 0.01)
    assert len(src) == 64 and [s["rhs"] for s in src] == list(range(64))
    assert all(abs(s["sigma"] - 0.2) < 1e-15 and abs(s["t0"] - 0.8) < 1e-15 for s in src)


def test_cpu_baseline_line_reports_single_and_all_core_rates():
    """The timed oracle leg on a tiny sample: one process and one spawned replica per host core."""
    import types
    line = bench.cpu_baseline_line(types.SimpleNamespace(cpu_n=2, cpu_steps=20))
    assert line["kind"] == "oracle" and line["cores"] == (os.cpu_count() or 1)
    assert line["value"] > 0 and line["single_thread"]["value"] > 0 and line["single_thread"]["cores"] == 1
    assert line["first_workload_in_full"]["value"] > 0
    assert "2^3 cube" in line["sample"]
