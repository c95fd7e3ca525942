"""Host-side logic of the benchmark that needs no GPU: the clock record
taken during the timed region and the weak-scaling seed split."""

import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def _line(sm, mx, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    # index, clocks.sm, clocks.max.sm, power.draw, reasons.active, hw_slowdown,
    # hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    return f"0, {sm}, {mx}, 900.5, 0x0000000000000000, {hw}, {hwt}, {swt}, {cap}"


def test_clock_summary_median_max_and_reasons():
    c = bench.Clocks(0)
    c.lines = [_line(2070, 2070), _line(1980, 2070, cap="Active"), _line(2070, 2070),
               _line(1500, 2070, hwt="Active"), "garbage", ""]
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2025.0  # median of 1500, 1980, 2070, 2070
    assert s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    c = bench.Clocks(0)
    c.lines = []
    assert c.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}


def test_rank_seeds_are_disjoint_and_cover():
    seen = []
    for r in range(4):
        seen += list(bench.rank_seeds(r, 4096))
    assert seen == list(range(4 * 4096))


def test_workloads_have_the_stated_shapes():
    ds, cfg = bench.workload("c1")
    assert len(ds) == 1 and ds[0].shape == (2, 40) and cfg["instances"] == 1
    ds, cfg = bench.workload("hard300")
    assert len(ds) == 1 and ds[0].shape == (2, 300)
    ds, cfg = bench.workload("cerny")
    assert [d.shape[1] for d in ds] == list(range(16, 29))
