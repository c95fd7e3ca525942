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


def test_workloads_hard400_shape():
    ds, cfg = bench.workload("hard400")
    assert len(ds) == 1 and ds[0].shape == (2, 400) and "7x64-bit" in cfg["workload"]


def test_stratified_seeds_spread_evenly():
    assert bench.stratified_seeds(4096, 16) == list(range(0, 4096, 256))
    assert bench.stratified_seeds(10, 3) == [0, 3, 6]


def _run_bench(*argv):
    import json
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), *argv], capture_output=True, text=True,
                         timeout=600, check=True).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out
    return json.loads(lines[0])


def test_reference_arm_runs_every_sampled_instance_to_completion():
    # the reference arm on the CPU: W warm-up and K timed steps of the
    # oracle over the declared stratum; no GPU is touched
    line = _run_bench("--impl", "reference", "--workload", "c1", "--steps", "2", "--warmup", "1")
    cores = os.cpu_count() or 1
    assert line["impl"] == "reference" and line["steps"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == cores
    assert f"{2 * cores} instances timed" in line["cpu_baseline"]["sample"]
    assert line["cpu_baseline"]["single_thread"] > 0
    assert line["e2e"]["value"] == line["value"]


def test_reference_arm_hard_instance_is_unavailable():
    line = _run_bench("--impl", "reference", "--workload", "hard300")
    assert line["impl"] == "reference" and "unavailable" in line


def test_cpu_baseline_line_counts_every_instance():
    from paper_2207_05495_gb300 import gen
    ds = [gen.random_automaton(12 + i, 2, i) for i in range(8)]
    cpu = bench.cpu_baseline_line(ds, 4, 2)
    assert cpu["cores"] == 2 and cpu["kind"] == "oracle"
    assert cpu["value"] > 0 and cpu["single_thread"] > 0
    assert "indices 0, 2, ... 6" in cpu["sample"] and "whole workload" in cpu["sample"]
    cpu = bench.cpu_baseline_line(ds, 4, 2, n_max=15)  # n = 12 .. 15: four instances
    assert "indices 0, 1, ... 3" in cpu["sample"] and "stratum n <= 15 (4 of 8" in cpu["sample"]


def test_reference_arm_large_beam_is_unavailable():
    line = _run_bench("--impl", "reference", "--workload", "beam5000")
    assert line["impl"] == "reference" and "unavailable" in line


def test_workloads_beam_shape():
    ds, cfg = bench.workload("beam5000")
    assert len(ds) == 1 and ds[0].shape == (2, 5000) and "beam n*ceil(log2 n) = 65000" in cfg["workload"]


def test_schedules_agree_words_only_when_unique():
    a = (5, [0, 1, 1, 0, 1], [1, 2, 3], [4, 6])
    same_sizes_other_word = (5, [1, 0, 1, 1, 0], [1, 2, 3, 5], [4])
    assert bench.schedules_agree(a, a, True)
    # another reset word of length r: a disagreement for the plain search
    # (its word is the least one), not with a reduced side or the inverse phase
    assert not bench.schedules_agree(a, same_sizes_other_word, True)
    assert bench.schedules_agree(a, same_sizes_other_word, False)
    # r or a level both computed that differ: never an agreement
    assert not bench.schedules_agree(a, (6,) + a[1:], False)
    assert not bench.schedules_agree(a, (5, a[1], [1, 2, 4], [4, 6]), False)


def test_meet_roofline_averages_the_timed_steps():
    base = dict(meet_launches=4, meet_lane_words=2)
    stats = [dict(base, meet_ms=10.0, pairs=100, and_iters=1000, rows_transposed=50),
             dict(base, meet_ms=20.0, pairs=300, and_iters=3000, rows_transposed=150)]
    assert bench.meet_roofline(stats, 152) == (15.0, 200.0, 2000.0, 100.0, 4.0, 2)
    # the direct test reports 0 lane words: counted as one
    stats[-1]["meet_lane_words"] = 0
    assert bench.meet_roofline(stats, 152)[5] == 1


def test_mark_roofline_counts_the_bitmap_work():
    stats = [dict(mark_ms=2.0, mark_steps=1e9, mark_rows=1e8, mark_pairs=5e12)]
    m = bench.mark_roofline(stats, lw=2, W=3, peak=40.0)
    ops = 1e9 * 64 * 2 + 1e8 * 2 * 3 * 25  # AND words per step, 25 ops per transposed 32-bit word
    assert abs(m["achieved"] - ops / 2e-3 / 1e12) < 1e-9
    assert abs(m["frac"] - m["achieved"] / 40.0) < 1e-12
    assert m["pairs_per_step"] == 5e12
    assert bench.mark_roofline([dict(mark_ms=0.0, mark_steps=0, mark_rows=0, mark_pairs=0)], 2, 3, 40.0) is None


def test_hbm_line_is_bytes_over_event_time():
    line = bench.hbm_line(10.0, 68e9, (6800.0, "measured"), "basis")
    assert abs(line["achieved"] - 6800.0) < 1e-9 and abs(line["frac"] - 1.0) < 1e-12
    assert line["peak_basis"] == "measured copy bandwidth" and line["traffic"] is None
    assert bench.hbm_line(0.0, 1e9, (6800.0, "fallback"), "b")["achieved"] == 0.0
