"""CPU checks of the benchmark's host logic: the algorithmic byte model of
the wa-tor phases, the choice of the roofline kernel, the reference arm's
JSON line (the oracle, run on the host), and the space-efficiency bisection
on a synthetic predicate."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_phase_bytes_follow_the_documented_model():
    # per visited object + 12 per listed block + per event
    assert bench.phase_bytes("F1", 1000, 20, 0, 0, 0) == 44 * 1000 + 12 * 20
    assert bench.phase_bytes("F2", 1000, 20, 300, 100, 0) == 16 * 1000 + 12 * 20 + 24 * 300 + 16 * 100
    assert bench.phase_bytes("S0", 50, 2, 0, 0, 7) == 8 * 50 + 12 * 2 + 12 * 7
    assert bench.phase_bytes("S2", 50, 2, 30, 5, 9) == 16 * 50 + 12 * 2 + 28 * 30 + 8 * 9 + 20 * 5


def test_roofline_takes_the_slowest_method_kernel():
    phases = {p: {"method_ms_per_step": 0.01, "gbs": 100.0, "kernel": "k" + p, "bytes_per_launch": 1.0}
              for p in bench.PHASES}
    phases["S1"].update(method_ms_per_step=0.2, gbs=500.0)
    r = bench.roofline(phases, 1000.0, "measured", 20, 5)
    assert r["phase"] == "S1" and r["achieved"] == 500.0 and r["frac"] == 0.5
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["kernel"] == "kS1"


def test_roofline_traffic_only_from_its_own_window(monkeypatch):
    # DRAM traffic measured by ncu over one (steps, warmup) window is
    # reported only for a run of that same window
    phases = {p: {"method_ms_per_step": 0.01, "gbs": 100.0, "kernel": "k" + p, "bytes_per_launch": 1.0}
              for p in bench.PHASES}
    phases["F2"].update(method_ms_per_step=0.2)
    monkeypatch.setattr(bench, "TRAFFIC", {"F2": {"bytes": 5.0e7, "steps": 20, "warmup": 5, "source": "x"}})
    assert bench.roofline(phases, 1000.0, "measured", 20, 5)["traffic"] == 5.0e7
    other = bench.roofline(phases, 1000.0, "measured", 50, 5)
    assert other["traffic"] is None and other["traffic_window"]["steps"] == 20
    monkeypatch.setattr(bench, "TRAFFIC", {})
    assert bench.roofline(phases, 1000.0, "measured", 20, 5)["traffic"] is None


def test_summary_carries_batched_and_plain_side_by_side():
    line = {"value": 2.0e10, "ms_per_step": 0.3, "e2e": {"value": 1.9e10}, "roofline": {"frac": 0.1},
            "batched": {"object_updates_per_s": 3.0e10, "speedup_vs_one_by_one": 10.0},
            "alloc_free_microbench": {"rows": [{"types": 2, "objects": 1 << 24, "allocs_per_s": 5e9,
                                                "frees_per_s": 6e10}]},
            "streaming_doall": {"K4": {"100%": {"frac": 0.99}}}, "nbody_65536": {"ms_per_step": 3.0},
            "served": {"jobs_done": 5, "step_ms_p50": 1.0, "step_ms_p99": 2.0, "job_s_p50": 3.0, "job_s_p99": 4.0,
                       "admit_ms_per_job_p50": 0.5, "admit_ms_per_job_p99": 0.9, "step_ms_per_mcell_p50": 0.1,
                       "step_ms_per_mcell_p99": 0.2}}
    s = bench.summary(line)
    assert s["batched_vs_plain"] == 1.5 and s["plain_object_updates_per_s"] == 2.0e10
    assert s["allocs_per_s"] == 5e9 and s["streaming_frac_of_hbm_100pct_fill"] == {"K4": 0.99}
    assert s["served"]["admit_ms_per_job_p99"] == 0.9 and s["served"]["step_ms_per_mcell_p99"] == 0.2
    assert len(json.dumps(s)) < 1200  # fits the tail a log keeps


def test_batched_hbm_estimate_uses_the_plain_bytes_per_update():
    # plain: 2e10 updates/s at 0.5 ms a step = 1e7 updates a step; 4e8 bytes
    # a step over the phases = 40 bytes an update; batched 3e10 updates/s
    phases = {p: {"bytes_per_launch": 8.0e7} for p in bench.PHASES}
    line = {"value": 2.0e10, "ms_per_step": 0.5, "phases": phases, "batched": {"object_updates_per_s": 3.0e10}}
    h = bench.batched_hbm_estimate(line, 6000.0)
    assert h["bytes_per_object_update"] == pytest.approx(40.0)
    assert h["algorithmic_gbs"] == pytest.approx(1200.0) and h["frac"] == pytest.approx(0.2)
    assert h["frac_of_nominal"] == pytest.approx(1200.0 / bench.NOMINAL_HBM_GBS)


def test_clock_reasons_decode_the_nvml_bits():
    # sw_power_cap 0x4, hw_slowdown 0x8, sw_thermal 0x20, hw_thermal 0x40;
    # idle (0x1) and the other reasons are not reported
    assert bench.nvml_reason_names(0) == []
    assert bench.nvml_reason_names(0x1 | 0x4) == ["sw_power_cap"]
    assert bench.nvml_reason_names(0x8 | 0x20 | 0x40) == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]


def test_reference_arm_prints_the_oracle_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == bench.UNIT and line["metric"] == bench.METRIC
    assert line["value"] > 0 and line["steps"] == 2 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


@pytest.mark.parametrize("limit", [17, 40, 100, 333])
def test_space_bisection_finds_the_largest_fitting_side(limit):
    pytest.importorskip("torch")
    from paper_1809_07444_gb300 import space

    calls = []

    def fits(side):
        calls.append(side)
        return side <= limit, side * 10

    side, peak = space._bisect(fits)
    assert side == limit and peak == limit * 10
    assert len(calls) < 40
