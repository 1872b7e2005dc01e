"""bench.py's host-side arithmetic, without a GPU: the roofline object of the
dominant kernel group and the clock record that rejects throttled runs."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def _stats(chase_ms, apply_ms, updates, apply_launches):
    return {"ms_chase": chase_ms, "ms_apply_q": apply_ms / 2, "ms_apply_p": apply_ms / 2, "ms_project": 1.0,
            "timed_updates": updates, "apply_launches": apply_launches}


@pytest.fixture
def size(monkeypatch):
    def set_size(k):
        monkeypatch.setattr(bench, "M", k)
        monkeypatch.setattr(bench, "N", k)
    return set_size


def test_chase_roofline_is_flops_over_time_against_the_fp64_peak(size):
    size(4096)
    st = _stats(chase_ms=1750.0, apply_ms=1110.0, updates=10, apply_launches=20)
    rot = 25_156_950
    r = bench.roofline(st, 1, rot, 10, steps_per_update=45_027)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    want = bench.CHASE_FLOPS_PER_ROTATION * rot / 0.175 / 1e12
    assert r["achieved"] == pytest.approx(want)
    assert r["peak"] == pytest.approx(152 * 2 * 2 * 2.070e9 / 1e12)
    assert r["frac"] == pytest.approx(want / r["peak"])
    assert r["traffic"] == bench.CHASE_TRAFFIC_4096
    assert r["critical_path"]["us_per_step"] == pytest.approx(175e3 / 45_027)
    assert r["share"] == pytest.approx(1750.0 / (1750.0 + 1110.0 + 1.0))


def test_traffic_is_only_reported_for_the_captured_workload(size):
    size(1024)
    r = bench.roofline(_stats(500.0, 100.0, 10, 20), 1, 1_500_000, 10)
    assert r["traffic"] is None


def test_apply_dominated_roofline_uses_the_apply_launches(size):
    size(4096)
    st = _stats(chase_ms=100.0, apply_ms=8000.0, updates=10, apply_launches=20)
    rot = 25_000_000
    r = bench.roofline(st, 0, rot, 10)
    per_launch = 8000.0 / 20
    want = 6 * rot / 2 * 4096 / (per_launch * 1e-3) / 1e12
    assert r["achieved"] == pytest.approx(want) and r["peak"] == pytest.approx(bench.ALU_FP64_TFLOPS)


def test_clock_samples_flag_throttling_and_take_the_median():
    ok = "0, 2070, 2070, 900.5, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x20, Not Active, Not Active, Active, Not Active"
    c = bench.parse_clock_samples([ok, ok, cap])
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0 and c["reasons"] == ["sw_power_cap"]
    c = bench.parse_clock_samples([ok, hot, hot, "garbage", ""])
    assert c["samples"] == 3 and c["sm_mhz"] == 1500.0 and c["reasons"] == ["sw_thermal_slowdown"]
    c = bench.parse_clock_samples([])
    assert c["sm_mhz"] is None and c["samples"] == 0


def test_latency_summary_names_p99_only_with_enough_samples():
    few = bench.latency_summary([5.0, 1.0, 3.0], "x")
    assert few["p50"] == 3.0 and few["max"] == 5.0 and "p99" not in few and few["samples"] == 3
    many = bench.latency_summary([float(i) for i in range(1, 201)], "x")
    assert many["p99"] == 198.0 and many["max"] == 200.0 and many["p50"] == 100.5


def test_apply_roofline_counts_factor_and_records_once(size, monkeypatch):
    size(4096)
    monkeypatch.setattr(bench, "peaks", lambda: {"hbm_gbs": 6800.0})
    st = _stats(chase_ms=0.0, apply_ms=100.0, updates=2, apply_launches=4)
    rot = 25_000_000
    r = bench.apply_roofline(st, rot)
    alg = 2 * 4096 * 4096 * 4 + 8 * rot / 2
    assert r["algorithmic_bytes"] == alg and r["ms_per_launch"] == pytest.approx(25.0)
    assert r["achieved"] == pytest.approx(alg / 25e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6800.0)
