"""Host logic of bench.py that needs no GPU: the clock record taken during the
timed region (nvidia-smi samples filtered to the region, throttle reasons,
median clock) and the whole-job rate of the replica runs."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _line(sm, smax, hw="Not Active", hw_thermal="Not Active", sw_thermal="Not Active", power="Not Active"):
    return f"0, {sm}, {smax}, 900.00, 0x0000000000000000, {hw}, {hw_thermal}, {sw_thermal}, {power}"


def test_clock_summary_keeps_the_timed_region_only():
    s = bench.ClockSampler(0)
    s.marks = [10.0, 11.0]
    s.samples = [(9.0, _line(1000, 2070, hw="Active")),   # before the region: ignored
                 (10.2, _line(2070, 2070)), (10.5, _line(2060, 2070, power="Active")),
                 (10.8, _line(2070, 2070)),
                 (12.0, _line(500, 2070, hw_thermal="Active"))]  # after: ignored
    out = s.summary()
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 3


def test_clock_summary_reports_slowdowns_and_skips_bad_lines():
    s = bench.ClockSampler(0)
    s.marks = [0.0, 5.0]
    s.samples = [(1.0, _line(1500, 2070, hw="Active", sw_thermal="Active")), (2.0, "garbage"),
                 (3.0, _line("[N/A]", 2070)), (4.0, _line(1600, 2070))]
    out = s.summary()
    assert out["sm_mhz"] == 1550.0
    assert out["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]


def test_clock_summary_without_nvidia_smi():
    out = bench.ClockSampler(0).summary()
    assert out["sm_mhz"] is None and out["samples"] == 0 and out["reasons"]


def test_whole_job_rate_counts_every_rank():
    assert bench.whole_job_mhash_s(1 << 24, 1, 4.0) == (1 << 24) / 4e-3 / 1e6
    assert bench.whole_job_mhash_s(1 << 24, 4, 4.0) == 4 * bench.whole_job_mhash_s(1 << 24, 1, 4.0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert [bench.rank_seed(1, r) for r in range(3)] == [1, 2, 3]
