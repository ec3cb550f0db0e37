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


def test_cpu_list_is_compacted_into_ranges():
    assert bench.compact_ranges([]) == ""
    assert bench.compact_ranges([0, 1, 2, 3, 7, 9, 10]) == "0-3,7,9-10"
    assert bench.compact_ranges([5]) == "5"


def test_numa_nodes_of_cpus_never_raises():
    nodes = bench.numa_nodes_of_cpus(sorted(os.sched_getaffinity(0)))
    assert isinstance(nodes, list) and all(isinstance(n, int) and n >= 0 for n in nodes)


def test_oracle_entry_extrapolates_by_permutations():
    e = bench.oracle_entry(k=100, n=1000, sample_perms=500, total_perms=10_000, dt=2.0, cores=8, what="messages")
    assert e["full_ms_extrapolated"] == 2.0 * 10_000 / 500 * 1e3
    assert e["mperm_s"] == 500 / 2.0 / 1e6 and e["cores"] == 8 and e["kind"] == "oracle"
    assert "100 of 1000 messages" in e["sample"]


def test_alu_fraction_of_a_batch_at_the_roofline():
    # perms x ops at exactly the peak rate is a fraction of 1.
    peak = bench.SM_COUNT_GB300 * bench.INT_LANES_PER_SM_CLK * bench.SM_MAX_MHZ * 1e6
    perms = 1_000_000
    ms = perms * bench.ops_per_permutation() / peak * 1e3
    assert abs(bench.alu_frac(perms, ms) - 1.0) < 1e-12


def test_link_bound_overlaps_the_two_directions():
    link = {"copy_engine_both_ways_gb_s": 340.0, "copy_engine_h2d_gb_s": 210.0, "copy_engine_d2h_gb_s": 130.0}
    n, in_b, out_b = 1 << 24, 1 << 30, 1 << 29
    # out_b moves while both directions share the link (170 GB/s each), the
    # rest of the input alone at 210 GB/s.
    want = n / (out_b / 170e9 + (in_b - out_b) / 210e9) / 1e6
    assert abs(bench.link_bound_mhash_s(link, in_b, out_b, n) - want) < 1e-6
    assert bench.link_bound_mhash_s({"copy_engine_h2d_gb_s": "probe failed"}, in_b, out_b, n) is None
