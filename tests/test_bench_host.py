"""Host logic of the benchmark that needs no GPU: the clock-sample summary
that goes into the JSON line's ``clocks`` (median SM clock under load, the
maximum, and every throttle reason seen)."""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402

IDLE = "0, 2070, 2070, 812.40, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
CAPPED = "0, 1965, 2070, 1398.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
HOT = "0, 1800, 2070, 1200.00, 0x0000000000000040, Not Active, Active, Not Active, Not Active"


def test_clock_summary_median_max_and_reasons():
    got = bench.ClockSampler.summarise([IDLE, CAPPED, IDLE, "garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d"])
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    got = bench.ClockSampler.summarise([HOT, CAPPED, CAPPED])
    assert got["sm_mhz"] == 1965.0 and got["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_samples():
    assert bench.ClockSampler.summarise([]) is None
    assert bench.ClockSampler.summarise(["not, enough, fields"]) is None


def test_kernel_hash_ignores_comments_and_layout():
    from paper_2309_14545_gb300.build import _code_only
    a = "int f(int x) {  // add one\n    return x + 1; /* the\n step */ }\n"
    b = "int f(int x) { return x + 1; }"
    assert _code_only(a) == _code_only(b)
    assert _code_only("return x + 1;") != _code_only("return x + 2;")
