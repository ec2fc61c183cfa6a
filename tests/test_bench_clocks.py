"""CPU checks of the benchmark's clock record: the median SM clock under load
and every throttle reason seen during the timed region."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_median_clock_and_no_reasons():
    text = "\n".join(["0, 2070, 2070, 812.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                      "0, 2055, 2070, 900.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
                      "0, 2070, 2070, 950.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"])
    r = bench.parse_clock_samples(text)
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}


def test_throttle_reasons_are_reported():
    text = "\n".join(["0, 1800, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
                      "0, 1650, 2070, 1400.0, 0x0000000000000048, Not Active, Active, Not Active, Not Active",
                      "garbage line",
                      "0, [N/A], 2070, 1400.0, 0x0, Not Active, Not Active, Not Active, Not Active"])
    r = bench.parse_clock_samples(text)
    assert r["samples"] == 2 and r["sm_mhz"] == 1725.0
    assert r["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_no_samples():
    assert bench.parse_clock_samples("")["reasons"] == ["no samples"]
