"""Host-side logic of bench.py that decides whether a run counts: the clock summary taken
from nvidia-smi samples (throttle reasons reject a measurement) and the fixed work count
behind the nominal rate."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_summary_reads_median_and_reasons():
    b = _bench()
    lines = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2070, 2070, 950.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
        "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    out = b.summarize_clock_lines(lines)
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_thermal_and_empty_input():
    b = _bench()
    out = b.summarize_clock_lines(["0, 1500, 2070, 1400, 0x40, Not Active, Active, Not Active, Not Active"])
    assert out["reasons"] == ["hw_thermal_slowdown"] and out["sm_mhz"] == 1500.0
    empty = b.summarize_clock_lines([])
    assert empty["sm_mhz"] is None and empty["samples"] == 0 and empty["reasons"] == []


def test_nominal_work_grows_with_size():
    b = _bench()
    w1 = b.nominal_flops_per_problem(2048, 140, 100, 20)
    w2 = b.nominal_flops_per_problem(4096, 140, 100, 20)
    assert w1 > 0 and w2 > 4 * w1   # the n^3 reduction dominates
