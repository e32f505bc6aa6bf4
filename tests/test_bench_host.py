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


def _bench_rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    b.barrier(world)
    t = b.max_over_ranks(1.5 + rank, world, "cpu")   # rank 1 is the slower one
    b.barrier(world)
    out.put((rank, t))
    dist.destroy_process_group()


def test_timing_is_the_max_over_two_gloo_ranks():
    # the N > 1 bench reports the slowest rank's time on every rank
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 30500 + os.getpid() % 1000
    procs = [ctx.Process(target=_bench_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}
