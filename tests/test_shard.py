"""Host logic of the multi-GPU batched form: the k-point partition across ranks, checked
alone and with two gloo ranks that agree on it and reduce their timings (max over ranks),
as bench.py does over NCCL."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def test_partition_is_balanced_and_complete():
    from paper_1007_4400_gb300 import shard, synth
    sizes = synth.batched_sizes(64)
    for world in (1, 2, 3, 4, 8):
        sh = shard.shard_kpoints(sizes, world)
        flat = sorted(k for s in sh for k in s)
        assert flat == list(range(64))
        loads = shard.shard_loads(sizes, sh)
        biggest = max(shard.problem_cost(n, nev + nex) for n, nev, nex in sizes)
        assert max(loads) - min(loads) <= biggest


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1007_4400_gb300 import shard, synth
    sizes = synth.batched_sizes(64)
    mine = shard.shard_kpoints(sizes, world)[rank]
    # every rank derives the same partition: gather and compare
    got = [None] * world
    dist.all_gather_object(got, mine)
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((got, float(t)))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    from paper_1007_4400_gb300 import shard, synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == shard.shard_kpoints(synth.batched_sizes(64), 2)
    assert sorted(got[0] + got[1]) == list(range(64))
    assert tmax == 2.0
