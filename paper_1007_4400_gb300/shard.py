"""Assignment of independent k-point sequences to ranks (one process per GPU).

The k-points of the batched form are independent problems (the paper solves Eq. 3 for
each k-point separately), so N GPUs split them with no exchange on the data path: each
rank solves its own subset with one gevp_solve_batched call and only the timings are
reduced. Subsets are balanced by the dominant cost of a problem of order n (the n^3
reduction and the n^2 m filter/Rayleigh-Ritz work, m ~ 0.084 n here), greedily largest
first onto the least loaded rank (LPT scheduling, within 4/3 of the optimal makespan).
"""
from __future__ import annotations


def problem_cost(n: int, m: int) -> float:
    return 4.0 * n ** 3 + 60.0 * n * n * m


def shard_kpoints(sizes, world: int):
    """sizes: list of (n, nev, nex). Returns a list of `world` sorted index lists."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda k: (-problem_cost(sizes[k][0], sizes[k][1] + sizes[k][2]), k))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        out[r].append(k)
        load[r] += problem_cost(sizes[k][0], sizes[k][1] + sizes[k][2])
    return [sorted(x) for x in out]


def shard_loads(sizes, shards):
    return [sum(problem_cost(sizes[k][0], sizes[k][1] + sizes[k][2]) for k in s) for s in shards]
