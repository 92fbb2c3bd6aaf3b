"""Sharding of independent problems across ranks (one process per GPU).

A single instance runs as replicas only (splitting its rows would need an
all-reduce per block step).  The batched form shards by instance: each rank
solves its share with rac_admm_batch and the results are gathered on the
host; there is no collective on the data path.
"""
from __future__ import annotations

from typing import Callable, List, Sequence


def lpt_shards(work: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment: instances sorted by decreasing work,
    each given to the currently least-loaded rank.  Returns per-rank index
    lists (each sorted ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += float(work[i])
    return [sorted(s) for s in out]


def run_sharded(problems: Sequence[dict], work: Sequence[float], solve_batch: Callable,
                rank: int, world: int, group=None):
    """Solve this rank's shard with `solve_batch(list_of_problems) -> (xs, infos)`
    and gather every rank's results (torch.distributed object gather over the
    host process group).  Returns (xs, infos) in the original order on every
    rank."""
    import torch.distributed as dist

    shards = lpt_shards(work, world)
    mine = shards[rank]
    xs, infos = solve_batch([problems[i] for i in mine]) if mine else ([], [])
    local = list(zip(mine, xs, infos))
    if world == 1:
        gathered = [local]
    else:
        gathered = [None] * world
        dist.all_gather_object(gathered, local, group=group)
    out_x = [None] * len(problems)
    out_i = [None] * len(problems)
    for part in gathered:
        for i, x, inf in part:
            out_x[i] = x
            out_i[i] = inf
    return out_x, out_i
