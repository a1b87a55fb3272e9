"""Host side of running on several GPUs of one node: one process per GPU.

A single system does not shard in this build (each rank integrates its own replica of the
workload); batches of independent systems shard by system, with no data-path collective.
Only scalars cross ranks: the barrier before and after a timed region, and the max / sum
of per-rank results.
"""
from __future__ import annotations

import os


def env_ranks():
    """(world, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _all_reduce(x, world, dev, op_name):
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op_name))
    return float(t.item())


def reduce_max(x, world, dev):
    return _all_reduce(x, world, dev, "MAX")


def reduce_sum(x, world, dev):
    return _all_reduce(x, world, dev, "SUM")


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def shard_greedy(costs, world):
    """Split units of the given costs over `world` ranks: largest cost first, each to the
    rank with the least load so far (lowest rank on ties) -- the division scheduler of
    Sec. 4.2 applied to ranks. Returns one ascending index list per rank."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += costs[i]
        parts[r].append(i)
    return [sorted(p) for p in parts]
