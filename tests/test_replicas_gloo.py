"""Host side of the multi-GPU path with two gloo ranks on the CPU (no GPU needed).

Each rank runs what bench.py runs around a timed region: the barrier, the max of the
per-rank times, the sum of the per-rank counts, and the greedy split of a batch of
independent systems (largest N^2 first, to the least-loaded rank), which must give every
system to exactly one rank and balance the work.
"""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    from paper_2001_03180_gb300 import replicas as R
    from paper_2001_03180_gb300 import workloads as W

    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", world_size=world, rank=rank)
    w, r, loc = R.env_ranks()
    R.barrier(w)
    mx = R.reduce_max(10.0 + rank, w, "cpu")
    sm = R.reduce_sum(1.5 * (rank + 1), w, "cpu")
    systems = W.batched_systems(64, 3)
    costs = [len(s.m) ** 2 for s in systems]
    mine = R.shard_greedy(costs, w)[r]
    load = R.reduce_sum(sum(costs[i] for i in mine), w, "cpu")
    R.barrier(w)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(dict(world=w, rank=r, local=loc, max=mx, sum=sm, mine=mine, load=load,
                       myload=sum(costs[i] for i in mine), total=sum(costs)), f)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_shard(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)]
    for k, d in enumerate(res):
        assert d["world"] == 2 and d["rank"] == k and d["local"] == k
        assert d["max"] == 11.0 and d["sum"] == 1.5 + 3.0
        assert d["load"] == d["total"]
    a, b = set(res[0]["mine"]), set(res[1]["mine"])
    assert not (a & b) and len(a | b) == 64
    # the greedy split leaves the ranks within one largest system (N <= 200) of each other
    assert abs(res[0]["myload"] - res[1]["myload"]) <= 200 ** 2


def test_shard_greedy_single_rank_and_ties():
    sys.path.insert(0, ROOT)
    from paper_2001_03180_gb300 import replicas as R

    assert R.shard_greedy([3, 1, 2], 1) == [[0, 1, 2]]
    assert R.shard_greedy([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]
    assert R.shard_greedy([], 3) == [[], [], []]
