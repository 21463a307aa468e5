"""Multi-rank path of the batched sweep (bench.py --sweep under torchrun),
on CPU with two gloo ranks: the instance shards are disjoint and cover the
sweep, every rank draws the same sweep, and the timed value uses the
slowest rank."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
from paper_2501_11767_gb300 import inputs  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    sweep = inputs.sweep_instances(64)
    mine = bench.shard(list(range(len(sweep))), rank, world)
    draws = [(i["n"], round(i["params"]["evap_rate"], 12), i["seed"]) for i in sweep]
    gathered = [None] * world
    dist.all_gather_object(gathered, (mine, draws))
    t = torch.tensor([1.0 + rank])            # this rank's timed seconds
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        q.put((gathered, float(t.item())))
    dist.destroy_process_group()


def test_two_rank_sharding():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [g[0] for g in gathered]
    assert sorted(shards[0] + shards[1]) == list(range(64))
    assert not set(shards[0]) & set(shards[1])
    assert gathered[0][1] == gathered[1][1]      # same sweep on every rank
    assert tmax == 2.0


def test_shard_is_round_robin():
    assert bench.shard(list("abcdefg"), 1, 3) == ["b", "e"]
    assert bench.shard([], 0, 2) == []
