"""Env sharding over ranks and the max-over-ranks timing reduction, run as
two gloo ranks on the CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2311_05945_b300.sharding import max_over_ranks, shard_envs


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shards_cover_every_env_once_and_balance(world):
    w = [2000, 19000, 3000, 3000, 7000, 12000, 2500, 8000, 4000, 16000, 2200, 6000]
    parts = shard_envs(w, world)
    assert len(parts) == world
    assert parts[0][0] == 0 and parts[-1][1] == len(w)
    for (a, b), (c, d) in zip(parts, parts[1:]):
        assert b == c and a <= b
    assert all(b > a for a, b in parts)  # no empty rank when envs >= ranks
    loads = [sum(w[a:b]) for a, b in parts]
    assert max(loads) <= sum(w) / world + max(w)


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = list(range(1, 17))
    a, b = shard_envs(w, world)[rank]
    # each rank "steps" its own envs; the job's work is the sum over ranks
    mine = torch.tensor([float(sum(w[a:b]))])
    dist.all_reduce(mine)
    t = max_over_ranks(1.0 + rank, dist)
    out[rank] = (float(mine.item()), t)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    mgr = mp.get_context("spawn").Manager()  # no fork of this (threaded) process
    out = mgr.dict()
    port = 29500 + (os.getpid() % 1000)
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (float(sum(range(1, 17))), 2.0)
