"""Multi-rank host logic on CPU process groups (gloo, world size 2)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2209_10643_b300.sharding import aggregate_throughput, shard_lpt


def test_shard_lpt_partitions_every_item_once():
    costs = [5, 1, 9, 3, 3, 7, 2, 8, 1, 4]
    for world in (1, 2, 3, 4, 16):
        parts = shard_lpt(costs, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(costs)))
        loads = [sum(costs[i] for i in p) for p in parts]
        if world <= len(costs):
            assert max(loads) - min(loads) <= max(costs)
    assert shard_lpt([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        shard_lpt([1.0], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, secs = aggregate_throughput(100.0 * (rank + 1), 0.5 + rank)
        out[rank] = (units, secs)
    finally:
        dist.destroy_process_group()


def test_aggregate_throughput_gloo_world2():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    assert out[0] == out[1] == (300.0, 1.5)


def test_aggregate_without_group_is_identity():
    assert aggregate_throughput(7.0, 2.0) == (7.0, 2.0)
