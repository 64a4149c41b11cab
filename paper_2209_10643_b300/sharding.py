"""Host-side logic for running the benchmark on several GPUs of one node.

The hot path partitions into independent problems (one Jacobi problem, or a
share of a batch of independent regions, per rank), so ranks exchange no data:
the only collectives are the timing barrier and the max/sum used to report
whole-job throughput.  This module holds that logic so it can be tested with
CPU (gloo) process groups.
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment (1 process: 0, 0, 1)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def shard_lpt(costs: list[float], world: int) -> list[list[int]]:
    """Longest-processing-time assignment of independent items to ``world`` ranks.

    Items are taken in decreasing cost (ties by index) and each goes to the rank
    with the least total so far (ties by rank), so every item lands on exactly
    one rank and the result is deterministic."""
    if world <= 0:
        raise ValueError("world must be positive")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += costs[i]
    for lst in out:
        lst.sort()
    return out


def aggregate_throughput(local_units: float, local_seconds: float, group=None) -> tuple[float, float]:
    """Whole-job (total units, max seconds) over the ranks of ``group``.

    With no process group initialised this is the identity.  Throughput is the
    units all ranks processed divided by the slowest rank's time."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return local_units, local_seconds
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([local_units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return float(u.item()), float(t.item())
