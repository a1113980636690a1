"""Host logic of the multi-process (one rank per GPU) runs.

The solve path shards by independent problems (geometries, requests): each rank solves
its own units with no data-path collective, and only the timing is combined — the
slowest rank's time bounds the job, and the whole-job rate counts every rank's units
(weak scaling).  Used by bench.py under torchrun; tested with gloo ranks on the CPU."""
from __future__ import annotations

import os


def dist_env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 alone)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws < 1 or not 0 <= rank < ws or local < 0:
        raise ValueError(f"bad torchrun environment: WORLD_SIZE={ws} RANK={rank} LOCAL_RANK={local}")
    return ws, rank, local


def shard_range(n_units: int, rank: int, ws: int):
    """Contiguous block [lo, hi) of n_units for this rank; the first n_units % ws ranks
    take one more, so every unit goes to exactly one rank."""
    if n_units < 0 or ws < 1 or not 0 <= rank < ws:
        raise ValueError("bad shard request")
    q, r = divmod(n_units, ws)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def max_over_ranks(x: float, device=None) -> float:
    """The maximum of x over the ranks of the default process group (x alone without one).
    device: where the reduction tensor lives (cuda for NCCL, cpu for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(n: int, device=None) -> int:
    """The sum of an integer count over the ranks (n alone without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return int(n)
    t = torch.tensor([int(n)], dtype=torch.int64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return int(t.item())


def job_rate(units_all_ranks: int, slowest_s: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    if slowest_s <= 0.0:
        raise ValueError("non-positive time")
    return units_all_ranks / slowest_s
