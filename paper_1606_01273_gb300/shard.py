"""Host logic of the multi-process (one rank per GPU) runs.

Two ways to shard.  Across independent problems (geometries, requests): each rank solves
its own units with no data-path collective, and only the timing is combined — the
slowest rank's time bounds the job, and the whole-job rate counts every rank's units
(weak scaling).  Within one solve: each rank takes a contiguous range of the closed
orbitals for the class-H and class-G work (options.closed_begin/closed_end; classes A-F
on the rank whose range starts at 0), and the one exchange step is a fixed-order sum of
the ranks' per-class moments (caspt2_get_moments), after which every rank forms H^eff,
E_MS, R and lambda from the same sum (caspt2_finalize_moments).  Used by bench.py under
torchrun; tested with gloo ranks on the CPU."""
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


def closed_range(nclosed: int, rank: int, ws: int):
    """(closed_begin, closed_end) of this rank's share of one solve's closed orbitals."""
    return shard_range(nclosed, rank, ws)


def sum_moments_fixed_order(local, device=None):
    """The element-wise sum over ranks of each rank's moment array, added in rank order
    (0, 1, ...) so that every rank obtains bitwise the same sum whatever the backend's
    reduction order; the array alone without a process group."""
    import numpy as np
    import torch
    import torch.distributed as dist
    a = np.ascontiguousarray(local, dtype=np.float64)
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return a.copy()
    t = torch.from_numpy(a).to(device or "cpu")
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    out = parts[0].clone()
    for p in parts[1:]:
        out += p
    return out.cpu().numpy()
