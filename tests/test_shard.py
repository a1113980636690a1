"""Host logic of the multi-rank runs (one rank per GPU, independent problems per rank):
contiguous sharding, the torchrun environment, and the max-over-ranks timing and
whole-job rate over a real two-rank gloo process group on the CPU."""
import os
import socket

import pytest

from paper_1606_01273_gb300 import shard


def test_shard_range_covers_every_unit_once():
    for n in range(0, 40):
        for ws in range(1, 9):
            seen = []
            sizes = []
            for r in range(ws):
                lo, hi = shard.shard_range(n, r, ws)
                assert 0 <= lo <= hi <= n
                seen.extend(range(lo, hi))
                sizes.append(hi - lo)
            assert seen == list(range(n))
            assert max(sizes) - min(sizes) <= 1


def test_dist_env(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert shard.dist_env() == (1, 0, 0)
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert shard.dist_env() == (2, 1, 1)
    monkeypatch.setenv("RANK", "2")
    with pytest.raises(ValueError):
        shard.dist_env()


def test_single_process_passthrough():
    assert shard.max_over_ranks(3.25) == 3.25
    assert shard.sum_over_ranks(7) == 7
    assert shard.job_rate(10, 2.0) == 5.0
    with pytest.raises(ValueError):
        shard.job_rate(1, 0.0)


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        # rank r "took" 1.5 + r seconds for 3 + r units of its own shard
        lo, hi = shard.shard_range(11, rank, ws)
        slowest = shard.max_over_ranks(1.5 + rank)
        units = shard.sum_over_ranks(hi - lo)
        rate = shard.job_rate(units, slowest)
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as fh:
            fh.write(f"{lo} {hi} {slowest} {units} {rate}\n")
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    rows = [open(tmp_path / f"r{r}.txt").read().split() for r in range(ws)]
    (lo0, hi0, s0, u0, v0), (lo1, hi1, s1, u1, v1) = rows
    assert (int(lo0), int(hi0), int(lo1), int(hi1)) == (0, 6, 6, 11)
    assert float(s0) == float(s1) == 2.5               # the slowest rank bounds the job
    assert int(u0) == int(u1) == 11                    # every rank's units count
    assert float(v0) == float(v1) == pytest.approx(11 / 2.5)


def _moments_main(rank, ws, port, out_dir):
    import numpy as np
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        rng = np.random.default_rng(100 + rank)
        local = rng.standard_normal((8, 5 ** 3 + 5 ** 2 + 5)) * 10.0 ** rng.integers(-8, 8, (8, 1))
        np.save(os.path.join(out_dir, f"m{rank}.npy"), local)
        tot = shard.sum_moments_fixed_order(local)
        np.save(os.path.join(out_dir, f"s{rank}.npy"), tot)
        lo, hi = shard.closed_range(70, rank, ws)
        with open(os.path.join(out_dir, f"c{rank}.txt"), "w") as fh:
            fh.write(f"{lo} {hi}\n")
    finally:
        dist.destroy_process_group()


def test_split_solve_exchange_two_gloo_ranks(tmp_path):
    """The one exchange step of a solve split over ranks: the closed orbitals are shared
    contiguously (every orbital to one rank) and the per-class moments are summed in rank
    order, so every rank holds bitwise the same sum, equal to the ordered sum computed
    alone."""
    import numpy as np
    import torch.multiprocessing as mp
    ws = 3
    mp.spawn(_moments_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    parts = [np.load(tmp_path / f"m{r}.npy") for r in range(ws)]
    ref = parts[0].copy()
    for p in parts[1:]:
        ref += p
    for r in range(ws):
        assert np.array_equal(np.load(tmp_path / f"s{r}.npy"), ref)
    ranges = [tuple(map(int, open(tmp_path / f"c{r}.txt").read().split())) for r in range(ws)]
    assert ranges == [(0, 24), (24, 47), (47, 70)]
