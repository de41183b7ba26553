"""Multi-GPU runs of the sort: one process per GPU, each sorting its own
arrays (replicas; no exchange on the data path).

The sort partitions into independent problems -- whole arrays, or the
segments of a batch -- so N GPUs run N independent sorts and the job's
throughput is the units sorted by all ranks over the slowest rank's time
(weak scaling).  The only collective is that maximum, taken once per
measurement.  These helpers hold the host-side logic, so it can be tested
with the gloo backend on CPU processes.
"""
from __future__ import annotations

import os


def world_info():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of a rank's own synthetic inputs (distinct per rank)."""
    return base + 1_000_003 * rank


def shard_range(n_units: int, rank: int, world: int):
    """[lo, hi) of the units (arrays, segments) that a rank sorts when a fixed
    set is split across ranks: contiguous, sizes differing by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    lo = n_units * rank // world
    hi = n_units * (rank + 1) // world
    return lo, hi


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the job's time is its slowest rank's);
    the value itself when no process group is running."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, seconds_per_rank, device=None) -> float:
    """Whole-job throughput: units of all ranks over the slowest rank's time."""
    import torch
    import torch.distributed as dist

    units = float(units_per_rank)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = torch.tensor([units], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        units = float(t.item())
    return units / max_over_ranks(seconds_per_rank, device)
