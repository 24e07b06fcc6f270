"""Replica (data-parallel) execution across GPUs of one node.

The columns of the solve are independent, so N GPUs run N independent batches
(weak scaling) with no data exchange: each rank draws its own columns (seed
offset by rank), solves them, and only the timing is reduced across ranks
(max over ranks) to form the whole-job throughput.
"""
from __future__ import annotations

import os


def dist_info():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_seed(base_seed: int, rank: int, ncol: int) -> int:
    """Seed of rank `rank`'s batch: disjoint per-column seed ranges."""
    return base_seed + rank * ncol


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a per-rank scalar (timing) over the process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ncol_per_rank: int, world: int, steps: int, max_seconds: float) -> float:
    """Whole-job column-solves per second: all ranks' columns over the slowest rank's time."""
    return ncol_per_rank * world * steps / max_seconds
