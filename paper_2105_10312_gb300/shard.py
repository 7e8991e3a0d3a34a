"""Host-side sharding for N GPUs (one process per GPU).

Task sets are independent, so N ranks shard the work with no data-path
collective: each rank draws and decides its own batch (weak scaling), and the
only communication is a barrier and a max/sum of scalars over ranks for the
timing and the aggregate counts.
"""
from __future__ import annotations

import os

_STRIDE = 1000003  # seed offset between ranks


def dist_env():
    """(rank, world, local_rank) from the torchrun environment (defaults: single process)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


def rank_seed(seed: int, rank: int) -> int:
    """Seed of a rank's own batch: ranks draw disjoint, reproducible batches."""
    return int(seed) + _STRIDE * int(rank)


def shard_bounds(n: int, rank: int, world: int):
    """Contiguous [lo, hi) share of n units for a rank (sizes differ by at most 1)."""
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi


def _reduce(value: float, op, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    if device is None:
        device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device=None) -> float:
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM, device)


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
