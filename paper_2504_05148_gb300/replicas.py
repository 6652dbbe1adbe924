"""Frame sharding across ranks (one process per GPU).

Frames are independent problems, so N GPUs run N replicas of the pipeline
on disjoint frame sets with no collective on the data path (weak scaling).
The only cross-rank operations are a barrier around the timed region and the
max of the per-rank elapsed times, which defines the job's step time.
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (defaults: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def frame_seeds(rank: int, batch: int, base: int = 2000, stride: int = 1000) -> list[int]:
    """Seeds of the frames rank `rank` processes: disjoint across ranks."""
    if batch > stride:
        raise ValueError("batch larger than the per-rank seed stride")
    return [base + rank * stride + i for i in range(batch)]


def max_over_ranks(value: float, device=None) -> float:
    """Max of a per-rank float over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()
