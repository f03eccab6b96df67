"""Data-parallel sharding of populations across ranks (one process per GPU).

Genomes are independent (Section 3.3's forward has no cross-genome term), so
a multi-GPU run shards by population: every rank evaluates its own genomes
and no collective touches the data path.  Only the timing is combined: the
job's time is the slowest rank's, and its throughput is the units of all
ranks over that time (weak scaling).
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def population_seed(rank: int, base: int = 0) -> int:
    """Seed of the population a rank evaluates (distinct per rank)."""
    return base + rank


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity with one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, slowest_seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return units_per_rank * world / slowest_seconds
