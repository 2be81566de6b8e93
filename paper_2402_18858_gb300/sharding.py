"""Multi-GPU layout of the chemistry step: cells are independent (Eq. 2 per cell), so N ranks
process N independent batches (weak scaling) with no data-path collective.  The only
collectives are the benchmark's barrier and the max-over-ranks reduction of the step time."""
from __future__ import annotations

import torch


def rank_state_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s batch: every rank integrates its own seeded cells."""
    return int(base_seed) + 1000 * int(rank)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(cells_per_rank: int, world: int, seconds_max: float) -> float:
    """Whole-job cells/s: all ranks' cells over the slowest rank's time."""
    return cells_per_rank * world / seconds_max
