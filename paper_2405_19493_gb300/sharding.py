"""Stream sharding across ranks (one process per GPU).

Streams are independent, so N ranks split the work with no collective on the
data path: rank r owns streams [r * n_per_rank, (r + 1) * n_per_rank) of the
global stream index, i.e. seeds base + r * n_per_rank + s.  The only collective
is the timing reduction (max over ranks) after the timed region.
"""

from __future__ import annotations

import numpy as np

from . import workloads


def rank_streams(rank: int, world: int, n_per_rank: int) -> tuple[int, int]:
    """Global stream range [lo, hi) owned by `rank` (weak scaling: fixed per-rank size)."""
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world {world}")
    return rank * n_per_rank, (rank + 1) * n_per_rank


def rank_seeds(rank: int, world: int, n_per_rank: int,
               base: int = workloads.SEED_BASE) -> np.ndarray:
    lo, _ = rank_streams(rank, world, n_per_rank)
    return workloads.seeds(n_per_rank, base=base + lo)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Max of a per-rank scalar over the process group (identity without one)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
