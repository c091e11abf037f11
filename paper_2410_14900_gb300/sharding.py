"""Work partition of the reconstruction across ranks (one GPU each).

The path shards into independent problems (one volume each), so N ranks
reconstruct N volumes with no collective on the data path; only the
benchmark's barrier and its max-over-ranks timing talk to each other.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the phantom that rank `rank` reconstructs (disjoint per rank)."""
    return int(base_seed) + 1000 * int(rank)


def rank_views(n_views: int, rank: int, world: int):
    """Contiguous view range of a rank when one problem's filter is split by
    views (each view is independent in the filter)."""
    per = (n_views + world - 1) // world
    lo = min(n_views, rank * per)
    return lo, min(n_views, lo + per)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The slowest rank's time (the whole job finishes with it)."""
    if dist is None or not dist.is_available() or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_ms_per_volume(ms_step_max: float, volumes_per_rank: int, world: int) -> float:
    """ms per volume of the whole job: all ranks' volumes in the slowest step."""
    return float(ms_step_max) / (int(volumes_per_rank) * int(world))
