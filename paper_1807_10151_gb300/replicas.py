"""Independent replicas, one process per GPU.

The SupPCG path shards only across independent problems: each rank solves its
own problem (its own seeds), and the ranks meet only at a barrier around the
timed region and to take the slowest rank's time; no collective touches the
data path.  These helpers are the rank arithmetic of the benchmark, kept free
of CUDA so that they run on CPU process groups too.
"""
from __future__ import annotations


def rank_seeds(rank: int, phantom_seed: int, noise_seed: int) -> tuple[int, int]:
    """Seeds of rank r's problem: the base seeds offset by r (distinct problems)."""
    return phantom_seed + rank, noise_seed + rank


def slowest(seconds: float, dist=None, device=None) -> float:
    """The maximum over ranks of a local duration (the job's time); `dist` is
    torch.distributed with an initialised group, or None for one process."""
    if dist is None:
        return float(seconds)
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds_max
