"""Host-side logic of multi-GPU runs: one independent lattice (replica) per rank.

The D2Q37 work partitions into independent lattices (Sec. 3: no dependency between sites within
a step; an ensemble's members never interact), so a run on N GPUs gives each rank its own lattice
and needs no collective on the data path. Ranks only meet at a barrier before and after the timed
region and agree on the slowest rank's time (weak scaling: work per rank is fixed).
"""
from __future__ import annotations

import os


def rank_env() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (1 process if unset)."""
    def get(name, default):
        try:
            return int(os.environ.get(name, default))
        except ValueError:
            return default
    return get("RANK", 0), get("WORLD_SIZE", 1), get("LOCAL_RANK", 0)


def replica_seed(rank: int, base: int = 0) -> int:
    """Seed of rank's replica: distinct lattices per rank, reproducible per (base, rank)."""
    return base + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of `value` over all ranks (the value itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_mlups(sites_per_rank: int, steps: int, max_ms: float, world: int) -> float:
    """Whole-job MLUPS: every rank's sites x steps over the slowest rank's time."""
    if max_ms <= 0:
        raise ValueError("elapsed time must be positive")
    return world * sites_per_rank * steps / (max_ms * 1e-3) / 1e6
