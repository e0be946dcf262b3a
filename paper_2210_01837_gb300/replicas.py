"""Independent replicas across ranks (one process per GPU).

The mobility product has no exchange step between problems: every rank owns a whole periodic
box with its own particles, so N GPUs run N independent products.  The only cross-rank traffic
is host-side bookkeeping around the timed region: a barrier on both sides and the maximum of
the per-rank elapsed times, from which the whole-job throughput is formed.  Nothing here
touches the data path.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass(frozen=True)
class RankEnv:
    rank: int
    world: int
    local: int


def rank_env(environ=None) -> RankEnv:
    """Rank, world size and local rank as set by torchrun (defaults: a single process)."""
    env = os.environ if environ is None else environ
    return RankEnv(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def replica_seed_offset(rank: int, base: int = 3) -> int:
    """Seed offset of a rank's particle draw: every replica simulates a different suspension."""
    if rank < 0:
        raise ValueError("rank must be non-negative")
    return base + rank


class Collective:
    """Barrier and max-reduction over ranks; a no-op object when there is one rank."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(world: int, units_per_rank: int, t_max: float) -> float:
    """Units processed by all ranks divided by the slowest rank's time (weak scaling)."""
    if world < 1 or units_per_rank < 0:
        raise ValueError("world must be >= 1 and units non-negative")
    if not (t_max > 0):
        raise ValueError("elapsed time must be positive")
    return world * units_per_rank / t_max
