"""Weak-scaling replicas: independent bundle-adjustment problems spread over
ranks, one process per GPU.

The optimiser's work partitions into independent problems (scenes, submaps,
jobs), so ranks share nothing on the data path: each rank loads and solves
its own problems with the library, and ranks meet only at a barrier before
and after a timed region and in one max-over-ranks reduction of the elapsed
time.  Throughput is the units all ranks processed divided by the slowest
rank's time.  Works with any torch.distributed backend (gloo on CPU, nccl on
GPUs); with world size 1 no process group is needed.
"""
from __future__ import annotations

import os
from typing import NamedTuple


class RankInfo(NamedTuple):
    rank: int
    world: int
    local: int


def rank_info(env=None) -> RankInfo:
    """RANK / WORLD_SIZE / LOCAL_RANK as set by torchrun (defaults: one rank)."""
    env = os.environ if env is None else env
    return RankInfo(int(env.get("RANK", "0")), int(env.get("WORLD_SIZE", "1")), int(env.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world: int) -> list[int]:
    """Items of this rank: round-robin, so ranks get similar size mixes when
    items are listed in arrival or generation order.  The shards partition
    range(n_items)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    return list(range(rank, n_items, world))


def scene_rep(rank: int, base: int = 0) -> int:
    """Replica index of a rank's scene: every rank solves a different seeded
    scene of the same configuration."""
    return base + rank


class Group:
    """Barrier and max-over-ranks reduction of one process group (or none)."""

    def __init__(self, dist=None, device=None):
        self.dist = dist
        self.device = device  # where reduction tensors live (a CUDA device for nccl)

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

    def sum(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())


def throughput(units_per_rank: float, seconds_this_rank: float, group: Group, world: int) -> tuple[float, float]:
    """(whole-job units per second, slowest rank's seconds): every rank
    processes units_per_rank units; the job ends when the slowest rank does."""
    slowest = group.max(seconds_this_rank)
    return units_per_rank * world / slowest, slowest
