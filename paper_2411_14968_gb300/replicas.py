"""Timing of N independent replicas, one process per GPU.

The partitioned skyline shards naturally (partitions are independent until
the final phase), but no cross-GPU exchange step is implemented: several
GPUs run independent replicas of the same workload (weak scaling), and no
data moves between ranks.  What the ranks share is only the measurement protocol -- a
barrier on both sides of the timed region and the maximum of the per-rank
times -- which this module provides over torch.distributed (NCCL on GPUs,
gloo on CPU for the tests).
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world size, local rank) from the torchrun environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Replicas:
    def __init__(self, world: int, device=None):
        self.world = world
        self.device = device

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(self, v: float) -> float:
        """The slowest rank's value: a job is done when its last rank is."""
        if self.world == 1:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum_over_ranks(self, v: float) -> float:
        if self.world == 1:
            return v
        import torch
        import torch.distributed as dist
        t = torch.tensor([v], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())


def throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time."""
    return units_per_rank * world / max_seconds
