"""Rank plumbing of the multi-GPU benchmark.

The batched scan shards by instance: the independent solves of one scan are
split into disjoint subsets of nearly equal cost, one per rank (strong
scaling: the job is fixed and each GPU takes 1/N of it), so the data path
has no collective.  Only a barrier around the timed region and the maximum
of the per-rank times cross ranks; the whole-job throughput is the units of
the whole scan divided by that maximum.  Ranks are read from the torchrun
environment (RANK, WORLD_SIZE, LOCAL_RANK, MASTER_ADDR/PORT).
"""
from __future__ import annotations

import os


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Ranks:
    """Barrier and max-reduce over the ranks of one job (no-ops alone)."""

    def __init__(self, backend: str = "nccl", device=None):
        self.rank, self.world, self.local = env_rank()
        self.device = device
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            kw = {"device_id": device} if backend == "nccl" and device is not None else {}
            dist.init_process_group(backend, **kw)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if self.dist is None:
            return float(x)
        import torch
        dev = self.device if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def shard(costs, world: int):
    """Split items of the given costs into ``world`` disjoint subsets of
    nearly equal total cost (longest first, each to the lightest subset);
    returns the item indices of each subset, in increasing order."""
    loads = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def job_throughput(total_units: float, t_max: float) -> float:
    """Whole-job units per second: the units of all ranks over the slowest
    rank's time."""
    return total_units / t_max
