"""Weak-scaling layout of the benchmark across GPUs (one process per GPU).

The path shards by point set: every rank holds its own field (its own seeded points, values
and model), refits and evaluates it with no data exchange.  The only collectives are the
timing barrier and the maximum of the per-rank times (the slowest rank sets the job time);
the whole-job throughput counts the points of all ranks.  Host logic only: it is exercised
with the gloo backend on CPU, and bench.py runs it over NCCL.
"""
from __future__ import annotations


def rank_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s workload: independent fields per rank, reproducible per run."""
    return int(base) + 17 * int(rank)


def job_time_ms(local_ms: float, world: int, device: str = "cpu") -> float:
    """The job's time: the maximum of the ranks' times (all-reduce MAX; no-op for one rank)."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(points_per_rank: int, world: int, steps: int, job_ms: float) -> float:
    """Whole-job Mpoints/s: all ranks' points over the slowest rank's time."""
    return world * points_per_rank * steps / (job_ms / 1e3) / 1e6
