"""Multi-GPU layouts (one process per GPU).

Weak scaling of the benchmark: the path shards by point set, every rank holds its own field
(its own seeded points, values and model), refits and evaluates it with no data exchange.
The only collectives are the timing barrier and the maximum of the per-rank times (the
slowest rank sets the job time); the whole-job throughput counts the points of all ranks.

One refit over several ranks (refit_split): the sampled rows of a single refit are split
over the ranks and the partial normal equations are summed by one all-reduce.

Host logic only: it is exercised with the gloo backend on CPU; bench.py runs the weak-scaling
layout over NCCL.
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


# ----------------------------------------------------------------------------- one refit over ranks
def row_range(m: int, world: int, rank: int) -> tuple[int, int]:
    """Rank `rank`'s contiguous share [start, end) of the m sampled rows (sizes differ by at
    most one)."""
    base, extra = divmod(int(m), int(world))
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def refit_split(partial, solve, m: int, world: int, rank: int, device: str = "cpu"):
    """One least-squares core refit (Sec. 5, eq. rand_core) with its m sampled rows split over
    the ranks.  The normal equations are sums over rows, so each rank forms the partial
    G_r = A_r^T A_r and h_r = A_r^T b_r of its rows, one all-reduce (SUM) of each gives
    G = A^T A and h = A^T b on every rank, rank 0 solves G alpha = h and broadcasts alpha.

    partial(start, end) -> (G_r, h_r): torch tensors (R x R with at least the lower triangle
    valid, and R) of this rank's rows [start, end) of the sample; on a GPU rank,
    fst.normal_matrix over idx[start:end].  solve(G, h) -> alpha (R,): rank 0's solve of the
    summed equations.  Returns alpha (float64, on `device`) on every rank."""
    import torch
    import torch.distributed as dist
    start, end = row_range(m, world, rank)
    G, h = partial(start, end)
    G = G.contiguous()
    h = h.contiguous()
    if world > 1:
        dist.all_reduce(G, op=dist.ReduceOp.SUM)
        dist.all_reduce(h, op=dist.ReduceOp.SUM)
    R = h.numel()
    alpha = solve(G, h) if rank == 0 else torch.empty(R, dtype=torch.float64, device=device)
    alpha = torch.as_tensor(alpha, dtype=torch.float64, device=device).contiguous()
    if world > 1:
        dist.broadcast(alpha, src=0)
    return alpha
