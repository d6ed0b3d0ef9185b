"""The multi-GPU layout of the benchmark (weak scaling by point set, no data-path
collective): two gloo ranks on CPU check the per-rank seeds, the max-over-ranks job time and
the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1907_05884_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 10.0 + 5.0 * rank                      # rank 1 is the slow one
        job = shard.job_time_ms(local, world)
        q.put((rank, shard.rank_seed(2024, rank), job, shard.job_throughput(1000, world, 4, job)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_weak_scaling():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = [r[1] for r in res]
    assert len(set(seeds)) == world                     # independent fields per rank
    assert all(r[2] == 15.0 for r in res)               # the slowest rank's time, on every rank
    # 2 ranks x 1000 points x 4 steps in 15 ms
    assert all(r[3] == pytest.approx(2 * 1000 * 4 / 0.015 / 1e6) for r in res)


def test_single_rank_is_identity():
    assert shard.job_time_ms(12.5, 1) == 12.5
    assert shard.job_throughput(2 ** 24, 1, 5, 100.0) == pytest.approx(5 * 2 ** 24 / 0.1 / 1e6)
