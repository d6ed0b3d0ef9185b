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


def _refit_worker(rank, world, port, q):
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1907_05884_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        model = synth.random_model((4, 3, 5), (7, 6, 8), seed=71, orthonormal=True)
        Q = 3000
        xyz = synth.points(Q, seed=72)
        u, _ = synth.field_values(xyz, synth.field_spec(73, 3), seed=74)
        m = 8 * model.R + 3
        idx = oracle.sample(75, Q, m)

        def partial(start, end):
            G, h, _ = oracle.normal_equations(model, xyz, u, idx[start:end])
            return torch.from_numpy(G), torch.from_numpy(h)

        def solve(G, h):
            L = np.linalg.cholesky(G.numpy())
            return np.linalg.solve(L.T, np.linalg.solve(L, h.numpy()))

        alpha = shard.refit_split(partial, solve, m, world, rank)
        q.put((rank, alpha.numpy(), shard.row_range(m, world, rank)))
    finally:
        dist.destroy_process_group()


def test_refit_rows_split_over_two_ranks(oracle_lib):
    """One refit with its sampled rows split over two gloo ranks: the all-reduced partial
    normal equations give the core of the single-rank refit (the oracle's, over all rows) on
    both ranks, and the two row ranges tile the sample."""
    import numpy as np
    from paper_1907_05884_gb300 import synth
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_refit_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    model = synth.random_model((4, 3, 5), (7, 6, 8), seed=71, orthonormal=True)
    Q = 3000
    xyz = synth.points(Q, seed=72)
    u, _ = synth.field_values(xyz, synth.field_spec(73, 3), seed=74)
    m = 8 * model.R + 3
    ref, rc = oracle_lib.refit(model, xyz, u, oracle_lib.sample(75, Q, m))
    assert rc == 0
    for _, alpha, _ in res:
        assert np.linalg.norm(alpha - ref.reshape(-1)) < 1e-10 * np.linalg.norm(ref)
    assert res[0][2] == (0, (m + 1) // 2) and res[1][2] == ((m + 1) // 2, m)


def test_row_range_tiles_the_sample():
    for m in (1, 7, 100, 110592):
        for world in (1, 2, 3, 8):
            ranges = [shard.row_range(m, world, r) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            assert max(e - s for s, e in ranges) - min(e - s for s, e in ranges) <= 1
