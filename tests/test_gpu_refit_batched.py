"""Batched refits (fst_refit_batched): many instances of uneven size refitted concurrently on
several streams give exactly the cores that one-at-a-time refits give (Sec. 5, eq. rand_core),
and those agree with the FP64 oracle."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

CASES = [((4, 5, 6), (7, 9, 8), 6000), ((8, 8, 8), (15, 15, 15), 30000), ((12, 10, 9), (15, 15, 15), 50000),
         ((2, 3, 4), (3, 4, 5), 700), ((16, 12, 10), (23, 19, 17), 120000), ((6, 6, 6), (11, 11, 11), 9000)]


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _instances(cases, seed0):
    out = []
    for i, (r, p, Q) in enumerate(cases):
        s = seed0 + 17 * i
        m = synth.random_model(r, p, seed=s, density=0.7, orthonormal=True)
        xyz = synth.points(Q, seed=s + 1, clustered=0.3).astype(np.float32)
        u, _ = synth.field_values(xyz.astype(np.float64), synth.field_spec(s + 2, 4), seed=s + 3)
        out.append((m, xyz, u.astype(np.float32), min(8 * m.R, Q), 1000 + s))
    return out


@pytest.mark.parametrize("prec,streams", [("bf16", 4), ("bf16x3", 3), ("tf32", 2), ("fp32", 6), ("bf16", 1)])
def test_batched_equals_sequential(F, prec, streams):
    import torch
    inst = _instances(CASES, 500)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    seq = []
    for (m, _, _, mm, sd), x, u in zip(inst, xs, us):
        M = F.Model(m)
        M.refit(x, u, mm, seed=sd, prec=prec)
        seq.append(M.read()["alpha"])
    models = [F.Model(m) for m, _, _, _, _ in inst]
    reps = F.refit_batched(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec=prec,
                           streams=streams)
    assert len(reps) == len(inst)
    for k, M in enumerate(models):
        got = M.read()["alpha"]
        assert np.array_equal(got, seq[k]), (k, prec, rel_l2(got, seq[k]))
        assert reps[k]["m"] == inst[k][3]


def test_batched_matches_oracle(F, oracle_lib):
    import torch
    inst = _instances(CASES[:4], 900)
    models = [F.Model(m) for m, _, _, _, _ in inst]
    F.refit_batched(models, [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst],
                    [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst], [i[3] for i in inst],
                    [i[4] for i in inst], prec="bf16x3", streams=4)
    for M, (m, x, u, mm, sd) in zip(models, inst):
        idx = oracle_lib.sample(sd, x.shape[1], mm)
        ref, rc = oracle_lib.refit(m, x.astype(np.float64), u.astype(np.float64), idx, nthreads=8)
        assert rc == 0
        assert rel_l2(M.read()["alpha"], ref) < 1e-5


def test_batched_edge_cases(F):
    import torch
    inst = _instances(CASES[:2], 1300)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    M = F.Model(inst[0][0])
    # the same model twice is refused before any work
    with pytest.raises(RuntimeError):
        F.refit_batched([M, M], xs, us, [inst[0][3]] * 2, [1, 2])
    # an empty batch is a no-op
    assert F.refit_batched([], [], [], [], []) == []
    # more streams than items
    models = [F.Model(m) for m, _, _, _, _ in inst]
    F.refit_batched(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec="bf16", streams=16)
    with pytest.raises(RuntimeError):
        F.refit_batched(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], streams=0)
    # a failing item (m < R) reports its error; the batch still returns
    with pytest.raises(RuntimeError):
        F.refit_batched(models, xs, us, [inst[0][3], 3], [1, 2], prec="bf16")


def test_batched_many_mixed(F):
    """Two dozen instances with residual/Gram kernels of different shared-memory sizes on eight
    streams at once (the launches interleave across host threads)."""
    import torch
    rng = np.random.default_rng(77)
    cases = []
    for _ in range(24):
        r = tuple(int(v) for v in rng.integers(3, 17, size=3))
        Q = int(rng.integers(9 * int(np.prod(r)), 90000))
        cases.append((r, tuple(min(2 * v + 3, 31) for v in r), Q))
    inst = _instances(cases, 2100)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    seq = []
    for (m, _, _, mm, sd), x, u in zip(inst, xs, us):
        M = F.Model(m)
        M.refit(x, u, mm, seed=sd, prec="bf16")
        seq.append(M.read()["alpha"])
    for rep in range(2):
        models = [F.Model(m) for m, _, _, _, _ in inst]
        F.refit_batched(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec="bf16", streams=8)
        for k, M in enumerate(models):
            assert np.array_equal(M.read()["alpha"], seq[k]), (rep, k)
