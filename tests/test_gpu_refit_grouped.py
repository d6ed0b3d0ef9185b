"""Grouped refits (fst_refit_grouped): the factorisations and conjugate gradients of many
instances of uneven size run in shared launches, and every core equals the one a refit of the
instance alone gives, bit for bit (Sec. 5, eq. rand_core; Algorithm 2 per instance); those
agree with the FP64 oracle."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

# every rank class of r3 (<= 8, 16, 24, 32), several panel counts of the factorisation (R up
# to 4,896 = 39 panels of 128, block rows of the solves from 1 to 77) and a ragged last panel
CASES = [((4, 5, 6), (7, 9, 8), 6000), ((8, 8, 8), (15, 15, 15), 30000), ((12, 10, 9), (15, 15, 15), 50000),
         ((2, 3, 4), (3, 4, 5), 700), ((16, 12, 10), (23, 19, 17), 120000), ((6, 6, 6), (11, 11, 11), 9000),
         ((17, 12, 24), (23, 15, 31), 90000), ((3, 2, 30), (7, 7, 31), 20000), ((1, 1, 1), (2, 2, 2), 50)]


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


def _alone(F, inst, xs, us, prec, **kw):
    cores, reps = [], []
    for (m, _, _, mm, sd), x, u in zip(inst, xs, us):
        M = F.Model(m)
        reps.append(M.refit(x, u, mm, seed=sd, prec=prec, **kw))
        cores.append(M.read()["alpha"])
    return cores, reps


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "tf32", "fp32"])
def test_grouped_equals_alone(F, prec):
    import torch
    inst = _instances(CASES, 500)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    seq, sreps = _alone(F, inst, xs, us, prec)
    models = [F.Model(m) for m, _, _, _, _ in inst]
    reps = F.refit_grouped(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec=prec)
    assert len(reps) == len(inst)
    for k, M in enumerate(models):
        got = M.read()["alpha"]
        assert np.array_equal(got, seq[k]), (k, prec, rel_l2(got, seq[k]))
        assert reps[k]["m"] == inst[k][3]
        assert reps[k]["refine_steps"] == sreps[k]["refine_steps"], k
        assert reps[k]["first_rel_change"] == sreps[k]["first_rel_change"], k


def test_grouped_matches_oracle(F, oracle_lib):
    import torch
    inst = _instances(CASES[:4] + CASES[7:8], 900)
    models = [F.Model(m) for m, _, _, _, _ in inst]
    F.refit_grouped(models, [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst],
                    [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst], [i[3] for i in inst],
                    [i[4] for i in inst], prec="bf16")
    for M, (m, x, u, mm, sd) in zip(models, inst):
        idx = oracle_lib.sample(sd, x.shape[1], mm)
        ref, rc = oracle_lib.refit(m, x.astype(np.float64), u.astype(np.float64), idx, nthreads=8)
        assert rc == 0
        assert rel_l2(M.read()["alpha"], ref) < 1e-5


def test_grouped_edge_cases(F):
    import torch
    inst = _instances(CASES[:3], 1300)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    M = F.Model(inst[0][0])
    with pytest.raises(RuntimeError):               # the same model twice
        F.refit_grouped([M, M], xs[:2], us[:2], [inst[0][3]] * 2, [1, 2])
    assert F.refit_grouped([], [], [], [], []) == []
    # a failing item (m < R) reports its error after the others have been refitted
    seq, _ = _alone(F, inst, xs, us, "bf16")
    models = [F.Model(m) for m, _, _, _, _ in inst]
    with pytest.raises(RuntimeError) as e:
        F.refit_grouped(models, xs, us, [inst[0][3], 3, inst[2][3]], [i[4] for i in inst], prec="bf16")
    assert "item 1" in str(e.value)
    assert np.array_equal(models[0].read()["alpha"], seq[0])
    assert np.array_equal(models[2].read()["alpha"], seq[2])
    assert np.array_equal(models[1].read()["alpha"], F.Model(inst[1][0]).read()["alpha"])   # unchanged
    # the FP64 factorisation runs every item alone, as fst_refit does with that option
    seq64, _ = _alone(F, inst, xs, us, "bf16", fp64_cholesky=True)
    models = [F.Model(m) for m, _, _, _, _ in inst]
    F.refit_grouped(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec="bf16", fp64_cholesky=True)
    for k, Mk in enumerate(models):
        assert np.array_equal(Mk.read()["alpha"], seq64[k]), k
    # no refinement: the factor's solution alone
    seq0, _ = _alone(F, inst, xs, us, "bf16", max_refine=0)
    models = [F.Model(m) for m, _, _, _, _ in inst]
    F.refit_grouped(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec="bf16", max_refine=0)
    for k, Mk in enumerate(models):
        assert np.array_equal(Mk.read()["alpha"], seq0[k]), k


def test_grouped_many_mixed(F):
    """Forty instances with ranks drawn per mode from 3..24 (the batching workload's range)."""
    import torch
    rng = np.random.default_rng(78)
    cases = []
    for _ in range(40):
        r = tuple(int(v) for v in rng.integers(3, 25, size=3))
        Q = int(rng.integers(9 * int(np.prod(r)), 150000))
        cases.append((r, tuple(min(v + 7, 31) for v in r), Q))
    inst = _instances(cases, 2100)
    xs = [cuda_tensor(x, torch.float32) for _, x, _, _, _ in inst]
    us = [cuda_tensor(u, torch.float32) for _, _, u, _, _ in inst]
    seq, _ = _alone(F, inst, xs, us, "bf16")
    for rep in range(2):
        models = [F.Model(m) for m, _, _, _, _ in inst]
        F.refit_grouped(models, xs, us, [i[3] for i in inst], [i[4] for i in inst], prec="bf16")
        for k, M in enumerate(models):
            assert np.array_equal(M.read()["alpha"], seq[k]), (rep, k)
