"""Batched evaluation (fst_eval_batched): many models with uneven ranks and point counts in
one persistent launch.  Every instance matches the FP64 oracle at the precision's tolerance and,
where it shares the batch's rank padding, the single-instance evaluation bit for bit."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import EVAL_TOL, rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

TOL = EVAL_TOL


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _instances(count, seed, r_lo=4, r_hi=24, n_lo=1e2, n_hi=3e4):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        r = tuple(int(v) for v in rng.integers(r_lo, r_hi + 1, size=3))
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        m = synth.random_model(r, (31, 31, 31), seed=seed * 1000 + i, density=0.6)
        xyz = synth.points(n, seed=seed * 1000 + i, clustered=0.3).astype(np.float32)
        out.append((m, xyz))
    return out


@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "fp32"])
def test_batched_matches_oracle(F, oracle_lib, prec):
    import torch
    inst = _instances(24, seed=7)
    models = [F.Model(m) for m, _ in inst]
    xs = [cuda_tensor(x, torch.float32) for _, x in inst]
    outs = F.eval_batched(models, xs, prec=prec)
    torch.cuda.synchronize()
    F.eval_check()
    for (m, x), o in zip(inst, outs):
        ref = oracle_lib.eval_points(m, x.astype(np.float64), nthreads=8)
        assert rel_l2(o.cpu().numpy(), ref) < TOL[prec], (m.r, x.shape)


def test_batched_equals_single_bitwise(F):
    """Instances whose r3 share the padding bucket (17..24) give bit-identical results alone
    and in the mix; an empty instance is allowed."""
    import torch
    inst = _instances(12, seed=8, r_lo=17, r_hi=24)
    models = [F.Model(m) for m, _ in inst]
    xs = [cuda_tensor(x, torch.float32) for _, x in inst]
    empty = torch.empty((3, 0), dtype=torch.float32, device="cuda")
    outs = F.eval_batched(models + [models[0]], xs + [empty], prec="bf16x3")
    for Mi, x, o in zip(models, xs, outs):
        alone = Mi.eval(x, prec="bf16x3")
        assert torch.equal(alone, o)
    assert outs[-1].numel() == 0


def test_plan_graph_replay(F, oracle_lib):
    """A prepared plan launches without allocating or synchronising: captured into a CUDA
    graph and replayed, it reproduces the eager batched result exactly."""
    import torch
    inst = _instances(16, seed=9)
    models = [F.Model(m) for m, _ in inst]
    xs = [cuda_tensor(x, torch.float32) for _, x in inst]
    eager = F.eval_batched(models, xs, prec="bf16x3")
    outs = [torch.zeros_like(o) for o in eager]
    plan = F.EvalPlan(models, xs, outs, prec="bf16x3")
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        plan.run()                     # warm-up outside capture (kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    for o in outs:
        o.zero_()
    with torch.cuda.graph(g):
        plan.run()
    g.replay()
    torch.cuda.synchronize()
    F.eval_check()
    for e, o in zip(eager, outs):
        assert torch.equal(e, o)
