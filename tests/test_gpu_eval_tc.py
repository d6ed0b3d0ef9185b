"""Parity of the tensor-core evaluation (fst_eval with TF32 / BF16 / BF16x3 core contraction)
with the FP64 oracle (Sec. 2, eq. func_tuck; Sec. 6, reconstruction by basis evaluation).

Tolerances (relative L2 over the evaluated points) follow the operand rounding of the
contraction: BF16x3 carries ~16 mantissa bits (hi+lo, the lo*lo product dropped), TF32 10,
BF16 7; the factor values are FP32 in every mode."""
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


CASES = [((24, 24, 24), (31, 31, 31), 3001), ((1, 1, 1), (0, 0, 0), 1), ((5, 9, 3), (11, 4, 13), 129),
         ((8, 8, 8), (15, 15, 15), 4096), ((13, 30, 17), (20, 31, 25), 1009), ((32, 7, 32), (40, 9, 63), 777),
         ((24, 24, 24), (63, 63, 63), 2500)]


@pytest.mark.parametrize("r,p,n", CASES)
@pytest.mark.parametrize("prec", ["bf16x3", "tf32", "bf16"])
def test_eval_tc_matches_oracle(F, oracle_lib, r, p, n, prec):
    import torch
    m = synth.random_model(r, p, seed=sum(r) + n, density=0.6)
    xyz = synth.points(n, seed=n + 11).astype(np.float32)
    ref = oracle_lib.eval_points(m, xyz.astype(np.float64), nthreads=8)
    M = F.Model(m)
    M.prepare(prec)
    got = M.eval(cuda_tensor(xyz, torch.float32), prec=prec).cpu().numpy()
    F.eval_check()
    err = rel_l2(got, ref)
    print(prec, r, n, err)
    assert err < TOL[prec]


def test_eval_tc_core_update_and_big_n(F, oracle_lib):
    """A core replaced after preparation is picked up; 2^22 points in one launch, sampled."""
    import torch
    m = synth.random_model((24, 24, 24), (31, 31, 31), seed=3, orthonormal=True)
    M = F.Model(m)
    n = 1 << 22
    xyz = synth.points(n, seed=4, clustered=0.3).astype(np.float32)
    xt = cuda_tensor(xyz, torch.float32)
    got1 = M.eval(xt, prec="bf16x3").cpu().numpy()
    new_core = np.random.default_rng(5).normal(size=m.alpha.shape)
    M.set_core(new_core)
    got2 = M.eval(xt, prec="bf16x3").cpu().numpy()
    F.eval_check()
    sel = np.random.default_rng(6).choice(n, 2048, replace=False)
    ref1 = oracle_lib.eval_points(m, xyz[:, sel].astype(np.float64), nthreads=8)
    ref2 = oracle_lib.eval_points(m.with_alpha(new_core), xyz[:, sel].astype(np.float64), nthreads=8)
    assert rel_l2(got1[sel], ref1) < TOL["bf16x3"]
    assert rel_l2(got2[sel], ref2) < TOL["bf16x3"]
