"""The evaluator autotuner: both variants of a size class (factor values on the CUDA cores,
or on the tensor cores) are measured and either one, forced by hand, matches the FP64 oracle
(eq. func_tuck) within the precision's tolerance."""
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


@pytest.mark.parametrize("prec", ["bf16x3", "bf16", "tf32"])
@pytest.mark.parametrize("r,p", [((24, 24, 24), (31, 31, 31)), ((6, 11, 9), (20, 63, 9)), ((5, 4, 3), (8, 8, 8))])
def test_autotune_variants_match_oracle(F, oracle_lib, prec, r, p):
    import torch
    model = synth.random_model(r, p, seed=sum(r) + sum(p), orthonormal=True)
    M = F.Model(model)
    res = M.autotune(prec, n_probe=1 << 16)
    assert res["choice"] in (0, 1)
    assert res["ms_cuda_core_factors"] > 0 and res["ms_tensor_core_factors"] > 0
    xyz = synth.points(20000, seed=3, clustered=0.3)
    ref = oracle_lib.eval_points(model, xyz, nthreads=8)
    X = cuda_tensor(xyz.astype(np.float32), torch.float32)
    outs = []
    for choice in (0, 1):
        M.set_variant(prec, choice)
        M.prepare(prec)
        outs.append(M.eval(X, prec=prec).cpu().numpy())
        assert rel_l2(outs[-1], ref) <= TOL[prec], choice
    M.set_variant(prec, -1)


def test_autotune_degree_beyond_tensor_core_factors(F):
    """Degree 64 and above: only the CUDA-core factor step can serve the class."""
    model = synth.random_model((8, 8, 8), (70, 10, 10), seed=5, orthonormal=True)
    M = F.Model(model)
    res = M.autotune("bf16x3", n_probe=1 << 14)
    assert res["choice"] == 0 and res["ms_tensor_core_factors"] == -1.0
