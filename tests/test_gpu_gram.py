"""Parity of the normal-matrix assembly (fst_normal_matrix): CUDA-core FP32 and tensor-core
TF32 / BF16 / BF16x3 against the oracle's FP64 normal equations (Sec. 5, eq. rand_core), and
the refit in every precision against the oracle after refinement."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

# Frobenius-relative error of the lower triangle of G: operand rounding (TF32 2^-11,
# BF16 2^-9 per factor product; BF16x3 drops the lo*lo term, ~2^-17) plus FP32 accumulation.
TOL_G = {"fp32": 1e-5, "tf32": 2e-3, "bf16": 1e-2, "bf16x3": 5e-5}


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _lower(A):
    return A[np.tril_indices(A.shape[0])]


@pytest.mark.parametrize("r,m", [((8, 8, 8), 4096), ((5, 7, 9), 1001), ((3, 2, 2), 64), ((12, 10, 14), 8192),
                                 ((1, 1, 1), 33)])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "bf16x3"])
def test_normal_matrix_matches_oracle(F, oracle_lib, r, m, prec):
    import torch
    model = synth.random_model(r, (15, 15, 15), seed=sum(r) + m, orthonormal=True)
    Q = 3 * m + 7
    xyz = synth.points(Q, seed=m).astype(np.float32)
    u, _ = synth.field_values(xyz, synth.field_spec(3, 4), seed=4)
    u = u.astype(np.float32)
    idx = oracle_lib.sample(17, Q, m)
    Gref, href, _ = oracle_lib.normal_equations(model, xyz.astype(np.float64), u.astype(np.float64), idx,
                                                nthreads=8)
    M = F.Model(model)
    G, h = F.normal_matrix(M, cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32),
                           cuda_tensor(idx, torch.int64), prec=prec)
    G = G.cpu().numpy().astype(np.float64)
    assert rel_l2(_lower(G), _lower(Gref)) < TOL_G[prec]
    assert rel_l2(h.cpu().numpy(), href) < 1e-5


@pytest.mark.parametrize("prec", ["tf32", "bf16", "bf16x3"])
def test_refit_tensor_core_precisions(F, oracle_lib, prec):
    """Refinement with the FP64-accumulated residual brings every Gram precision to the
    FP32 tolerance of the oracle's least-squares solution."""
    import torch
    model = synth.random_model((12, 10, 11), (15, 15, 15), seed=5, orthonormal=True)
    Q = 40000
    xyz = synth.points(Q, seed=6).astype(np.float32)
    u, _ = synth.field_values(xyz, synth.field_spec(7, 5), seed=8)
    u = u.astype(np.float32)
    mm = 8 * model.R
    idx = oracle_lib.sample(9, Q, mm)
    ref, _ = oracle_lib.refit(model, xyz.astype(np.float64), u.astype(np.float64), idx, nthreads=8)
    M = F.Model(model)
    rep = M.refit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), mm, seed=9, prec=prec)
    assert rel_l2(M.read()["alpha"], ref) < 1e-5, rep
