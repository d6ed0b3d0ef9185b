"""Parity of the GPU Algorithm 2 with mixing (fst_refit_mixed: random signs D, normalised
Walsh-Hadamard F over the padded rows, uniform sampling S; Sec. 5) with the FP64 oracle."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


@pytest.fixture(scope="module")
def mix(oracle_lib):
    from oracle import mixing
    return mixing


def _problem(r, p, Q, seed, clustered=0.3):
    m = synth.random_model(r, p, seed=seed, density=0.8, orthonormal=True)
    xyz = synth.points(Q, seed=seed + 1, clustered=clustered)
    u, _ = synth.field_values(xyz, synth.field_spec(seed + 2, 5), seed=seed + 3)
    return m, xyz, u


@pytest.mark.parametrize("r,p,Q,mult", [((4, 3, 5), (7, 6, 8), 1500, 4), ((6, 6, 6), (11, 11, 11), 5000, 4),
                                        ((8, 8, 8), (15, 15, 15), 20000, 4), ((3, 4, 2), (5, 6, 4), 1024, 8),
                                        ((5, 7, 3), (9, 6, 11), 3000, 2)])
def test_mixed_refit_matches_oracle(F, mix, oracle_lib, r, p, Q, mult):
    import torch
    m, xyz, u = _problem(r, p, Q, seed=sum(r) + Q)
    mm = mult * m.R
    ref, rc = mix.refit_mixed(m, xyz, u, mm, seed_signs=17 + Q, seed_rows=19 + Q)
    assert rc == 0
    M = F.Model(m)
    rep = F.refit_mixed(M, cuda_tensor(xyz, torch.float64), cuda_tensor(u, torch.float64), mm, 17 + Q, 19 + Q)
    got = M.read()["alpha"]
    # both sides solve the same sampled mixed system in FP64 (the oracle by QR, the GPU by the
    # normal equations): they agree to the FP64 bound kappa(A)^2 eps of the normal equations
    A, b = mix.mixed_system(m, xyz, u, 17 + Q)
    idx = oracle_lib.sample(19 + Q, A.shape[0], mm)
    kappa = np.linalg.cond(A[idx])
    assert rel_l2(got, ref) < max(1e-10, 10 * kappa ** 2 * np.finfo(np.float64).eps), kappa
    assert rep["m"] == mm


def test_all_mixed_rows_give_the_full_least_squares(F, oracle_lib):
    """With all N mixed rows the solution is the plain least squares over the Q points."""
    import torch
    m, xyz, u = _problem((4, 4, 4), (7, 7, 7), 3000, seed=91)
    Q = xyz.shape[1]
    N = 4096
    M = F.Model(m)
    F.refit_mixed(M, cuda_tensor(xyz, torch.float64), cuda_tensor(u, torch.float64), N, 5, 6)
    A = oracle_lib.design_matrix(m, xyz, np.arange(Q, dtype=np.int64))
    ref = np.linalg.lstsq(A, u, rcond=None)[0]
    assert rel_l2(M.read()["alpha"].ravel(), ref) < 1e-10


def test_noise_free_recovery_and_errors(F, oracle_lib):
    import torch
    m = synth.random_model((3, 4, 2), (5, 6, 4), seed=71, density=1.0, orthonormal=True)
    xyz = synth.points(2000, seed=72)
    W = oracle_lib.design_matrix(m, xyz, np.arange(2000, dtype=np.int64))
    a_true = np.random.default_rng(73).standard_normal(m.R)
    u = W @ a_true
    M = F.Model(m)
    xt, ut = cuda_tensor(xyz, torch.float64), cuda_tensor(u, torch.float64)
    F.refit_mixed(M, xt, ut, 3 * m.R, 74, 75)
    assert rel_l2(M.read()["alpha"].ravel(), a_true) < 1e-10
    with pytest.raises(RuntimeError):
        F.refit_mixed(M, xt, ut, m.R - 1, 1, 2)       # fewer rows than unknowns
    with pytest.raises(RuntimeError):
        F.refit_mixed(M, xt, ut, 4096, 1, 2)          # more rows than the 2048 mixed rows
