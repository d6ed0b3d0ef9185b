"""Parity of the GPU core refit (fst_refit / fst_refit_f64) with the FP64 oracle
(Sec. 5, eq. rand_core; Algorithm 2 with uniform sampling)."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _problem(r, p, Q, seed, n_gauss=5, clustered=0.3, orthonormal=False):
    m = synth.random_model(r, p, seed=seed, density=0.7, orthonormal=orthonormal)
    xyz = synth.points(Q, seed=seed + 1, clustered=clustered)
    u, _ = synth.field_values(xyz, synth.field_spec(seed + 2, n_gauss), seed=seed + 3)
    return m, xyz, u


@pytest.mark.parametrize("r,p,Q,ms", [((2, 3, 2), (4, 5, 3), 500, 4.0), ((4, 4, 4), (7, 7, 7), 3000, 4.0),
                                      ((8, 8, 8), (15, 15, 15), 20000, 4.0), ((5, 7, 3), (9, 6, 11), 4000, 8.0),
                                      ((6, 5, 9), (10, 10, 10), 270, 1.0)])
def test_refit_fp64_matches_oracle(F, oracle_lib, r, p, Q, ms):
    import torch
    m, xyz, u = _problem(r, p, Q, seed=sum(r) + Q)
    R = m.R
    mm = min(int(np.ceil(ms * R)), Q)
    seed = 1234 + Q
    idx = oracle_lib.sample(seed, Q, mm)
    ref, rc = oracle_lib.refit(m, xyz, u, idx, nthreads=8)
    assert rc == 0
    M = F.Model(m)
    rep = M.refit(cuda_tensor(xyz, torch.float64), cuda_tensor(u, torch.float64), mm, seed=seed, prec="fp64")
    got = M.read()["alpha"]
    # both sides solve the same normal equations in FP64: they agree to the FP64 rounding
    # bound kappa(G) * eps, which only matters for the square (m = R) edge case
    G, _, _ = oracle_lib.normal_equations(m, xyz, u, idx)
    kappa = np.linalg.cond(G)
    assert rel_l2(got, ref) < max(TOL_FP64, 10 * kappa * np.finfo(np.float64).eps), kappa
    assert rep["m"] == mm


@pytest.mark.parametrize("r,p,Q", [((4, 4, 4), (7, 7, 7), 3000), ((8, 8, 8), (15, 15, 15), 20000),
                                   ((12, 10, 11), (15, 15, 15), 40000)])
def test_refit_fp32_matches_oracle(F, oracle_lib, r, p, Q):
    """FP32 Gram + FP32 Cholesky preconditioner, FP64-accumulated refinement; the oracle is
    given the same FP32-rounded data.  Explicit rows (idx) and seeded rows agree."""
    import torch
    m, xyz, u = _problem(r, p, Q, seed=sum(r) * 3 + Q, orthonormal=True)
    x32, u32 = xyz.astype(np.float32), u.astype(np.float32)
    mm = min(8 * m.R, Q)
    seed = 99 + Q
    idx = oracle_lib.sample(seed, Q, mm)
    ref, rc = oracle_lib.refit(m, x32.astype(np.float64), u32.astype(np.float64), idx, nthreads=8)
    M = F.Model(m)
    xt, ut = cuda_tensor(x32, torch.float32), cuda_tensor(u32, torch.float32)
    rep = M.refit(xt, ut, mm, seed=seed, prec="fp32")
    got = M.read()["alpha"]
    assert rel_l2(got, ref) < TOL_FP32, rep
    M2 = F.Model(m)
    M2.refit(xt, ut, mm, prec="fp32", idx=cuda_tensor(idx, torch.int64))
    assert rel_l2(M2.read()["alpha"], ref) < TOL_FP32
    # predictions with the refitted core
    pred = M.eval(xt).cpu().numpy()
    refp = oracle_lib.eval_points(m.with_alpha(ref), x32.astype(np.float64), nthreads=8)
    assert rel_l2(pred, refp) < TOL_FP32


def test_refit_all_rows_is_full_ls(F, oracle_lib):
    import torch
    m, xyz, u = _problem((3, 4, 3), (6, 6, 6), 2000, seed=17)
    M = F.Model(m)
    M.refit(cuda_tensor(xyz, torch.float64), cuda_tensor(u, torch.float64), 2000, seed=5, prec="fp64")
    A = oracle_lib.design_matrix(m, xyz, np.arange(2000))
    ref = np.linalg.lstsq(A, u, rcond=None)[0]
    assert rel_l2(M.read()["alpha"].ravel(), ref) < TOL_FP64


def test_refit_errors(F):
    import torch
    m, xyz, u = _problem((4, 4, 4), (5, 5, 5), 1000, seed=23)
    M = F.Model(m)
    xt, ut = cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32)
    with pytest.raises(F.FstError) as e:
        M.refit(xt, ut, 63, prec="fp32")          # m < R
    assert e.value.status == -5
    # every row at the same point: A has rank one, G is singular in any precision
    same = np.repeat(xyz[:, :1], 1000, axis=1)
    with pytest.raises(F.FstError) as e:
        M.refit(cuda_tensor(same, torch.float32), ut, 640, prec="fp32")
    assert e.value.status == -4
    # the model is unchanged by the failed refits
    assert np.array_equal(M.read()["alpha"], m.alpha)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_refit_full_size_normal_residual(F, oracle_lib, prec):
    """2^24 points, ranks 24^3, degree 31, m = 8R = 110,592 rows: the refitted core satisfies the
    normal equations of the sampled problem, checked by the oracle in FP64 with the exact design.
    BF16 is the benchmark's path (packed operand, tensor-core Gram over five strips of
    super-tiles, tensor-core Cholesky, conjugate gradients)."""
    import torch
    Q = 1 << 24
    m = synth.random_model((24, 24, 24), (31, 31, 31), seed=202, orthonormal=True)
    xyz = synth.points(Q, seed=203, clustered=0.3, dtype=np.float32)
    u, _ = synth.field_values(xyz, synth.field_spec(204, 20), seed=205)
    u = u.astype(np.float32)
    M = F.Model(m)
    R = m.R
    mm = 8 * R
    rep = M.refit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), mm, seed=206, prec=prec)
    alpha = M.read()["alpha"]
    idx = oracle_lib.sample(206, Q, mm)
    x64 = xyz.astype(np.float64)
    u64 = u.astype(np.float64)
    g = oracle_lib.normal_residual(m, x64, u64, idx, alpha, nthreads=16)
    h = oracle_lib.normal_residual(m, x64, u64, idx, np.zeros(R), nthreads=16)
    print(prec, "normal residual", np.linalg.norm(g) / np.linalg.norm(h), rep)
    assert np.linalg.norm(g) < 1e-5 * np.linalg.norm(h), rep
