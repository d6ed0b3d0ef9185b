"""Order-4 models on the GPU (fst_model4_create, fst_eval4, fst_eval4_f64, fst_refit4; eq.
func_tuck with d = 4, eq. rand_core) against the order-4 oracle (oracle/order4.py): every rank
bucket of the fourth mode, the paper's SP4D ranks 30 x 38 x 5 x 11 (Table 1), ragged point
counts and points outside the box."""
import numpy as np
import pytest

from oracle import order4 as O4
from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


SHAPES = [((3, 4, 2, 5), (6, 7, 5, 8)), ((30, 38, 5, 11), (40, 40, 15, 20)), ((7, 1, 9, 16), (12, 0, 10, 17)),
          ((2, 3, 4, 31), (3, 5, 6, 40)), ((9, 2, 3, 64), (10, 4, 6, 70)), ((1, 1, 1, 1), (0, 3, 0, 2))]


def _points(n, seed):
    x = synth.points4(n, seed=seed)
    x[:, :4] = np.array([[1.0, -1.0, 1.05, -1.1]] * 4)      # box corners and slight extrapolation
    return x


@pytest.mark.parametrize("r,p", SHAPES)
@pytest.mark.parametrize("n", [1, 129, 3001])
def test_eval4_matches_oracle(F, r, p, n):
    import torch
    m = synth.random_model4(r, p, seed=sum(r) + n, density=0.6, lo=[-1, -2, 0, 0], hi=[1, 2, 3, 1])
    x = _points(max(n, 4), sum(r) + 1)[:, :n]
    x[1] = 2 * x[1]            # the second box is [-2, 2], the third [0, 3]
    x[2] = 1.5 * (x[2] + 1)
    x[3] = 0.5 * (x[3] + 1)
    ref = O4.eval_points(m, x)
    M = F.Model4(m)
    got64 = M.eval(cuda_tensor(np.ascontiguousarray(x), torch.float64)).cpu().numpy()
    assert rel_l2(got64, ref) < 1e-10, rel_l2(got64, ref)
    got32 = M.eval(cuda_tensor(np.ascontiguousarray(x.astype(np.float32)), torch.float32)).cpu().numpy()
    ref32 = O4.eval_points(m, x.astype(np.float32).astype(np.float64))
    assert rel_l2(got32, ref32) < 1e-5, rel_l2(got32, ref32)


def test_eval4_empty_and_core_roundtrip(F):
    import torch
    m = synth.random_model4((3, 2, 4, 2), (4, 4, 4, 4), seed=5)
    M = F.Model4(m)
    out = M.eval(torch.empty((4, 0), device="cuda", dtype=torch.float32))
    assert out.numel() == 0
    assert np.array_equal(M.core(), m.alpha)


@pytest.mark.parametrize("r,p,Q", [((3, 4, 2, 5), (6, 7, 5, 8), 6000), ((5, 6, 4, 7), (9, 9, 6, 9), 20000),
                                   ((2, 9, 3, 33), (4, 11, 5, 40), 30000)])
def test_refit4_matches_oracle(F, oracle_lib, r, p, Q):
    """The refitted core against the oracle's least-squares solution over the same rows."""
    import torch
    m = synth.random_model4(r, p, seed=Q, orthonormal=True)
    x = synth.points4(Q, seed=Q + 1).astype(np.float32)
    u, _ = synth.field_values4(x.astype(np.float64), synth.field_spec(Q + 2, 4), seed=Q + 3)
    u = u.astype(np.float32)
    mm = 4 * m.R
    idx = oracle_lib.sample(Q + 4, Q, mm)
    ref = O4.refit(m, x.astype(np.float64), u.astype(np.float64), idx)
    M = F.Model4(m)
    rep = M.refit(cuda_tensor(x, torch.float32), cuda_tensor(u, torch.float32), mm, seed=Q + 4)
    got = M.core()
    assert rel_l2(got, ref) < 1e-5, (rel_l2(got, ref), rep)
    assert rep["refine_steps"] >= 1 and rep["m"] == mm
    # the residual of the refitted core is orthogonal to the columns, in FP64 over those rows
    assert O4.normal_residual(m, x.astype(np.float64), u.astype(np.float64), idx, got) < 1e-5


def _torch_rows(m, x, idx):
    """FP64 factor values of the rows idx, computed here with torch (the Legendre recurrence of
    eq. sparse, independent of the library) for a normal-residual check at full size."""
    import torch
    U = []
    for k in range(4):
        t = torch.from_numpy(2 * (x[k, idx] - m.lo[k]) / (m.hi[k] - m.lo[k]) - 1).cuda()
        L = [torch.ones_like(t), t]
        for n in range(1, m.p[k]):
            L.append(((2 * n + 1) * t * L[n] - n * L[n - 1]) / (n + 1))
        P = torch.stack(L[:m.p[k] + 1], 1) * torch.sqrt(2 * torch.arange(m.p[k] + 1, device="cuda",
                                                                           dtype=torch.float64) + 1)
        W = torch.zeros(m.p[k] + 1, m.r[k], dtype=torch.float64, device="cuda")
        for j in range(m.r[k]):
            s0, e0 = m.colptr[k][j], m.colptr[k][j + 1]
            W[torch.from_numpy(m.rowidx[k][s0:e0].astype(np.int64)).cuda(), j] = torch.from_numpy(m.val[k][s0:e0]).cuda()
        U.append(P @ W)
    return U


def test_refit4_sp4d_ranks_recover_an_exact_core(F, oracle_lib):
    """The paper's SP4D ranks (R = 62,700) at m = 4R rows: values of a model at the points (its
    FP64 evaluation, rounded to FP32), refitted from a zero core.  The refitted core solves the
    sampled normal equations (the residual of A^T A alpha = A^T b, in FP64 at full size, below
    1e-5 of A^T b), and it is the model's core up to the perturbation of the least-squares
    solution by the FP32 rounding of u and of the factor values (relative 6e-8 each), which
    kappa(A) amplifies: below 1e-4 for kappa(A) <= 1,000."""
    import torch
    m = synth.random_model4((30, 38, 5, 11), (40, 40, 15, 20), seed=77, orthonormal=True)
    Q = 1 << 19
    x = synth.points4(Q, seed=78)
    M = F.Model4(m)
    u = M.eval(cuda_tensor(x, torch.float64)).float().contiguous()
    M0 = F.Model4(m.with_alpha(np.zeros(m.r)))
    mm = 4 * m.R
    x32 = x.astype(np.float32)
    rep = M0.refit(cuda_tensor(x32, torch.float32), u, mm, seed=79, prec="bf16x3", max_refine=200)
    got = M0.core()
    print("SP4D refit", rep, "rel-L2 vs the model's core", rel_l2(got, m.alpha))
    assert rel_l2(got, m.alpha) < 1e-4, (rel_l2(got, m.alpha), rep)
    # the normal residual over the sampled rows, FP64, in blocks of rows
    idx = oracle_lib.sample(79, Q, mm)
    U = _torch_rows(m, x32.astype(np.float64), idx)
    b = u.double()[torch.from_numpy(idx.astype(np.int64)).cuda()]
    a = torch.from_numpy(got.reshape(-1)).cuda()
    res = torch.zeros_like(a)
    atb = torch.zeros_like(a)
    for s0 in range(0, mm, 4096):
        sl = slice(s0, min(mm, s0 + 4096))
        A = torch.einsum("ni,nj,nk,nl->nijkl", U[0][sl], U[1][sl], U[2][sl], U[3][sl]).reshape(-1, m.R)
        res += A.T @ (A @ a - b[sl])
        atb += A.T @ b[sl]
        del A
    nr = float(res.norm() / atb.norm())
    print("SP4D normal residual", nr)
    assert nr < 1e-5, nr


def test_refit4_errors(F):
    import torch
    m = synth.random_model4((3, 3, 3, 3), (4, 4, 4, 4), seed=9)
    M = F.Model4(m)
    x = cuda_tensor(synth.points4(100, seed=10).astype(np.float32), torch.float32)
    u = torch.zeros(100, device="cuda")
    with pytest.raises(F.FstError) as e:
        M.refit(x, u, 50, seed=1)                  # m < R = 81
    assert e.value.status == -5
    with pytest.raises(F.FstError):
        F.Model4(synth.random_model4((65, 1, 1, 1), (70, 1, 1, 1), seed=1))   # rank above 64
