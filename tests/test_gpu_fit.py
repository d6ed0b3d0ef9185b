"""Parity of the GPU construction (fst_fit: Algorithm 1 followed by the core refit of
Algorithm 2) with the FP64 oracle of oracle/fit.py, step by step: the interpolated and
filled grid (Sec. 4.1), the ST-HOSVD spectrum, factors and core (Sec. 4.1), the sparse
Legendre columns chosen by leave-one-out (Sec. 3, 4.2), and the final model's predictions."""
import math

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

from oracle import fit as OF
from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _scattered(Q, seed, n_gauss, clustered):
    """FP32 points and values; the oracle gets the same FP32-rounded numbers in FP64."""
    xyz = synth.points(Q, seed=seed, clustered=clustered).astype(np.float32)
    u, clean = synth.field_values(xyz.astype(np.float64), synth.field_spec(seed + 1, n_gauss), seed=seed + 2)
    return xyz, u.astype(np.float32), clean


CASES = [
    dict(Q=20000, grid=(16, 20, 24), frac=0.2, eps=1e-2, max_rank=(5, 6, 4), deg=9, seed=3, cl=0.3, ng=3),
    dict(Q=60000, grid=(32, 32, 32), frac=0.05, eps=1e-3, max_rank=(8, 8, 8), deg=15, seed=5, cl=0.3, ng=6),
    dict(Q=30000, grid=(9, 40, 17), frac=0.02, eps=3e-3, max_rank=(6, 8, 7), deg=12, seed=8, cl=0.0, ng=4),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "x".join(map(str, c["grid"])))
def test_fit_steps_match_oracle(F, oracle_lib, case):
    import torch
    xyz, u, _ = _scattered(case["Q"], case["seed"], case["ng"], case["cl"])
    x64, u64 = xyz.astype(np.float64), u.astype(np.float64)
    Q, grid = case["Q"], case["grid"]
    params = OF.FitParams(grid=grid, sample_frac=case["frac"], eps=case["eps"], max_rank=case["max_rank"],
                          max_degree=case["deg"], oversample=4.0, seed=case["seed"] + 100)
    # oracle, step by step
    n_sub = int(math.ceil(params.sample_frac * Q))
    sub = oracle_lib.sample(params.seed, Q, n_sub)
    U0, filled = OF.interpolate_splat(x64[:, sub], u64[sub], grid)
    U, sweeps = OF.fill_jacobi(U0, filled)
    core, Ws, lams = OF.st_hosvd(U, params.eps, params.max_rank)
    omodel, orep = OF.fit(x64, u64, params, nthreads=8)
    # GPU
    M, rep, tr = F.fit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), grid=grid,
                       sample_frac=params.sample_frac, eps=params.eps, max_rank=params.max_rank,
                       max_degree=params.max_degree, oversample=params.oversample, seed=params.seed,
                       prec="fp32", trace=True)
    # step 1: same subset, same splat and fill (FP64 atomics only reorder the sums)
    assert rep["n_interp"] == n_sub
    assert rep["fill_sweeps"] == sweeps
    assert np.max(np.abs(tr["grid_values"] - U)) <= 1e-12 * np.max(np.abs(U))
    # step 2: spectrum, ranks, factors (sign rule fixes them), core
    assert rep["r_hosvd"] == orep.hosvd_ranks
    assert rep["r"] == orep.ranks
    for k in range(3):
        assert np.max(np.abs(tr["eigvals"][k] - lams[k])) <= 1e-11 * lams[k][0], k
        assert np.max(np.abs(tr["W"][k] - Ws[k])) <= 1e-7, k
    assert rel_l2(tr["core_hosvd"], core) <= 1e-8
    # step 3: the same supports (hence nnz) and leave-one-out errors
    onnz = [n for k in range(3) for n in orep.nnz[k]]
    oloo = [e for k in range(3) for e in orep.loo[k]]
    assert list(tr["col_nnz"]) == onnz
    assert np.allclose(tr["col_loo"], oloo, rtol=1e-6, atol=1e-14)
    okept = [int(j not in orep.dropped[k]) for k in range(3) for j in range(orep.hosvd_ranks[k])]
    assert list(tr["col_kept"]) == okept
    d = M.read()
    for k in range(3):
        assert np.array_equal(d["rowidx"][k], omodel.rowidx[k]), k
        assert np.max(np.abs(d["val"][k] - omodel.val[k])) <= 1e-7, k
    # step 4: the refit (FP32 Gram + PCG vs FP64 Cholesky on the same rows)
    assert rep["m"] == orep.m
    test = synth.points(4000, seed=case["seed"] + 7, clustered=0.0)
    got = M.eval_f64(cuda_tensor(test, torch.float64)).cpu().numpy()
    ref = oracle_lib.eval_points(omodel, test)
    assert rel_l2(got, ref) <= 1e-5
    assert rep["compression_ratio"] == pytest.approx(orep.compression_ratio, rel=1e-12)


def test_fit_drops_dependent_factor_functions(F, oracle_lib):
    """Grid 64^3 with rank caps 24: several noise singular vectors of mode 1 collapse to the
    same constant fit.  The GPU drops exactly the columns the oracle drops (steps 1-3 compared
    with the oracle), and the refit on the independent functions succeeds."""
    import torch
    Q, grid, caps, deg = 1 << 21, (64, 64, 64), (24, 24, 24), 31
    xyz = synth.points(Q, seed=5, clustered=0.3).astype(np.float32)
    u, clean = synth.field_values(xyz.astype(np.float64), synth.field_spec(6, 20), seed=7)
    u = u.astype(np.float32)
    x64, u64 = xyz.astype(np.float64), u.astype(np.float64)
    seed, frac, eps = 11, 0.16, 1e-3
    sub = oracle_lib.sample(seed, Q, int(math.ceil(frac * Q)))
    U0, filled = OF.interpolate_splat(x64[:, sub], u64[sub], grid)
    U, _ = OF.fill_jacobi(U0, filled)
    _, Ws, _ = OF.st_hosvd(U, eps, caps)
    kept_ref, nnz_ref = [], []
    for k in range(3):
        Phi = OF.legendre_matrix(OF.grid_nodes(grid[k]), deg)
        C = np.zeros((deg + 1, Ws[k].shape[1]))
        for j in range(Ws[k].shape[1]):
            rows, coef, _ = OF.sparse_fit(Phi, Ws[k][:, j])
            C[rows, j] = coef
            nnz_ref.append(rows.size)
        kk = OF.independent_columns(C)
        kept_ref += [int(j in kk) for j in range(C.shape[1])]
    assert sum(kept_ref) < len(kept_ref)            # the case does drop columns
    M, rep, tr = F.fit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), grid=grid,
                       sample_frac=frac, eps=eps, max_rank=caps, max_degree=deg, oversample=8.0, seed=seed,
                       prec="bf16", trace=True)
    assert rep["r_hosvd"] == tuple(W.shape[1] for W in Ws)
    assert list(tr["col_nnz"]) == nnz_ref
    assert list(tr["col_kept"]) == kept_ref
    assert sum(rep["r"]) == sum(kept_ref)
    pred = M.eval(cuda_tensor(xyz[:, :200000], torch.float32), prec="fp32").cpu().numpy()
    assert rel_l2(pred, clean[:200000]) < 0.1


def _poly_field(seed, deg, r):
    rng = np.random.default_rng(seed)
    facs = [rng.normal(size=(deg + 1, r[k])) for k in range(3)]
    core = rng.normal(size=r)

    def field(y):
        ws = [npl.legval(y[k], facs[k]).T for k in range(3)]
        return np.einsum("abc,na,nb,nc->n", core, *ws)
    return field


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-6), ("fp32", 1e-5)])
def test_fit_exact_low_rank_polynomial(F, oracle_lib, prec, tol):
    """A separable rank-(2,3,2) polynomial of degree 5 given on the grid is recovered: ranks
    exact, and the refitted model reproduces the field up to the FP32 rounding of the data."""
    import torch
    r, I = (2, 3, 2), 24
    field = _poly_field(7, 5, r)
    g = OF.grid_nodes(I)
    G = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
    gv = field(G).reshape(I, I, I)
    xyz = np.random.default_rng(8).uniform(-1, 1, size=(3, 4000)).astype(np.float32)
    u = field(xyz.astype(np.float64)).astype(np.float32)
    M, rep = F.fit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), grid=(I, I, I), eps=1e-6,
                   max_rank=(4, 4, 4), max_degree=8, oversample=4.0, seed=9, prec=prec, grid_values=gv)
    assert rep["r"] == r
    assert rep["fill_sweeps"] == 0 and rep["n_interp"] == 0
    test = np.random.default_rng(10).uniform(-1, 1, size=(3, 500))
    got = M.eval_f64(cuda_tensor(test, torch.float64)).cpu().numpy()
    assert rel_l2(got, field(test)) <= tol
    # the oracle on the same inputs
    om, orep = OF.fit(xyz.astype(np.float64), u.astype(np.float64),
                      OF.FitParams(grid=(I, I, I), eps=1e-6, max_rank=(4, 4, 4), max_degree=8, oversample=4.0,
                                   seed=9), grid_values=gv)
    assert orep.ranks == r
    assert rel_l2(got, oracle_lib.eval_points(om, test)) <= (1e-9 if prec == "fp64" else 1e-5)


def test_fit_fixed_rank_and_box(F, oracle_lib):
    """fixed_rank keeps min(max_rank, grid) per mode; a non-unit box maps onto [-1,1]^3."""
    import torch
    xyz, u, _ = _scattered(8000, 21, 3, 0.0)
    lo, hi = np.array([2.0, -5.0, 0.5]), np.array([4.0, 3.0, 0.75])
    xb = (lo[:, None] + (xyz.astype(np.float64) + 1) / 2 * (hi - lo)[:, None]).astype(np.float32)
    params = OF.FitParams(grid=(12, 3, 10), sample_frac=0.5, eps=1e-1, max_rank=(5, 5, 5), max_degree=7,
                          oversample=3.0, seed=22, fixed_rank=True)
    M, rep = F.fit(cuda_tensor(xb, torch.float32), cuda_tensor(u, torch.float32), grid=params.grid,
                   sample_frac=params.sample_frac, eps=params.eps, max_rank=params.max_rank,
                   max_degree=params.max_degree, oversample=params.oversample, seed=params.seed,
                   fixed_rank=True, lo=lo, hi=hi)
    assert rep["r"] == (5, 3, 5)
    om, orep = OF.fit(xb.astype(np.float64), u.astype(np.float64), params, lo=lo, hi=hi, nthreads=8)
    assert orep.ranks == (5, 3, 5)
    d = M.read()
    assert np.allclose(d["lo"], lo) and np.allclose(d["hi"], hi)
    got = M.eval_f64(cuda_tensor(xb.astype(np.float64), torch.float64)).cpu().numpy()
    assert rel_l2(got, oracle_lib.eval_points(om, xb.astype(np.float64))) <= 1e-5


def test_fit_degenerate_fields(F):
    """A zero field gives ranks (1,1,1) and a zero model; a constant field gives ranks (1,1,1),
    one degree-0 coefficient per mode, and reproduces the constant."""
    import torch
    xyz = synth.points(5000, seed=31, clustered=0.0).astype(np.float32)
    X = cuda_tensor(xyz, torch.float32)
    M, rep = F.fit(X, torch.zeros(5000, device="cuda"), grid=(8, 8, 8), sample_frac=0.5, max_rank=(3, 3, 3),
                   max_degree=5, prec="fp64")
    assert rep["r"] == (1, 1, 1)
    assert np.all(M.eval_f64(cuda_tensor(xyz, torch.float64)).cpu().numpy() == 0.0)
    M, rep = F.fit(X, torch.full((5000,), 3.0, device="cuda"), grid=(8, 8, 8), sample_frac=0.5,
                   max_rank=(3, 3, 3), max_degree=5, prec="fp64")
    assert rep["r"] == (1, 1, 1) and rep["nnz"] == (1, 1, 1)
    d = M.read()
    assert all(list(d["rowidx"][k]) == [0] for k in range(3))
    got = M.eval_f64(cuda_tensor(xyz, torch.float64)).cpu().numpy()
    assert np.max(np.abs(got - 3.0)) <= 1e-12


def test_fit_smallest_grid(F):
    """grid 2 x 2 x 2 with degree 0..1: the construction runs at its minimum sizes."""
    import torch
    xyz, u, _ = _scattered(3000, 41, 2, 0.0)
    M, rep = F.fit(cuda_tensor(xyz, torch.float32), cuda_tensor(u, torch.float32), grid=(2, 2, 2),
                   sample_frac=1.0, max_rank=(2, 2, 2), max_degree=1, eps=0.0)
    assert rep["r"] == (2, 2, 2)
    assert rep["m"] == 32


@pytest.mark.parametrize("bad", [dict(grid=(1, 8, 8)), dict(grid=(8, 8, 257)), dict(max_degree=64),
                                 dict(max_rank=(0, 2, 2)), dict(max_rank=(33, 2, 2)), dict(sample_frac=0.0),
                                 dict(sample_frac=1.5), dict(oversample=0.0), dict(eps=-1.0)])
def test_fit_rejects_bad_parameters(F, bad):
    import torch
    xyz = torch.zeros((3, 100), device="cuda")
    u = torch.zeros(100, device="cuda")
    kw = dict(grid=(8, 8, 8), max_rank=(2, 2, 2), max_degree=3)
    kw.update(bad)
    with pytest.raises(F.FstError) as e:
        F.fit(xyz, u, **kw)
    assert e.value.status == -1
