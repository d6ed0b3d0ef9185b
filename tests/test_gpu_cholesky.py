"""Parity of the FP32 Cholesky of the refit (fst_cholesky_f32: FP32 panels, BF16x3 tensor-core
trailing updates) with the FP64 oracle factorisation (the solve step of Algorithm 2)."""
import numpy as np
import pytest

from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

# BF16x3 products carry ~2^-16 relative error; the backward error ||L L^T - G|| / ||G|| of the
# factorisation is bounded by a small multiple of that, independent of the conditioning.
TOL_BACKWARD = 2e-5


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _spd(R, seed, rows_per_col=4):
    """A normal matrix A^T A / m of m = rows_per_col * R Gaussian rows (kappa ~ 9 for 4)."""
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(rows_per_col * R, R))
    return ((A.T @ A) / A.shape[0]).astype(np.float32)


# sizes: below one panel, exactly one/two panels, ragged tails, several trailing tiles
@pytest.mark.parametrize("R", [1, 7, 100, 128, 129, 255, 256, 300, 640, 1000, 2053])
def test_cholesky_matches_oracle(F, oracle_lib, R):
    import torch
    G = _spd(R, seed=R)
    # the strict upper triangle is not read: poison it, and check it is left untouched
    Gp = G.copy()
    iu = np.triu_indices(R, 1)
    Gp[iu] = np.float32(7.0)
    Gd = cuda_tensor(Gp, torch.float32)
    F.cholesky_f32(Gd)
    out = Gd.cpu().numpy()
    assert np.array_equal(out[iu], Gp[iu])
    L = np.tril(out).astype(np.float64)
    G64 = G.astype(np.float64)
    assert np.linalg.norm(L @ L.T - G64) / np.linalg.norm(G64) <= TOL_BACKWARD
    Lref, rc = oracle_lib.cholesky(G64)
    assert rc == 0
    Lref = np.tril(Lref)
    # forward error: kappa(G) ~ 9 amplifies the backward error modestly
    assert rel_l2(L, Lref) <= 20 * TOL_BACKWARD
    assert np.all(np.diag(L) > 0)


def test_cholesky_ill_conditioned_still_backward_stable(F):
    """kappa ~ 1e5: the factor is still a backward-stable factor of G (what a preconditioner needs)."""
    import torch
    R = 700
    rng = np.random.default_rng(3)
    Qm, _ = np.linalg.qr(rng.normal(size=(R, R)))
    lam = np.logspace(0, -5, R)
    G = ((Qm * lam) @ Qm.T).astype(np.float32)
    G = (G + G.T) / 2
    Gd = cuda_tensor(G, torch.float32)
    F.cholesky_f32(Gd)
    L = np.tril(Gd.cpu().numpy()).astype(np.float64)
    G64 = G.astype(np.float64)
    assert np.linalg.norm(L @ L.T - G64) / np.linalg.norm(G64) <= TOL_BACKWARD


@pytest.mark.parametrize("R,bad", [(50, 10), (300, 200), (1000, 999)])
def test_cholesky_reports_not_spd(F, R, bad):
    """A matrix with one negative eigen-direction is reported, not hung on or silently factored."""
    import torch
    G = _spd(R, seed=5).astype(np.float64)
    v = np.zeros(R)
    v[bad] = 1.0
    G = G - 3.0 * np.max(np.diag(G)) * np.outer(v, v)
    Gd = cuda_tensor(G.astype(np.float32), torch.float32)
    with pytest.raises(F.FstError) as e:
        F.cholesky_f32(Gd)
    assert e.value.status == -4
