"""Pins of the oracle's least-squares core refit (Sec. 5, eq. rand_core, Algorithm 2)."""
import numpy as np
import numpy.polynomial.legendre as npl
import pytest
import scipy.fft

from paper_1907_05884_gb300 import synth


def _design_numpy(model, xyz, idx):
    """Measurement matrix built independently: w_j by numpy legval, rows as np.kron(w1, w2, w3)."""
    ws = []
    for k in range(3):
        t = 2 * (xyz[k, idx] - model.lo[k]) / (model.hi[k] - model.lo[k]) - 1
        W = model.dense(k) * np.sqrt(2 * np.arange(model.p[k] + 1) + 1)[:, None]
        ws.append(np.stack([npl.legval(t, W[:, j]) for j in range(model.r[k])], axis=1))
    return np.stack([np.kron(np.kron(ws[0][s], ws[1][s]), ws[2][s]) for s in range(len(idx))])


@pytest.fixture(scope="module")
def problem():
    m = synth.random_model((4, 3, 5), (7, 6, 8), seed=41, density=0.8)
    xyz = synth.points(3000, seed=42)
    u, _ = synth.field_values(xyz, synth.field_spec(43, 5), seed=44)
    return m, xyz, u


def test_design_matrix_order(oracle_lib, problem):
    m, xyz, _ = problem
    idx = synth.row_indices(xyz.shape[1], 100, seed=45)
    A = oracle_lib.design_matrix(m, xyz, idx)
    assert np.max(np.abs(A - _design_numpy(m, xyz, idx))) < 1e-12


def test_normal_equations_against_numpy(oracle_lib, problem):
    m, xyz, u = problem
    idx = synth.row_indices(xyz.shape[1], 400, seed=46)
    G, h, btb = oracle_lib.normal_equations(m, xyz, u, idx, nthreads=2)
    A = _design_numpy(m, xyz, idx)
    assert np.max(np.abs(G - A.T @ A)) < 1e-10 * np.max(np.abs(G))
    assert np.max(np.abs(h - A.T @ u[idx])) < 1e-10 * np.max(np.abs(h))
    assert abs(btb - u[idx] @ u[idx]) < 1e-10 * btb


def test_refit_normal_residual_and_full_ls(oracle_lib, problem):
    """m = Q: the sampled problem is the full LS of eq. rand_core; compare numpy lstsq."""
    m, xyz, u = problem
    Q = xyz.shape[1]
    idx = oracle_lib.sample(7, Q, Q)
    alpha, rc = oracle_lib.refit(m, xyz, u, idx)
    assert rc == 0
    A = _design_numpy(m, xyz, idx)
    ref = np.linalg.lstsq(A, u, rcond=None)[0]
    assert np.linalg.norm(alpha.ravel() - ref) < 1e-10 * np.linalg.norm(ref)
    g = A.T @ (A @ alpha.ravel() - u)
    assert np.linalg.norm(g) < 1e-12 * np.linalg.norm(A.T @ u)
    g2 = oracle_lib.normal_residual(m, xyz, u, idx, alpha)
    assert np.linalg.norm(g2) < 1e-12 * np.linalg.norm(A.T @ u)


def test_refit_exact_recovery(oracle_lib, problem):
    """u in span(W): any sampled set of full column rank recovers alpha exactly."""
    m, xyz, _ = problem
    Q = xyz.shape[1]
    idx_all = np.arange(Q)
    u = oracle_lib.eval_points(m, xyz)
    for mm in (2 * m.R, 4 * m.R):
        idx = oracle_lib.sample(8 + mm, Q, mm)
        alpha, rc = oracle_lib.refit(m, xyz, u, idx)
        assert rc == 0
        assert np.linalg.norm(alpha - m.alpha) < 1e-9 * np.linalg.norm(m.alpha)


def test_qr_and_cholesky_paths(oracle_lib, problem):
    m, xyz, u = problem
    idx = synth.row_indices(xyz.shape[1], 500, seed=47)
    A = _design_numpy(m, xyz, idx)
    x, rc = oracle_lib.lsq_qr(A, u[idx])
    assert rc == 0
    ref = np.linalg.lstsq(A, u[idx], rcond=None)[0]
    assert np.linalg.norm(x - ref) < 1e-10 * np.linalg.norm(ref)
    L, rc = oracle_lib.cholesky(A.T @ A)
    assert rc == 0
    assert np.max(np.abs(L - np.linalg.cholesky(A.T @ A))) < 1e-10 * np.max(np.abs(L))
    assert np.linalg.norm(oracle_lib.cholesky_solve(L, A.T @ u[idx]) - ref) < 1e-9 * np.linalg.norm(ref)


def test_mixing_invariance(oracle_lib, problem):
    """Algorithm 2 with a sign flip D and an orthonormal real transform F and every row
    kept leaves the LS solution unchanged (F D is orthogonal)."""
    m, xyz, u = problem
    Q = xyz.shape[1]
    idx = np.arange(Q)
    alpha, _ = oracle_lib.refit(m, xyz, u, idx)
    A = _design_numpy(m, xyz, idx)
    D = np.where(np.random.default_rng(3).random(Q) < 0.5, -1.0, 1.0)
    FA = scipy.fft.dct(D[:, None] * A, norm="ortho", axis=0)
    Fu = scipy.fft.dct(D * u, norm="ortho")
    x, rc = oracle_lib.lsq_qr(FA, Fu)
    assert rc == 0
    assert np.linalg.norm(x - alpha.ravel()) < 1e-9 * np.linalg.norm(alpha)


def test_underdetermined_is_an_error(oracle_lib, problem):
    m, xyz, u = problem
    idx = synth.row_indices(xyz.shape[1], m.R // 2, seed=48)
    _, rc = oracle_lib.refit(m, xyz, u, idx)
    assert rc < 0
