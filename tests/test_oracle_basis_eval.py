"""Pins of the oracle's Legendre basis and evaluation (Sec. 2, eq. func_tuck, eq. sparse)
against closed forms and numpy's independent Legendre routines."""
import math

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

from paper_1907_05884_gb300 import synth


def test_legendre_endpoints_and_zero(oracle_lib):
    p = 63
    assert np.allclose(oracle_lib.legendre(1.0, p), 1.0, rtol=0, atol=1e-13)
    assert np.allclose(oracle_lib.legendre(-1.0, p), (-1.0) ** np.arange(p + 1), rtol=0, atol=1e-13)
    L0 = oracle_lib.legendre(0.0, p)
    for n in range(p + 1):
        if n % 2:
            assert abs(L0[n]) < 1e-15
        else:
            k = n // 2
            exact = (-1) ** k * math.comb(2 * k, k) / 4 ** k   # (2k)!/(4^k (k!)^2)
            assert abs(L0[n] - exact) < 1e-14


def test_legendre_matches_numpy_legval(oracle_lib):
    rng = np.random.default_rng(0)
    p = 63
    for t in rng.uniform(-1, 1, size=25):
        L = oracle_lib.legendre(t, p)
        ref = np.array([npl.legval(t, np.eye(p + 1)[n]) for n in range(p + 1)])
        assert np.max(np.abs(L - ref)) < 1e-12


def test_orthonormal_by_gauss_legendre(oracle_lib):
    """phi_n = sqrt(2n+1) L_n is orthonormal for dt/2 on [-1,1] (the orthonormal basis of Sec. 2)."""
    from oracle.fit import legendre_matrix
    p = 40
    x, w = npl.leggauss(64)
    Phi = legendre_matrix(x, p)
    M = (Phi * (w / 2.0)[:, None]).T @ Phi
    assert np.max(np.abs(M - np.eye(p + 1))) < 1e-12
    L = np.stack([oracle_lib.legendre(t, p) for t in x])
    assert np.max(np.abs(L * np.sqrt(2 * np.arange(p + 1) + 1) - Phi)) < 1e-12


def _w_numpy(model, k, t):
    """w^(k)_j(t) through numpy legval on the orthonormal coefficients."""
    W = model.dense(k) * np.sqrt(2 * np.arange(model.p[k] + 1) + 1)[:, None]
    return np.stack([npl.legval(t, W[:, j]) for j in range(model.r[k])])


def test_rank_one_core_is_product_of_series(oracle_lib):
    m = synth.random_model((1, 1, 1), (7, 11, 5), seed=3, density=0.7)
    xyz = synth.points(300, seed=5)
    f = oracle_lib.eval_points(m, xyz)
    ref = m.alpha[0, 0, 0] * _w_numpy(m, 0, xyz[0])[0] * _w_numpy(m, 1, xyz[1])[0] * _w_numpy(m, 2, xyz[2])[0]
    assert np.max(np.abs(f - ref)) < 1e-12 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("r,p", [((3, 4, 2), (6, 5, 7)), ((5, 5, 5), (9, 9, 9))])
def test_eval_equals_full_tensor_product_expansion(oracle_lib, r, p):
    """The Tucker form equals the full expansion of Sec. 2 with beta = alpha x1 W1 x2 W2 x3 W3,
    evaluated by numpy's legval3d."""
    m = synth.random_model(r, p, seed=11, density=0.5)
    xyz = synth.points(200, seed=12)
    f = oracle_lib.eval_points(m, xyz)
    beta = np.einsum("abc,ia,jb,kc->ijk", m.alpha, m.dense(0), m.dense(1), m.dense(2))
    s = [np.sqrt(2 * np.arange(pk + 1) + 1) for pk in m.p]
    coef = beta * s[0][:, None, None] * s[1][None, :, None] * s[2][None, None, :]
    ref = npl.legval3d(xyz[0], xyz[1], xyz[2], coef)
    assert np.max(np.abs(f - ref)) < 1e-11 * max(1.0, np.max(np.abs(ref)))


def test_eval_affine_box_map(oracle_lib):
    lo, hi = np.array([2.0, -5.0, 0.5]), np.array([4.0, 3.0, 0.75])
    m1 = synth.random_model((3, 2, 4), (5, 6, 4), seed=21, lo=lo, hi=hi)
    m0 = synth.random_model((3, 2, 4), (5, 6, 4), seed=21)
    t = synth.points(100, seed=22)
    y = lo[:, None] + (t + 1.0) / 2.0 * (hi - lo)[:, None]
    assert np.max(np.abs(oracle_lib.eval_points(m1, y) - oracle_lib.eval_points(m0, t))) < 1e-12


def test_eval_threads_bitwise(oracle_lib):
    m = synth.random_model((4, 4, 4), (8, 8, 8), seed=31)
    xyz = synth.points(1000, seed=32)
    a = oracle_lib.eval_points(m, xyz, nthreads=1)
    b = oracle_lib.eval_points(m, xyz, nthreads=4)
    assert np.array_equal(a, b)
