"""Pins of the order-4 oracle (oracle/order4.py; eq. func_tuck with d = 4, eq. sparse,
eq. rand_core) against numpy's independent Legendre series, the pinned order-3 oracle,
brute-force sums over the core and exact recovery."""
import itertools

import numpy as np
import numpy.polynomial.legendre as npl

from oracle import order4 as O4
from paper_1907_05884_gb300 import synth


def _series(rows, vals, t):
    """sum_n c_n sqrt(2n+1) L_n(t) through numpy's Legendre series (independent of the oracle)."""
    c = np.zeros(int(max(rows)) + 1)
    for n, v in zip(rows, vals):
        c[n] = v * np.sqrt(2 * n + 1)
    return npl.legval(t, c)


def test_rank_one_model_is_a_product_of_legendre_series():
    m = synth.random_model4((1, 1, 1, 1), (5, 9, 3, 7), seed=3, density=0.7,
                            lo=[-2.0, 0.0, -1.0, 1.0], hi=[2.0, 3.0, 0.5, 4.0])
    m = m.with_alpha(np.array([[[[-1.75]]]]))
    x = np.stack([np.random.default_rng(k).uniform(m.lo[k], m.hi[k], 50) for k in range(4)])
    got = O4.eval_points(m, x)
    ref = -1.75 * np.ones(50)
    for k in range(4):
        t = 2 * (x[k] - m.lo[k]) / (m.hi[k] - m.lo[k]) - 1
        ref *= _series(m.rowidx[k], m.val[k], t)
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_constant_fourth_factor_reduces_to_the_order3_oracle(oracle_lib):
    """A fourth mode of rank 1 whose function is phi_0 = 1 leaves the order-3 model of the
    first three modes (evaluated by the C oracle)."""
    m3 = synth.random_model((5, 4, 6), (9, 7, 11), seed=11, density=0.6)
    m4 = synth.Model4(r=(5, 4, 6, 1), p=(9, 7, 11, 4), colptr=list(m3.colptr) + [np.array([0, 1], np.int32)],
                      rowidx=list(m3.rowidx) + [np.array([0], np.int32)], val=list(m3.val) + [np.array([1.0])],
                      alpha=np.asarray(m3.alpha).reshape(5, 4, 6, 1))
    x = synth.points4(700, seed=12)
    got = O4.eval_points(m4, x)
    ref = oracle_lib.eval_points(m3, np.ascontiguousarray(x[:3]))
    assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    # and its design matrix is the order-3 one
    idx = np.arange(0, 700, 7)
    A4 = O4.design_matrix(m4, x, idx)
    A3 = oracle_lib.design_matrix(m3, np.ascontiguousarray(x[:3]), idx)
    assert np.max(np.abs(A4 - A3)) <= 1e-12 * np.max(np.abs(A3))


def test_brute_force_sum_over_the_core():
    m = synth.random_model4((2, 3, 2, 3), (4, 5, 3, 6), seed=21, density=0.8)
    x = synth.points4(9, seed=22)
    got = O4.eval_points(m, x)
    for q in range(9):
        w = []
        for k in range(4):
            t = x[k, q]
            w.append([_series(m.rowidx[k][m.colptr[k][j]:m.colptr[k][j + 1]],
                              m.val[k][m.colptr[k][j]:m.colptr[k][j + 1]], t) for j in range(m.r[k])])
        s = 0.0
        for i, j, k, l in itertools.product(*[range(v) for v in m.r]):
            s += m.alpha[i, j, k, l] * w[0][i] * w[1][j] * w[2][k] * w[3][l]
        assert abs(got[q] - s) <= 1e-12 * max(1.0, abs(s)), q
    # the design matrix row is the Kronecker product in C order of the core
    A = O4.design_matrix(m, x, np.arange(9))
    assert np.allclose(A @ m.alpha.reshape(-1), got, rtol=0, atol=1e-12)


def test_mode_permutation_consistency():
    """Reordering the modes (factors, coordinates and core axes together) keeps every value."""
    m = synth.random_model4((3, 2, 4, 2), (6, 4, 7, 5), seed=31, lo=[-1, -2, 0, -1], hi=[1, 2, 1, 3])
    x = synth.points4(300, seed=32)
    perm = (2, 0, 3, 1)
    mp = synth.Model4(r=tuple(m.r[k] for k in perm), p=tuple(m.p[k] for k in perm),
                      colptr=[m.colptr[k] for k in perm], rowidx=[m.rowidx[k] for k in perm],
                      val=[m.val[k] for k in perm], alpha=np.transpose(m.alpha, perm),
                      lo=np.asarray(m.lo)[list(perm)], hi=np.asarray(m.hi)[list(perm)])
    a = O4.eval_points(m, x)
    b = O4.eval_points(mp, x[list(perm)])
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))


def test_refit_recovers_an_exact_core():
    m = synth.random_model4((3, 4, 2, 3), (5, 6, 4, 5), seed=41, orthonormal=True)
    x = synth.points4(3000, seed=42)
    u = O4.eval_points(m, x)
    idx = np.sort(np.random.default_rng(43).choice(3000, size=4 * m.R, replace=False))
    start = m.with_alpha(np.zeros(m.r))
    got = O4.refit(start, x, u, idx)
    assert np.max(np.abs(got - m.alpha)) <= 1e-9 * np.max(np.abs(m.alpha))
    assert O4.normal_residual(start, x, u, idx, got) <= 1e-12


def test_refit_least_squares_property_on_noisy_data():
    """For noisy data the refitted core makes the residual orthogonal to every column."""
    m = synth.random_model4((2, 3, 3, 2), (4, 5, 5, 4), seed=51, orthonormal=True)
    x = synth.points4(2000, seed=52)
    u, _ = synth.field_values4(x, synth.field_spec(53, 3), seed=54)
    idx = np.arange(0, 2000, 3)
    a = O4.refit(m, x, u, idx)
    A = O4.design_matrix(m, x, idx)
    r = u[idx] - A @ a.reshape(-1)
    assert np.max(np.abs(A.T @ r)) <= 1e-10 * np.linalg.norm(A.T @ u[idx])
    # and any perturbation of the core increases the residual
    d = np.random.default_rng(55).normal(size=a.size) * 1e-3
    assert np.linalg.norm(u[idx] - A @ (a.reshape(-1) + d)) > np.linalg.norm(r)
