"""Pins of the multiwavelet spaces W_{s,q} (oracle/wavelet.py) and of the fit's choice
between P_p and W_{s,q} per column (Sec. 4.2, Algorithm 1's basis choice, Fig. 3)."""
import numpy as np
import pytest
from numpy.polynomial.legendre import leggauss

from oracle import fit as F
from oracle import wavelet as W


def _cell_quadrature(s, deg):
    """Gauss-Legendre nodes and weights (for dt/2) on every finest cell of [-1, 1]."""
    xg, wg = leggauss(deg // 2 + 2)
    nc = 2 ** s
    t = np.concatenate([-1.0 + (2.0 * c + 1.0 + xg) / nc for c in range(nc)])
    w = np.concatenate([wg / nc / 2.0 for _ in range(nc)])
    return t, w


@pytest.mark.parametrize("s,q", [(0, 3), (1, 0), (2, 1), (3, 5), (4, 2)])
def test_basis_is_orthonormal(s, q):
    """<B_a, B_b> = delta_ab for every pair of functions of W_{s,q} (exact quadrature on the
    finest cells, where every function is one polynomial)."""
    t, w = _cell_quadrature(s, 2 * q)
    B = W.basis_matrix(t, -1.0, 1.0, s, q)
    assert B.shape[1] == (q + 1) * 2 ** s
    assert np.max(np.abs(B.T @ (w[:, None] * B) - np.eye(B.shape[1]))) < 1e-12


def test_haar_case():
    """q = 0: the Haar system, written out from its textbook definition: 1, and for level l,
    cell c the function -2^{l/2} on the left half of the cell, +2^{l/2} on the right half."""
    s = 3
    y = np.linspace(-1, 1, 1001)
    B = W.basis_matrix(y, -1.0, 1.0, s, 0)
    H = np.zeros_like(B)
    H[:, 0] = 1.0
    for l in range(s):
        for c in range(2 ** l):
            a, b = -1.0 + 2.0 * c / 2 ** l, -1.0 + 2.0 * (c + 1) / 2 ** l
            mid = 0.5 * (a + b)
            last = c == 2 ** l - 1
            left = (y >= a) & (y < mid)
            right = (y >= mid) & ((y < b) | (last & (y <= b)))
            H[:, 2 ** l + c] = 2.0 ** (l / 2) * (right.astype(float) - left.astype(float))
    assert np.max(np.abs(B - H)) < 1e-14


@pytest.mark.parametrize("q", [0, 2, 5])
def test_mother_wavelets_vanishing_moments(q):
    """Every mother wavelet is orthogonal to t^m, m = 0 .. q (its defining property)."""
    t, w = _cell_quadrature(1, 2 * q + 2)
    B = W.basis_matrix(t, -1.0, 1.0, 1, q)
    for i in range(q + 1):
        psi = B[:, q + 1 + i]
        for mm in range(q + 1):
            assert abs(np.sum(w * psi * t ** mm)) < 1e-13
        assert abs(np.sum(w * psi * t ** (q + 1))) > 0 or i != q   # not orthogonal to everything


def test_cells_by_boundary_comparison():
    s = 3
    b = W.cell_boundaries(0.0, 4.0, s)
    assert np.array_equal(b, np.arange(1, 8) * 0.5)
    y = np.array([-1.0, 0.0, 0.49, 0.5, 3.5, 3.999, 4.0, 5.0])
    assert W.finest_cells(y, 0.0, 4.0, s).tolist() == [0, 0, 0, 1, 7, 7, 7, 7]


def test_piecewise_polynomials_recovered():
    """W_{s,q} is every piecewise polynomial of degree <= q on the 2^s cells: a random one,
    sampled at q + 2 points per cell, is fitted by least squares and reproduced at other
    points of each cell to 1e-12."""
    rng = np.random.default_rng(0)
    s, q = 3, 4
    nc = 2 ** s
    coef = rng.normal(size=(nc, q + 1))

    def f(t):
        c = np.minimum(((t + 1.0) * nc / 2.0).astype(int), nc - 1)
        x = t - (-1.0 + (2.0 * c + 1.0) / nc)
        return sum(coef[c, d] * x ** d for d in range(q + 1))

    t_fit = np.concatenate([-1.0 + (2.0 * c + 1.0 + np.linspace(-0.9, 0.9, q + 2)) / nc for c in range(nc)])
    B = W.basis_matrix(t_fit, -1.0, 1.0, s, q)
    x = np.linalg.lstsq(B, f(t_fit), rcond=None)[0]
    t_chk = np.concatenate([-1.0 + (2.0 * c + 1.0 + np.linspace(-0.97, 0.97, 11)) / nc for c in range(nc)])
    got = W.basis_matrix(t_chk, -1.0, 1.0, s, q) @ x
    assert np.max(np.abs(got - f(t_chk))) < 1e-11 * np.max(np.abs(f(t_chk)))


def test_sparse_wavelet_expansion_recovered_by_lars_loo():
    """A column that is an exact sparse combination of three multiwavelets is recovered by the
    Lasso-LARS / leave-one-out fit in W_{s,q} (support and coefficients)."""
    s, q, I = 3, 2, 64
    Phi = W.grid_basis_matrix(I, s, q)
    rows = np.array([1, 9, 20])
    vals = np.array([0.8, -0.5, 0.3])
    y = Phi[:, rows] @ vals
    got_rows, got_vals, loo = F.sparse_fit(Phi, y)
    assert got_rows.tolist() == rows.tolist()
    assert np.max(np.abs(got_vals - vals)) < 1e-10
    assert loo < 1e-20


def test_basis_choice_per_column():
    """The fit keeps W_{s,q} for a step-like column (exact there, poorly fitted by
    polynomials) and P_p for a polynomial column of degree above q (exact in P_p only)."""
    I, p, s, q = 48, 9, 3, 2
    g = F.grid_nodes(I)
    step = np.where(g < -0.25, -1.0, 1.0) + np.where(g >= 0.5, 0.5, 0.0)
    poly = F.legendre_matrix(g, p) @ np.r_[0.3, -0.2, 0.5, 0.1, -0.4, 0.2, 0.1, -0.3, 0.2, 0.15]
    Phi = F.legendre_matrix(g, p)
    Phw = W.grid_basis_matrix(I, s, q)
    for y, want_wavelet in ((step, True), (poly, False)):
        leg, wav = F.sparse_fit(Phi, y), F.sparse_fit(Phw, y)
        chose = wav[2] < leg[2] - 1e-12 * float(np.mean(y * y))
        assert chose == want_wavelet, (leg[2], wav[2])


def test_rank_one_wavelet_model_evaluation():
    """A rank-one model whose three factor functions are single Haar functions: the oracle's
    evaluation is the product of the three textbook values times the core entry."""
    from paper_1907_05884_gb300 import synth
    cp = [np.array([0, 1], np.int32)] * 3
    rows = [np.array([1], np.int32), np.array([2], np.int32), np.array([5], np.int32)]
    vals = [np.array([1.0]), np.array([1.0]), np.array([1.0])]
    m = synth.Model((1, 1, 1), (0, 0, 0), cp, rows, vals, np.array([[[2.0]]]), wav=(3, 0),
                    col_wavelet=[np.array([True])] * 3)
    y = np.array([[-0.5, 0.5, 0.1], [-0.75, -0.25, 0.6], [0.3, 0.9, -0.9]])
    # index 1: psi_{0,0} = sgn; index 2: psi_{1,0} (cell [-1, 0)); index 5: psi_{2,1} (cell [-0.5, 0))
    def haar(l, c, t):
        a, b = -1.0 + 2.0 * c / 2 ** l, -1.0 + 2.0 * (c + 1) / 2 ** l
        mid = 0.5 * (a + b)
        return 2.0 ** (l / 2) * (((t >= mid) & (t < b)).astype(float) - ((t >= a) & (t < mid)).astype(float))
    want = 2.0 * haar(0, 0, y[0]) * haar(1, 0, y[1]) * haar(2, 1, y[2])
    import oracle
    assert np.allclose(oracle.eval_points(m, y), want, rtol=0, atol=1e-15)


def test_fit_recovers_piecewise_low_rank_field():
    """Algorithm 1 + the refit on a field that is an exact rank-(2,2,2) Tucker tensor of
    piecewise-linear factors on 4 cells (in W_{2,1}, not in any P_p): the columns choose the
    multiwavelet space and the fitted model reproduces the field at scattered points."""
    import oracle
    rng = np.random.default_rng(3)
    s, q, I = 2, 1, 32

    def pw(c4, t):
        c = np.minimum(((t + 1.0) * 2.0).astype(int), 3)
        return c4[c, 0] + c4[c, 1] * t
    facs = [[rng.normal(size=(4, 2)) for _ in range(2)] for _ in range(3)]
    core = rng.normal(size=(2, 2, 2))
    g = F.grid_nodes(I)
    Us = [np.stack([pw(facs[k][j], g) for j in range(2)], axis=1) for k in range(3)]
    grid = np.einsum("abc,ia,jb,kc->ijk", core, *Us)
    xyz = rng.uniform(-1, 1, size=(3, 3000))
    u = np.einsum("abc,na,nb,nc->n", core,
                  *[np.stack([pw(facs[k][j], xyz[k]) for j in range(2)], axis=1) for k in range(3)])
    m, rep = F.fit(xyz, u, F.FitParams(grid=(I, I, I), eps=1e-6, max_rank=(4, 4, 4), max_degree=3,
                                       oversample=8.0, wavelet=(s, q)), grid_values=grid)
    assert rep.ranks == (2, 2, 2)
    assert all(all(c) for c in rep.chose_wavelet)
    pred = oracle.eval_points(m, xyz)
    assert np.linalg.norm(pred - u) < 1e-9 * np.linalg.norm(u)
