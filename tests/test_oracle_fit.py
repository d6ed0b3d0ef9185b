"""Pins of the oracle's construction steps (Algorithm 1): interpolation, ST-HOSVD,
Lasso-LARS with leave-one-out selection, and the end-to-end exact-recovery case."""
import itertools
import math
from pathlib import Path

import numpy as np
import numpy.polynomial.legendre as npl
import pytest

from oracle import fit as F


# ----------------------------------------------------------------------------- interpolation
def test_splat_samples_on_nodes_are_exact():
    I = (5, 6, 7)
    g = [F.grid_nodes(i) for i in I]
    rng = np.random.default_rng(0)
    pts = np.array([(g[0][a], g[1][b], g[2][c]) for a in range(5) for b in range(6) for c in range(7)
                    if rng.random() < 0.4]).T
    vals = rng.normal(size=pts.shape[1])
    U, filled = F.interpolate_splat(pts, vals, I)
    for s in range(pts.shape[1]):
        ia = [int(np.argmin(np.abs(g[k] - pts[k, s]))) for k in range(3)]
        assert filled[tuple(ia)]
        assert abs(U[tuple(ia)] - vals[s]) < 1e-14
    # every node sampled: the grid equals the data
    full = np.array([(g[0][a], g[1][b], g[2][c]) for a in range(5) for b in range(6) for c in range(7)]).T
    fv = rng.normal(size=full.shape[1])
    U, filled = F.interpolate_splat(full, fv, I)
    assert filled.all() and np.max(np.abs(U.reshape(-1) - fv)) < 1e-14


def test_splat_single_sample_reaches_its_cell_corners():
    U, filled = F.interpolate_splat(np.array([[0.1], [-0.2], [0.3]]), np.array([2.5]), (4, 4, 4))
    assert filled.sum() == 8 and np.allclose(U[filled], 2.5)


def test_splat_off_node_weights_by_hand():
    """Two samples inside cell (0,0,0) of a 3x3x3 node grid (nodes -1, 0, 1): sample 1 at
    fractions (1/4, 1/2, 3/4) of the cell with value 2, sample 2 at (9/10, 1/5, 2/5) with
    value -1.  Corner (a,b,c) receives the trilinear weight prod_k (f_k if bit else 1-f_k)
    from each sample and takes sum(w u) / sum(w).  The eight node values below were worked
    out by hand in exact fractions (e.g. corner (0,0,0): w1 = 3/4*1/2*1/4 = 3/32,
    w2 = 1/10*4/5*3/5 = 6/125, (2*3/32 - 6/125) / (3/32 + 6/125) = 62/63); swapped
    w / 1-w, squared fractions or nearest-node splatting all give other values."""
    t = np.array([[-0.75, -0.1], [-0.5, -0.8], [-0.25, -0.6]])
    U, filled = F.interpolate_splat(t, np.array([2.0, -1.0]), (3, 3, 3))
    expect = {(0, 0, 0): 62 / 63, (0, 0, 1): 2122 / 1253, (0, 1, 0): 78 / 47, (0, 1, 1): 2218 / 1157,
              (1, 0, 0): -1478 / 1853, (1, 0, 1): -134 / 509, (1, 1, 0): -182 / 557, (1, 1, 1): 154 / 221}
    assert filled.sum() == 8
    for ix, v in expect.items():
        assert filled[ix]
        assert abs(U[ix] - v) < 1e-14, (ix, U[ix], v)


def test_fill_from_one_node():
    U = np.zeros((5, 4, 3))
    filled = np.zeros_like(U, dtype=bool)
    U[0, 0, 0], filled[0, 0, 0] = 3.0, True
    V, sweeps = F.fill_jacobi(U, filled)
    assert np.allclose(V, 3.0)
    assert sweeps == 4 + 3 + 2          # the largest Manhattan distance from the seed node


# ----------------------------------------------------------------------------- ST-HOSVD
def _orth(rng, n, r):
    return np.linalg.qr(rng.normal(size=(n, r)))[0]


def test_st_hosvd_exact_low_rank():
    rng = np.random.default_rng(1)
    r, I = (2, 3, 4), (10, 9, 12)
    Ws = [_orth(rng, I[k], r[k]) for k in range(3)]
    X = F.tucker_reconstruct(rng.normal(size=r), Ws)
    core, Vs, _ = F.st_hosvd(X, 1e-6, (8, 8, 8))
    assert tuple(V.shape[1] for V in Vs) == r
    rec = F.tucker_reconstruct(core, Vs)
    assert np.linalg.norm(rec - X) < 1e-12 * np.linalg.norm(X)
    for V in Vs:
        assert np.max(np.abs(V.T @ V - np.eye(V.shape[1]))) < 1e-12
        assert np.all(V[np.argmax(np.abs(V), axis=0), np.arange(V.shape[1])] > 0)


def test_st_hosvd_truncation_rule_known_spectrum():
    """Superdiagonal core sigma_i with orthonormal factors: each mode Gram has eigenvalues
    sigma_i^2, so the rank is the smallest r with sum_{i>r} sigma_i^2 <= eps^2 ||X||^2 / 3."""
    rng = np.random.default_rng(2)
    sig = np.array([1.0, 0.5, 0.1, 0.03, 0.01, 0.001])
    n = sig.size
    core = np.zeros((n, n, n))
    core[np.arange(n), np.arange(n), np.arange(n)] = sig
    X = F.tucker_reconstruct(core, [_orth(rng, 12, n) for _ in range(3)])
    tot = np.sum(sig ** 2)
    for eps in (0.3, 0.05, 0.012, 0.004):
        thr = eps ** 2 * tot / 3
        expect = next(r for r in range(1, n + 1) if np.sum(sig[r:] ** 2) <= thr)
        _, Vs, _ = F.st_hosvd(X, eps, (n, n, n))
        assert tuple(V.shape[1] for V in Vs) == (expect,) * 3
        _, Vs, _ = F.st_hosvd(X, eps, (2, 2, 2))
        assert tuple(V.shape[1] for V in Vs) == (min(expect, 2),) * 3


def test_st_hosvd_fixed_rank():
    X = np.random.default_rng(3).normal(size=(6, 7, 8))
    _, Vs, _ = F.st_hosvd(X, 0.0, (3, 4, 5), fixed_rank=True)
    assert tuple(V.shape[1] for V in Vs) == (3, 4, 5)


# ----------------------------------------------------------------------------- Lasso-LARS + LOO
def test_lars_breakpoints_satisfy_lasso_kkt():
    """At every breakpoint the coefficients solve the Lasso of eq. min_P1lambda for the
    unit-norm columns: X^T (y - X b) = lam sign(b) on the support, |.| <= lam elsewhere."""
    rng = np.random.default_rng(4)
    for trial in range(5):
        X = rng.normal(size=(30, 8))
        y = rng.normal(size=30)
        Xn = X / np.linalg.norm(X, axis=0)
        bps = []
        F.lars_lasso_path(X, y, breakpoints=bps)
        assert bps
        for beta, lam in bps:
            c = Xn.T @ (y - Xn @ beta)
            on = beta != 0
            assert np.all(np.abs(c) <= lam + 1e-9)
            assert np.allclose(c[on], lam * np.sign(beta[on]), atol=1e-9)


def test_lars_path_matches_brute_force_lasso():
    """For P <= 8, solve the Lasso at each breakpoint's lam by brute force over all supports and
    signs (closed form on each), keep the KKT-feasible one, and compare the coefficients."""
    rng = np.random.default_rng(5)
    X = rng.normal(size=(20, 6))
    y = X @ np.array([1.5, 0, -2.0, 0, 0.5, 0]) + 0.1 * rng.normal(size=20)
    Xn = X / np.linalg.norm(X, axis=0)
    bps = []
    F.lars_lasso_path(X, y, breakpoints=bps)
    P = X.shape[1]
    for beta, lam in bps[:-1]:
        best = None
        for S in itertools.chain.from_iterable(itertools.combinations(range(P), k) for k in range(P + 1)):
            S = list(S)
            for sg in itertools.product((-1.0, 1.0), repeat=len(S)):
                b = np.zeros(P)
                if S:
                    XS = Xn[:, S]
                    b[S] = np.linalg.solve(XS.T @ XS, XS.T @ y - lam * np.array(sg))
                    if np.any(np.sign(b[S]) != np.array(sg)):
                        continue
                c = Xn.T @ (y - Xn @ b)
                if np.all(np.abs(c) <= lam + 1e-9):
                    obj = 0.5 * np.sum((y - Xn @ b) ** 2) + lam * np.sum(np.abs(b))
                    if best is None or obj < best[0]:
                        best = (obj, b)
        assert best is not None
        assert np.max(np.abs(best[1] - beta)) < 1e-8


def test_loo_shortcut_equals_brute_force():
    rng = np.random.default_rng(6)
    Phi = F.legendre_matrix(F.grid_nodes(25), 9)
    y = rng.normal(size=25)
    S = (0, 2, 3, 7)
    loo, _ = F.loo_error(Phi, y, S)
    errs = []
    for i in range(25):
        keep = np.arange(25) != i
        c = np.linalg.lstsq(Phi[keep][:, S], y[keep], rcond=None)[0]
        errs.append((y[i] - Phi[i, S] @ c) ** 2)
    assert abs(loo - np.mean(errs)) < 1e-12 * np.mean(errs)


def test_sparse_fit_recovers_exact_sparse_polynomial():
    Phi = F.legendre_matrix(F.grid_nodes(64), 15)
    c = np.zeros(16)
    c[[0, 3, 7, 12]] = [0.8, -1.1, 0.45, 0.2]
    rows, coef, err = F.sparse_fit(Phi, Phi @ c)
    assert list(rows) == [0, 3, 7, 12]
    assert np.max(np.abs(coef - c[rows])) < 1e-12
    assert err < 1e-20


def test_independent_columns_drops_dependent_factor_functions():
    """In-order Gram-Schmidt keeps a column only if it adds a direction: duplicates, scalings,
    sums of kept columns and zero columns go; a 1e-5 relative new direction stays."""
    rng = np.random.default_rng(4)
    a, b, c, d = (rng.normal(size=16) for _ in range(4))
    C = np.stack([a, b, 2 * a, a + b, np.zeros(16), c, -3 * c + b, a + 1e-5 * d], axis=1)
    assert F.independent_columns(C) == [0, 1, 5, 7]
    assert F.independent_columns(rng.normal(size=(16, 9))) == list(range(9))
    # more columns than the dimension: exactly the first 4 survive
    assert F.independent_columns(rng.normal(size=(4, 7))) == [0, 1, 2, 3]


# ----------------------------------------------------------------------------- end to end
def test_fit_exact_low_rank_legendre_field(oracle_lib):
    """A field that is an exact separable low-rank polynomial of degree <= p is recovered
    by Algorithm 1 + refit (grid values supplied directly, every point used in the refit)."""
    rng = np.random.default_rng(7)
    deg, r = 5, (2, 3, 2)
    facs = [rng.normal(size=(deg + 1, r[k])) for k in range(3)]
    core = rng.normal(size=r)

    def field(y):
        ws = [npl.legval(y[k], facs[k]).T for k in range(3)]   # (n, r_k)
        return np.einsum("abc,na,nb,nc->n", core, *ws)

    I = 24
    g = F.grid_nodes(I)
    G = np.stack(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1)
    grid_vals = field(G).reshape(I, I, I)
    xyz = np.random.default_rng(8).uniform(-1, 1, size=(3, 4000))
    u = field(xyz)
    params = F.FitParams(grid=(I, I, I), eps=1e-6, max_rank=(4, 4, 4), max_degree=8,
                         oversample=4.0, seed=9)
    model, rep = F.fit(xyz, u, params, grid_values=grid_vals)
    assert rep.ranks == r
    test = np.random.default_rng(10).uniform(-1, 1, size=(3, 500))
    got = oracle_lib.eval_points(model, test)
    ref = field(test)
    assert np.linalg.norm(got - ref) < 1e-11 * np.linalg.norm(ref)


def test_fit_runs_on_scattered_data(oracle_lib):
    from paper_1907_05884_gb300 import synth
    xyz = synth.points(6000, seed=11, clustered=0.0)
    u, clean = synth.field_values(xyz, synth.field_spec(12, 3), seed=13)
    params = F.FitParams(grid=(16, 16, 16), sample_frac=0.2, eps=1e-2, max_rank=(5, 5, 5),
                         max_degree=9, oversample=4.0, seed=14)
    model, rep = F.fit(xyz, u, params)
    pred = oracle_lib.eval_points(model, xyz)
    rel = np.linalg.norm(pred - clean) / np.linalg.norm(clean)
    assert rel < 0.2
    assert rep.m == min(4 * model.R, 6000)
    assert rep.compression_ratio == pytest.approx(6000 / (model.R + model.nnz()))


# ----------------------------------------------------------------------------- Table 2
def test_compression_ratio_matches_table2():
    gold = Path(__file__).parent / "golden" / "table2_compression.txt"
    rows = [l.split() for l in gold.read_text().splitlines() if l.strip() and not l.startswith("#")]
    for name, npts, orig, ratio, reduced in rows:
        npts, orig, ratio, reduced = map(float, (npts, orig, ratio, reduced))
        assert 8 * npts == pytest.approx(orig, rel=1e-12)          # 8 bytes per value
        values = reduced / 8.0
        got = F.compression_ratio(int(npts), 0, int(values))
        # printed reduced sizes are rounded to the KB: allow that rounding
        assert got == pytest.approx(ratio, rel=max(0.5e3 / reduced, 0.01))
