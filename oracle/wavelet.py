"""Oracle for the multiresolution (multiwavelet) spaces W_{s,q} of Algorithm 1's per-column
basis choice (Sec. 4.2, Fig. 3), in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Reading (the paper names no wavelet family): W_{s,q} is the space of piecewise polynomials
of degree <= q on the 2^s equal cells of [-1, 1], with the multiresolution orthonormal basis
(inner product <f, g> = 1/2 int_{-1}^{1} f g dt, the one under which the Legendre functions
phi_n = sqrt(2n+1) L_n are orthonormal):

  * the scaling functions phi_0 .. phi_q on the whole interval;
  * for levels l = 0 .. s-1 and cells c = 0 .. 2^l - 1 of level l, the wavelets
    psi_{l,c,i}(t) = 2^{l/2} psi_i(2^l (t + 1) - 2c - 1) on that cell (zero elsewhere),
    i = 0 .. q, where the mother wavelets psi_0 .. psi_q are piecewise polynomials of
    degree <= q on [-1, 0) and [0, 1], orthogonal to every polynomial of degree <= q:
    the Gram-Schmidt orthonormalisation, in the order of i, of sgn(t) phi_i(t) against
    phi_0 .. phi_q and the earlier psi (Alpert's construction spans the same spaces).

Functions are indexed 0 .. q for the scaling functions and (q+1)(2^l + c) + i for
psi_{l,c,i}; the dimension is (q+1) 2^s.

A point belongs to cell f of the finest level when it lies at or beyond the first f interior
cell boundaries lo + ((hi - lo) c) 2^-s (c = 1 .. 2^s - 1) of the model's box: cells are
closed on the left, the last one also on the right, and points outside the box extrapolate
the first or last cell's polynomial.  The cell is decided by comparing the coordinate with
those boundaries (no rounded arithmetic), so every implementation that compares exactly
agrees on it; the cell of level l is f >> (s - l).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial.legendre import leggauss


def legendre_ortho(t: np.ndarray, q: int) -> np.ndarray:
    """phi_n(t) = sqrt(2n+1) L_n(t), n = 0 .. q (orthonormal for dt/2 on [-1, 1])."""
    t = np.asarray(t, dtype=np.float64)
    L = np.empty((t.size, q + 1))
    L[:, 0] = 1.0
    if q >= 1:
        L[:, 1] = t
    for n in range(1, q):
        L[:, n + 1] = ((2 * n + 1) * t * L[:, n] - n * L[:, n - 1]) / (n + 1)
    return L * np.sqrt(2.0 * np.arange(q + 1) + 1.0)


def mother_wavelets(q: int) -> np.ndarray:
    """a[i, h, m] with psi_i(t) = sum_m a[i, h, m] phi_m(tau) on half h (h = 0: t in [-1, 0),
    tau = 2t + 1; h = 1: t in [0, 1], tau = 2t - 1).

    Coordinates in the orthonormal basis e_{h,m} = sqrt(2) phi_m(tau_h) 1_{half h} of the
    two-half piecewise space, by Gauss-Legendre quadrature (exact at these degrees)."""
    xg, wg = leggauss(q + 2)
    half = [(xg - 1.0) / 2.0, (xg + 1.0) / 2.0]          # nodes in t on each half
    Pl = legendre_ortho(xg, q)                            # phi_m(tau) at the nodes
    def coords(fvals):
        # <f, e_{h,m}> = 1/2 int_half f sqrt(2) phi_m(tau) dt = sqrt(2)/4 int f phi_m dtau
        return np.stack([math.sqrt(2.0) / 4.0 * (wg * fvals[h]) @ Pl for h in range(2)])
    P = [coords([legendre_ortho(half[h], q)[:, n] for h in range(2)]).reshape(-1) for n in range(q + 1)]
    G = [coords([np.sign(half[h]) * legendre_ortho(half[h], q)[:, i] for h in range(2)]).reshape(-1)
         for i in range(q + 1)]
    # sign(0) never occurs at interior Gauss nodes
    basis = list(P)
    out = []
    for i in range(q + 1):
        v = G[i].copy()
        for _ in range(2):                                 # twice, for rounding
            for b in basis:
                v -= (b @ v) * b
        v /= np.linalg.norm(v)
        basis.append(v)
        out.append(v.reshape(2, q + 1) * math.sqrt(2.0))  # back to phi_m(tau) coefficients
    return np.stack(out)


def cell_boundaries(lo: float, hi: float, s: int) -> np.ndarray:
    """Interior boundaries of the 2^s finest cells of [lo, hi]: lo + ((hi - lo) c) 2^-s."""
    c = np.arange(1, 2 ** s, dtype=np.float64)
    return lo + ((hi - lo) * c) * 2.0 ** -s


def finest_cells(y: np.ndarray, lo: float, hi: float, s: int) -> np.ndarray:
    """Index of the finest cell of each coordinate: the number of boundaries at or below it."""
    b = cell_boundaries(lo, hi, s)
    y = np.asarray(y, dtype=np.float64)
    return (y[:, None] >= b[None, :]).sum(axis=1).astype(np.int64)


def basis_matrix(y: np.ndarray, lo: float, hi: float, s: int, q: int) -> np.ndarray:
    """B[i, idx]: every function of W_{s,q} at the coordinates y (mapped to t by the box)."""
    y = np.asarray(y, dtype=np.float64)
    t = 2.0 * (y - lo) / (hi - lo) - 1.0
    f = finest_cells(y, lo, hi, s)
    a = mother_wavelets(q)
    B = np.zeros((y.size, (q + 1) * 2 ** s))
    B[:, :q + 1] = legendre_ortho(t, q)
    for l in range(s):
        c = f >> (s - l)
        u = 2.0 ** l * (t + 1.0) - 2.0 * c - 1.0          # coordinate inside the level-l cell
        h = (f >> (s - l - 1)) & 1                         # its half: the level-(l+1) cell
        tau = np.where(h == 1, 2.0 * u - 1.0, 2.0 * u + 1.0)
        Pl = legendre_ortho(tau, q)
        for i in range(q + 1):
            val = 2.0 ** (l / 2.0) * np.where(h == 1, Pl @ a[i, 1], Pl @ a[i, 0])
            col = (q + 1) * (2 ** l + c) + i
            B[np.arange(y.size), col] = val
    return B


def grid_basis_matrix(I: int, s: int, q: int) -> np.ndarray:
    """W_{s,q} at the node grid g_i = -1 + 2 i / (I - 1) of the interpolation (box [-1, 1])."""
    g = -1.0 + 2.0 * np.arange(I) / (I - 1)
    return basis_matrix(g, -1.0, 1.0, s, q)


# ----------------------------------------------------------------------------- models
def has_wavelets(m) -> bool:
    cw = getattr(m, "col_wavelet", None)
    return cw is not None and any(np.any(np.asarray(c, dtype=bool)) for c in cw)


def factor_values(m, k: int, y: np.ndarray) -> np.ndarray:
    """w^(k)_j(y) for every column j of mode k (Sec. 2, eq. sparse), Legendre columns in
    P_p and wavelet columns in W_{s,q} (indices as above)."""
    y = np.asarray(y, dtype=np.float64)
    lo, hi = float(m.lo[k]), float(m.hi[k])
    t = 2.0 * (y - lo) / (hi - lo) - 1.0
    Pl = legendre_ortho(t, int(m.p[k]))
    cw = np.zeros(m.r[k], dtype=bool) if getattr(m, "col_wavelet", None) is None else \
        np.asarray(m.col_wavelet[k], dtype=bool)
    Bw = basis_matrix(y, lo, hi, int(m.wav[0]), int(m.wav[1])) if cw.any() else None
    U = np.zeros((y.size, m.r[k]))
    for j in range(m.r[k]):
        s0, e0 = int(m.colptr[k][j]), int(m.colptr[k][j + 1])
        rows = np.asarray(m.rowidx[k][s0:e0], dtype=np.int64)
        vals = np.asarray(m.val[k][s0:e0], dtype=np.float64)
        U[:, j] = (Bw if cw[j] else Pl)[:, rows] @ vals
    return U


def eval_points(m, xyz: np.ndarray) -> np.ndarray:
    """The model at points xyz (3, n): sum_ijk alpha_ijk w1_i w2_j w3_k (eq. func_tuck)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    U = [factor_values(m, k, xyz[k]) for k in range(3)]
    return np.einsum("ijk,ni,nj,nk->n", np.asarray(m.alpha, dtype=np.float64).reshape(m.r), *U)


def design_matrix(m, xyz: np.ndarray, idx) -> np.ndarray:
    """Rows q of idx of the measurement matrix of eq. rand_core: u1(y_q) (x) u2 (x) u3."""
    xyz = np.asarray(xyz, dtype=np.float64)[:, np.asarray(idx, dtype=np.int64)]
    U = [factor_values(m, k, xyz[k]) for k in range(3)]
    return np.einsum("ni,nj,nk->nijk", *U).reshape(xyz.shape[1], -1)


def refit(m, xyz: np.ndarray, u: np.ndarray, idx) -> np.ndarray:
    """The least-squares core over the rows idx (eq. rand_core), by the normal equations and
    a Cholesky factorisation (numpy), Householder QR (numpy lstsq) if that fails."""
    A = design_matrix(m, xyz, idx)
    b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
    G = A.T @ A
    try:
        L = np.linalg.cholesky(G)
        return np.linalg.solve(L.T, np.linalg.solve(L, A.T @ b)).reshape(m.r)
    except np.linalg.LinAlgError:
        return np.linalg.lstsq(A, b, rcond=None)[0].reshape(m.r)
