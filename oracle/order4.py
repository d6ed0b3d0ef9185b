"""Oracle for order-4 functional sparse Tucker models (eq. func_tuck with d = 4, the SP4D case
of Sec. 6 and Table 1: three space axes and time), in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The model is f(y) = sum_{j1 j2 j3 j4} alpha_{j1 j2 j3 j4} w1_{j1}(y1) w2_{j2}(y2) w3_{j3}(y3)
w4_{j4}(y4), each factor function a sparse combination of the orthonormal Legendre functions
phi_n = sqrt(2n+1) L_n of the coordinate mapped to [-1, 1] by the model's box (eq. sparse).
The core refit is the least-squares problem of eq. rand_core over the sampled rows, whose
measurement-matrix row is the Kronecker product w1 (x) w2 (x) w3 (x) w4 (column index
((j1 r2 + j2) r3 + j3) r4 + j4, the C order of the core), solved here through the normal
equations and a Cholesky factorisation (numpy), Householder QR (numpy lstsq) when that fails.

Pinned by ``tests/test_oracle_order4.py``: a rank-one model against numpy's Legendre series,
the reduction to the order-3 oracle (``fst_oracle.c``) when the fourth factor is constant,
brute-force loops over the core on tiny models, consistency under a permutation of the modes,
and exact recovery of the core from exact model values.
"""
from __future__ import annotations

import numpy as np


def legendre_ortho(t: np.ndarray, p: int) -> np.ndarray:
    """phi_n(t) = sqrt(2n+1) L_n(t), n = 0 .. p, by the three-term recurrence (columns)."""
    t = np.asarray(t, dtype=np.float64)
    L = np.empty((t.size, p + 1))
    L[:, 0] = 1.0
    if p >= 1:
        L[:, 1] = t
    for n in range(1, p):
        L[:, n + 1] = ((2 * n + 1) * t * L[:, n] - n * L[:, n - 1]) / (n + 1)
    return L * np.sqrt(2.0 * np.arange(p + 1) + 1.0)


def factor_values(m, k: int, y: np.ndarray) -> np.ndarray:
    """w^(k)_j(y) for every column j of mode k: (n, r_k)."""
    y = np.asarray(y, dtype=np.float64)
    lo, hi = float(m.lo[k]), float(m.hi[k])
    t = 2.0 * (y - lo) / (hi - lo) - 1.0
    P = legendre_ortho(t, int(m.p[k]))
    U = np.zeros((y.size, m.r[k]))
    for j in range(m.r[k]):
        s, e = int(m.colptr[k][j]), int(m.colptr[k][j + 1])
        rows = np.asarray(m.rowidx[k][s:e], dtype=np.int64)
        U[:, j] = P[:, rows] @ np.asarray(m.val[k][s:e], dtype=np.float64)
    return U


def eval_points(m, x: np.ndarray) -> np.ndarray:
    """The model at points x (4, n): the four-way contraction of eq. func_tuck."""
    x = np.asarray(x, dtype=np.float64)
    U = [factor_values(m, k, x[k]) for k in range(4)]
    return np.einsum("ijkl,ni,nj,nk,nl->n", np.asarray(m.alpha, dtype=np.float64).reshape(m.r), *U,
                     optimize=True)


def design_matrix(m, x: np.ndarray, idx) -> np.ndarray:
    """Rows idx of the measurement matrix of eq. rand_core: w1 (x) w2 (x) w3 (x) w4, (m, R)."""
    x = np.asarray(x, dtype=np.float64)[:, np.asarray(idx, dtype=np.int64)]
    U = [factor_values(m, k, x[k]) for k in range(4)]
    return np.einsum("ni,nj,nk,nl->nijkl", *U, optimize=True).reshape(x.shape[1], -1)


def normal_equations(m, x, u, idx):
    """G = A^T A and h = A^T b over the rows idx (b = u at those rows)."""
    A = design_matrix(m, x, idx)
    b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
    return A.T @ A, A.T @ b


def refit(m, x, u, idx) -> np.ndarray:
    """The least-squares core over the rows idx (eq. rand_core), shaped like the core."""
    A = design_matrix(m, x, idx)
    b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
    G = A.T @ A
    try:
        L = np.linalg.cholesky(G)
        a = np.linalg.solve(L.T, np.linalg.solve(L, A.T @ b))
    except np.linalg.LinAlgError:
        a = np.linalg.lstsq(A, b, rcond=None)[0]
    return a.reshape(m.r)


def normal_residual(m, x, u, idx, alpha) -> float:
    """|| A^T (A alpha - b) || / || A^T b || over the rows idx."""
    A = design_matrix(m, x, idx)
    b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
    a = np.asarray(alpha, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(A.T @ (A @ a - b)) / np.linalg.norm(A.T @ b))
