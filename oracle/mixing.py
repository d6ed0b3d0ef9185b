"""Algorithm 2 of Sec. 5 with its mixing step, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (the same rule as the rest of ``oracle/``: only the tests, the
smoke check and the benchmark's CPU legs may import it).

Algorithm 2 solves the least-squares problem of eq. rand_core on the rows S F D W of the
design matrix W (the Khatri-Rao rows of all Q points), with D a diagonal of random signs, F
a fast orthonormal mixing transform acting along the Q rows and S a uniform sampling of m
rows.  The paper does not fix F beyond "fast mixing" (the DCT-like transforms of the
randomized-LS literature it cites); this oracle takes the normalised Walsh-Hadamard
transform over the rows padded with zeros to N = 2^ceil(log2 Q) (a real orthonormal
transform with a fast algorithm), the signs D_q = -1 when the top bit of the splitmix64 key
of row q under the sign seed is set (+1 otherwise), and S = the uniform sampler of
``oracle.sample`` over the N mixed rows under the row seed.

Pins (``tests/test_oracle_mixing.py``): the transform equals ``scipy.linalg.hadamard`` / sqrt(N)
on small N and is an involution; the signs follow the published splitmix64 definition and
are balanced; with every mixed row kept the solution equals the unmixed full least squares
(F D is orthogonal); noise-free data are recovered exactly from m >= R mixed rows.
"""
from __future__ import annotations

import numpy as np

from . import design_matrix, key, lsq_qr, sample


def padded_rows(Q: int) -> int:
    """N = 2^ceil(log2 Q), at least 1."""
    N = 1
    while N < Q:
        N *= 2
    return N


def signs(seed: int, N: int) -> np.ndarray:
    """D_q = -1 if bit 63 of splitmix64 key(seed, q) is set, else +1, q < N."""
    return np.array([-1.0 if (key(seed, q) >> 63) & 1 else 1.0 for q in range(N)])


def fwht(X: np.ndarray) -> np.ndarray:
    """Normalised Walsh-Hadamard transform along axis 0 (length a power of 2): H_N X / sqrt(N)
    with H_1 = [1], H_2n = [[H_n, H_n], [H_n, -H_n]]; butterflies (a, b) -> (a + b, a - b) / sqrt(2)
    over strides h = 1, 2, 4, ..."""
    Y = np.array(X, dtype=np.float64, copy=True)
    N = Y.shape[0]
    assert N & (N - 1) == 0, "length must be a power of 2"
    s = 1.0 / np.sqrt(2.0)
    h = 1
    while h < N:
        Y = Y.reshape((N // (2 * h), 2, h) + Y.shape[1:])
        a = Y[:, 0].copy()
        b = Y[:, 1].copy()
        Y[:, 0] = (a + b) * s
        Y[:, 1] = (a - b) * s
        Y = Y.reshape((N,) + Y.shape[3:])
        h *= 2
    return Y


def mixed_system(model, xyz: np.ndarray, u: np.ndarray, seed_signs: int):
    """(F D W, F D u) over the N padded rows (W: design matrix of all Q points)."""
    Q = xyz.shape[1]
    N = padded_rows(Q)
    W = design_matrix(model, xyz, np.arange(Q, dtype=np.int64))
    WB = np.zeros((N, W.shape[1] + 1))
    WB[:Q, :-1] = W
    WB[:Q, -1] = u
    WB *= signs(seed_signs, N)[:, None]
    WB = fwht(WB)
    return WB[:, :-1], WB[:, -1]


def refit_mixed(model, xyz: np.ndarray, u: np.ndarray, m: int, seed_signs: int, seed_rows: int):
    """Algorithm 2: the core minimising || S F D W alpha - S F D u ||, S the m rows of
    ``sample(seed_rows, N, m)``; solved by Householder QR.  Returns (alpha (r1, r2, r3), rc)."""
    A, b = mixed_system(model, xyz, u, seed_signs)
    idx = sample(seed_rows, A.shape[0], m)
    x, rc = lsq_qr(A[idx], b[idx])
    r = model.r if hasattr(model, "r") else model["r"]
    return x.reshape(tuple(r)), rc
