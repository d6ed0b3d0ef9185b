"""Oracle for the construction of a functional sparse Tucker model (Algorithm 1)
plus the core refit of Algorithm 2, in plain FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Steps, in the paper's order:
  1. interpolate a fraction of the data onto an equispaced grid (Sec. 4.1);
  2. ST-HOSVD of the grid tensor at precision eps (Sec. 4.1, Algorithm 1);
  3. for every column W^(k)_{:,j}, a sparse Legendre expansion by Lasso-LARS
     with the leave-one-out error choosing the support (Sec. 3, Sec. 4.2);
  4. re-estimate the core by least squares on sampled original rows
     (Sec. 5, eq. rand_core, Algorithm 2) -- done by the C oracle.

Readings where the paper is silent (stated again in the design notes):
  * the subset is uniform without replacement (random sort keys, as the C sampler);
  * the grid is a node grid with both ends of [-1,1] included;
  * "linear interpolation" of scattered points is a trilinear splat: each sample
    adds its value to the 8 nodes of its cell with trilinear weights, a node takes
    the weighted mean; nodes with no weight are filled by Jacobi sweeps that give
    an empty node the mean of its filled 6-neighbours from the previous sweep;
  * ST-HOSVD processes modes 1,2,3 with the mode Gram matrix and keeps the smallest
    rank r_k >= 1 whose discarded eigenvalues sum to at most eps^2 ||U||_F^2 / d,
    capped at max_rank; each eigenvector's largest-magnitude entry is made positive;
  * the stored coefficients are the least-squares fit on the chosen support
    (hybrid LARS), the support being the path breakpoint with the least LOO error;
  * with a multiwavelet space W_{s,q} given (Sec. 4.2, Algorithm 1's basis choice, Fig. 3),
    every column is fitted in P_p and in W_{s,q} and keeps the fit with the smaller LOO
    error (within 1e-12 mean(y^2) of each other, P_p); wavelet.py defines the space;
  * a fitted factor function that lies in the span of the earlier ones of its mode
    (relative residual norm <= 1e-6 after in-order Gram-Schmidt on the orthonormal
    Legendre coefficients) is dropped: the refit's least squares (Sec. 5) needs
    linearly independent Khatri-Rao columns, and noise columns of the ST-HOSVD often
    collapse to the same low-degree fit.  The refit re-estimates the whole core.
Parity of the whole fit against the GPU fit is unpinned pointwise (support, rank
and sign choices are discrete); it is compared by reconstruction error.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import refit as _c_refit, sample as _c_sample
from . import wavelet as _wav

REFIT_SEED_OFFSET = 0x632BE59BD9B4E019


# ----------------------------------------------------------------------------- basis
def legendre_matrix(t: np.ndarray, p: int) -> np.ndarray:
    """Phi[i, n] = sqrt(2n+1) L_n(t_i), n = 0..p (orthonormal for dt/2, Sec. 2)."""
    t = np.asarray(t, dtype=np.float64)
    L = np.empty((t.size, p + 1))
    L[:, 0] = 1.0
    if p >= 1:
        L[:, 1] = t
    for n in range(1, p):
        L[:, n + 1] = ((2 * n + 1) * t * L[:, n] - n * L[:, n - 1]) / (n + 1)
    return L * np.sqrt(2.0 * np.arange(p + 1) + 1.0)


def grid_nodes(I: int) -> np.ndarray:
    return -1.0 + 2.0 * np.arange(I) / (I - 1)


# ----------------------------------------------------------------------------- step 1
def interpolate_splat(t: np.ndarray, u: np.ndarray, grid):
    """Trilinear splat of samples at normalised coordinates t (3, n) in [-1,1]
    onto the node grid; returns (U, filled) with U the weighted node means."""
    grid = tuple(int(g) for g in grid)
    num = np.zeros(grid)
    den = np.zeros(grid)
    cells, fracs = [], []
    for k in range(3):
        h = 2.0 / (grid[k] - 1)
        s = (np.asarray(t[k], dtype=np.float64) + 1.0) / h
        c = np.clip(np.floor(s).astype(np.int64), 0, grid[k] - 2)
        cells.append(c)
        fracs.append(s - c)
    for a in (0, 1):
        wa = fracs[0] if a else 1.0 - fracs[0]
        for b in (0, 1):
            wb = fracs[1] if b else 1.0 - fracs[1]
            for c in (0, 1):
                wc = fracs[2] if c else 1.0 - fracs[2]
                w = wa * wb * wc
                ix = (cells[0] + a, cells[1] + b, cells[2] + c)
                np.add.at(num, ix, w * u)
                np.add.at(den, ix, w)
    filled = den > 0.0
    U = np.zeros(grid)
    U[filled] = num[filled] / den[filled]
    return U, filled


def fill_jacobi(U: np.ndarray, filled: np.ndarray, max_sweeps: int = 100000):
    """Fill empty nodes: each sweep gives every empty node with a filled
    6-neighbour the mean of those neighbours (values of the previous sweep)."""
    U = U.copy()
    filled = filled.copy()
    if not filled.any():
        raise ValueError("no grid node received a sample")
    sweeps = 0
    while not filled.all():
        s = np.zeros_like(U)
        cnt = np.zeros(U.shape)
        Uf = np.where(filled, U, 0.0)
        F = filled.astype(np.float64)
        for ax in range(3):
            for sh in (1, -1):
                src = [slice(None)] * 3
                dst = [slice(None)] * 3
                if sh == 1:
                    src[ax], dst[ax] = slice(0, -1), slice(1, None)
                else:
                    src[ax], dst[ax] = slice(1, None), slice(0, -1)
                s[tuple(dst)] += Uf[tuple(src)]
                cnt[tuple(dst)] += F[tuple(src)]
        new = (~filled) & (cnt > 0)
        U[new] = s[new] / cnt[new]
        filled |= new
        sweeps += 1
        if sweeps > max_sweeps:
            raise RuntimeError("fill did not converge")
    return U, sweeps


# ----------------------------------------------------------------------------- step 2
def unfold(X: np.ndarray, k: int) -> np.ndarray:
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1)


def mode_product(X: np.ndarray, M: np.ndarray, k: int) -> np.ndarray:
    """X x_k M (M has shape (J, I_k))."""
    Y = np.tensordot(M, X, axes=([1], [k]))
    return np.moveaxis(Y, 0, k)


def st_hosvd(U: np.ndarray, eps: float, max_rank, fixed_rank: bool = False):
    """Sequentially truncated HOSVD (Sec. 4.1): returns (core, [W1, W2, W3], eigvals).

    The eigen-decomposition of the mode Gram matrix uses numpy.linalg.eigh as a
    library step."""
    X = np.asarray(U, dtype=np.float64)
    d = X.ndim
    norm2 = float(np.sum(X * X))
    Ws, lams = [], []
    for k in range(d):
        Xk = unfold(X, k)
        S = Xk @ Xk.T
        lam, V = np.linalg.eigh(S)
        order = np.argsort(-lam, kind="stable")
        lam, V = lam[order], V[:, order]
        cap = min(int(max_rank[k]), X.shape[k])
        if fixed_rank:
            r = cap
        else:
            tail = np.concatenate([np.cumsum(lam[::-1])[::-1], [0.0]])  # tail[r] = sum_{i>=r}
            thr = eps * eps * norm2 / d
            r = next(rr for rr in range(1, lam.size + 1) if tail[rr] <= thr)
            r = min(r, cap)
        V = V[:, :r].copy()
        for j in range(r):
            i = int(np.argmax(np.abs(V[:, j])))
            if V[i, j] < 0:
                V[:, j] = -V[:, j]
        Ws.append(V)
        lams.append(lam)
        X = mode_product(X, V.T, k)
    return X, Ws, lams


def tucker_reconstruct(core: np.ndarray, Ws) -> np.ndarray:
    X = core
    for k, W in enumerate(Ws):
        X = mode_product(X, W, k)
    return X


# ----------------------------------------------------------------------------- step 3
def lars_lasso_path(X: np.ndarray, y: np.ndarray, max_steps: int | None = None,
                    breakpoints: list | None = None):
    """Least angle regression with the Lasso modification (Efron et al. 2004).

    Columns are scaled to unit norm for the correlations.  Returns the list of
    active sets (sorted tuples of column indices) visited by the path, in order.
    If ``breakpoints`` is a list, each step appends (beta, lam): the coefficients
    of the unit-norm columns after the step and the common absolute correlation
    lam of the active columns there (the Lasso penalty at that breakpoint)."""
    N, P = X.shape
    norms = np.linalg.norm(X, axis=0)
    usable = norms > 0
    Xn = np.zeros_like(X)
    Xn[:, usable] = X[:, usable] / norms[usable]
    beta = np.zeros(P)
    mu = np.zeros(N)
    active: list[int] = []
    path: list[tuple] = []
    ynorm = float(np.linalg.norm(y))
    if ynorm == 0.0:
        return path
    max_steps = max_steps or 8 * P + 8
    c = Xn.T @ y
    c[~usable] = 0.0
    nxt = int(np.argmax(np.abs(c)))
    for _ in range(max_steps):
        if nxt is not None:
            active.append(nxt)
            path.append(tuple(sorted(active)))
        c = Xn.T @ (y - mu)
        c[~usable] = 0.0
        A = np.array(active)
        C = float(np.max(np.abs(c[A])))
        if C <= 1e-14 * ynorm:
            break
        s = np.sign(c[A])
        s[s == 0] = 1.0
        XA = Xn[:, A] * s
        GA = XA.T @ XA
        try:
            g1 = np.linalg.solve(GA, np.ones(A.size))
        except np.linalg.LinAlgError:
            break
        denom = float(np.ones(A.size) @ g1)
        if denom <= 0:
            break
        AA = 1.0 / math.sqrt(denom)
        w = AA * g1
        uA = XA @ w
        a = Xn.T @ uA
        # step to the point where an inactive column's correlation ties the active ones
        gamma_enter, j_enter = C / AA, None
        if len(active) < min(N, int(usable.sum())):
            for j in range(P):
                if not usable[j] or j in active:
                    continue
                for cand in ((C - c[j]) / (AA - a[j]) if AA != a[j] else np.inf,
                             (C + c[j]) / (AA + a[j]) if AA != -a[j] else np.inf):
                    if 1e-15 < cand < gamma_enter:
                        gamma_enter, j_enter = cand, j
        # Lasso modification: stop where an active coefficient would change sign
        dvec = s * w
        gamma_drop, i_drop = np.inf, None
        for i, j in enumerate(active):
            if dvec[i] != 0:
                g = -beta[j] / dvec[i]
                if 1e-15 < g < gamma_drop:
                    gamma_drop, i_drop = g, i
        if gamma_drop < gamma_enter:
            gamma = gamma_drop
        else:
            gamma = gamma_enter
            i_drop = None
        mu = mu + gamma * uA
        beta[A] += gamma * dvec
        if i_drop is not None:
            j = active.pop(i_drop)
            beta[j] = 0.0
            path.append(tuple(sorted(active)))
            nxt = None
        else:
            nxt = j_enter
        if breakpoints is not None:
            breakpoints.append((beta.copy(), C - gamma * AA))
        if i_drop is None and nxt is None:   # reached the least-squares fit of the active set
            break
    return path


def loo_error(Phi: np.ndarray, y: np.ndarray, support) -> tuple[float, np.ndarray]:
    """Least-squares fit on a support and its leave-one-out error
    mean(((y_i - yhat_i) / (1 - h_ii))^2), h the hat matrix of the support."""
    S = list(support)
    B = Phi[:, S]
    Qm, Rm = np.linalg.qr(B)
    coef = np.linalg.solve(Rm, Qm.T @ y)
    res = y - B @ coef
    hdiag = np.sum(Qm * Qm, axis=1)
    if np.any(hdiag >= 1.0 - 1e-10):
        return math.inf, coef
    return float(np.mean((res / (1.0 - hdiag)) ** 2)), coef


def sparse_fit(Phi: np.ndarray, y: np.ndarray):
    """Sparse expansion of one column: the LARS-Lasso breakpoint whose least-squares
    refit has the least LOO error; ties within 1e-12 * mean(y^2) go to the smaller set,
    then to the earlier breakpoint.  Returns (rows, coefs, loo)."""
    path = lars_lasso_path(Phi, y)
    if not path:
        return np.zeros(1, np.int32), np.zeros(1), 0.0
    scale = float(np.mean(y * y))
    best = None
    seen = set()
    for order, S in enumerate(path):
        if S in seen or len(S) >= Phi.shape[0]:
            continue
        seen.add(S)
        err, coef = loo_error(Phi, y, S)
        key = (err, len(S), order)
        if best is None:
            best = (key, S, coef)
            continue
        (berr, blen, bord), _, _ = best
        if err < berr - 1e-12 * scale:
            best = (key, S, coef)
        elif abs(err - berr) <= 1e-12 * scale and (len(S), order) < (blen, bord):
            best = (key, S, coef)
    (err, _, _), S, coef = best
    return np.asarray(S, dtype=np.int32), np.asarray(coef, dtype=np.float64), err


def independent_columns(C: np.ndarray, tol: float = 1e-12) -> list:
    """Columns of C kept, in order, by modified Gram-Schmidt (two passes): column j is
    dropped when its squared residual against the kept ones is <= tol * ||c_j||^2, or it
    is zero.  With orthonormal basis functions the coefficient inner product is the
    function inner product, so this is linear dependence of the factor functions."""
    kept, Qs = [], []
    for j in range(C.shape[1]):
        c = np.asarray(C[:, j], dtype=np.float64)
        n2 = float(c @ c)
        v = c.copy()
        for _ in range(2):
            for q in Qs:
                v -= (q @ v) * q
        r2 = float(v @ v)
        if n2 == 0.0 or r2 <= tol * n2:
            continue
        kept.append(j)
        Qs.append(v / math.sqrt(r2))
    return kept


# ----------------------------------------------------------------------------- driver
@dataclass
class FitModel:
    """Fitted model: CSC coefficients per mode (degrees, values) and the C-ordered core."""
    r: tuple
    p: tuple
    colptr: list
    rowidx: list
    val: list
    alpha: np.ndarray
    lo: np.ndarray
    hi: np.ndarray

    @property
    def R(self) -> int:
        return int(self.r[0] * self.r[1] * self.r[2])

    def nnz(self) -> int:
        return int(sum(len(v) for v in self.val))

    wav: tuple | None = None            # (s, q) when some columns use W_{s,q}
    col_wavelet: list | None = None     # per mode, a bool per column

    def with_alpha(self, alpha) -> "FitModel":
        return FitModel(self.r, self.p, self.colptr, self.rowidx, self.val,
                        np.asarray(alpha, dtype=np.float64).reshape(self.r), self.lo, self.hi,
                        self.wav, self.col_wavelet)


@dataclass
class FitParams:
    grid: tuple = (32, 32, 32)
    sample_frac: float = 0.05
    eps: float = 1e-3
    max_rank: tuple = (8, 8, 8)
    max_degree: int = 15
    oversample: float = 4.0
    seed: int = 1
    fixed_rank: bool = False
    wavelet: tuple | None = None      # (s, q): also fit every column in W_{s,q} and keep the better


@dataclass
class FitReport:
    ranks: tuple = ()                 # after dropping dependent factor functions
    hosvd_ranks: tuple = ()           # chosen by the ST-HOSVD
    dropped: list = field(default_factory=list)   # per mode: dropped column indices
    chose_wavelet: list = field(default_factory=list)   # per mode, per ST-HOSVD column
    nnz: list = field(default_factory=list)       # per ST-HOSVD column
    loo: list = field(default_factory=list)
    fill_sweeps: int = 0
    m: int = 0
    refit_rc: int = 0
    compression_ratio: float = 0.0


def function_samples(p: int, wav, rows_vals_wavelet) -> np.ndarray:
    """Columns sampled so that dot products are the inner products <f, g> = 1/2 int f g
    of the functions: sqrt(weight / 2) f(x) at Gauss-Legendre nodes of every finest cell
    (exact for the piecewise polynomials of degree <= max(p, q) here).  rows_vals_wavelet:
    per column (rows, values, is_wavelet)."""
    s_, q_ = wav
    nc = 2 ** s_
    xg, wg = np.polynomial.legendre.leggauss(max(p, q_) + 1)
    nodes = np.concatenate([-1.0 + (2.0 * c + 1.0 + xg) / nc for c in range(nc)])
    wts = np.concatenate([wg / nc for _ in range(nc)])          # weights in t
    Pl = legendre_matrix(nodes, p)
    Bw = _wav.basis_matrix(nodes, -1.0, 1.0, s_, q_)
    S = np.empty((nodes.size, len(rows_vals_wavelet)))
    for j, (rows, vals, isw) in enumerate(rows_vals_wavelet):
        S[:, j] = (Bw if isw else Pl)[:, rows] @ vals
    return S * np.sqrt(wts / 2.0)[:, None]


def compression_ratio(Q: int, R: int, nnz: int) -> float:
    """Original storage over reduced storage, 8 bytes per value and only the values of
    nonzero coefficients counted, not their positions (Sec. 2; Table 2)."""
    return (8.0 * Q) / (8.0 * (R + nnz))


def fit(xyz: np.ndarray, u: np.ndarray, params: FitParams, lo=None, hi=None,
        grid_values: np.ndarray | None = None, nthreads: int = 1):
    """Algorithm 1 followed by the core refit of Algorithm 2 (uniform sampling form).

    ``grid_values`` replaces steps 1 (the test hook for exact-recovery pins)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    Q = xyz.shape[1]
    lo = np.full(3, -1.0) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.full(3, 1.0) if hi is None else np.asarray(hi, dtype=np.float64)
    t = 2.0 * (xyz - lo[:, None]) / (hi - lo)[:, None] - 1.0
    rep = FitReport()
    if grid_values is None:
        n_sub = int(math.ceil(params.sample_frac * Q))
        sub = _c_sample(params.seed, Q, n_sub)
        U, filled = interpolate_splat(t[:, sub], u[sub], params.grid)
        U, rep.fill_sweeps = fill_jacobi(U, filled)
    else:
        U = np.asarray(grid_values, dtype=np.float64)
    core, Ws, _ = st_hosvd(U, params.eps, params.max_rank, params.fixed_rank)
    rep.hosvd_ranks = tuple(W.shape[1] for W in Ws)
    colptr, rowidx, val, colwav = [], [], [], []
    for k in range(3):
        Phi = legendre_matrix(grid_nodes(U.shape[k]), params.max_degree)
        fits = [sparse_fit(Phi, Ws[k][:, j]) for j in range(Ws[k].shape[1])]
        isw = [False] * len(fits)
        if params.wavelet is not None:
            Phw = _wav.grid_basis_matrix(U.shape[k], int(params.wavelet[0]), int(params.wavelet[1]))
            for j in range(len(fits)):
                fw = sparse_fit(Phw, Ws[k][:, j])
                y = Ws[k][:, j]
                # the smaller LOO error; within 1e-12 mean(y^2) of each other, P_p
                if fw[2] < fits[j][2] - 1e-12 * float(np.mean(y * y)):
                    fits[j], isw[j] = fw, True
        rep.chose_wavelet.append(list(isw))
        rep.nnz.append([int(f[0].size) for f in fits])
        rep.loo.append([f[2] for f in fits])
        if params.wavelet is None:
            C = np.zeros((params.max_degree + 1, len(fits)))
            for j, (rows, coef, _) in enumerate(fits):
                C[rows, j] = coef
        else:
            C = function_samples(params.max_degree, params.wavelet,
                                 [(f[0], f[1], isw[j]) for j, f in enumerate(fits)])
        kept = independent_columns(C)
        rep.dropped.append([j for j in range(len(fits)) if j not in kept])
        colwav.append(np.asarray([isw[j] for j in kept], dtype=bool))
        core = np.take(core, kept, axis=k)
        cp = np.concatenate([[0], np.cumsum([fits[j][0].size for j in kept])]).astype(np.int32)
        colptr.append(cp)
        rowidx.append(np.concatenate([fits[j][0] for j in kept]).astype(np.int32))
        val.append(np.concatenate([fits[j][1] for j in kept]))
    r = tuple(c.size - 1 for c in colptr)
    rep.ranks = r
    p3 = (params.max_degree,) * 3
    anyw = params.wavelet is not None and any(c.any() for c in colwav)
    model = FitModel(r, p3, colptr, rowidx, val, core, lo, hi,
                     tuple(params.wavelet) if anyw else None, colwav if anyw else None)
    R = model.R
    m = min(int(math.ceil(params.oversample * R)), Q)
    idx = _c_sample((params.seed + REFIT_SEED_OFFSET) & 0xFFFFFFFFFFFFFFFF, Q, m)
    if anyw:
        alpha, rc = _wav.refit(model, xyz, u, idx), 0
    else:
        alpha, rc = _c_refit(model, xyz, u, idx, nthreads=nthreads)
    rep.m, rep.refit_rc = m, rc
    model = model.with_alpha(alpha)
    rep.compression_ratio = compression_ratio(Q, R, model.nnz())
    return model, rep
