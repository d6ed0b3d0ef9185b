"""Seeded synthetic inputs for the FST evaluation and refit path.

This module only *draws* inputs: point clouds, field values, random functional
sparse Tucker models and explicit row-index sets.  It contains none of the
method's arithmetic (no basis evaluation, no contraction, no least squares), so
the CUDA path and the CPU oracle can both be fed from it without sharing any
computation.

The combustion datasets of Sec. 6 (S3D "statistically planar" flame, SP3D/SP4D)
are not available; these fields stand in for them: a thin reaction front
(a tanh layer of width 0.1 across a curved surface) plus Gaussian blobs and a
small noise floor, sampled at unstructured points of which a fixed share is
clustered in a band around the front (the way an adaptive DNS mesh would
concentrate its points).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field as dc_field

import numpy as np


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed) & 0xFFFFFFFFFFFFFFFF, int(stream)])


# ----------------------------------------------------------------------------- points
def points(Q: int, seed: int, clustered: float = 0.3, dtype=np.float64) -> np.ndarray:
    """Q points in [-1,1]^3 as a (3, Q) structure-of-arrays array.

    A share ``1 - clustered`` is uniform in the cube; the rest lie in a band of
    width 0.05 (measured along x1) around the front surface
    x1 = -0.3 sin(3 x2) + 0.2 x3, redrawn until inside the cube.  The two
    groups are interleaved by a random permutation, so consecutive points are
    unstructured.
    """
    Q = int(Q)
    rng = _rng(seed, 1)
    n_c = int(round(clustered * Q))
    n_u = Q - n_c
    uni = rng.uniform(-1.0, 1.0, size=(3, n_u))
    cl = np.empty((3, n_c))
    todo = np.arange(n_c)
    while todo.size:
        x2 = rng.uniform(-1.0, 1.0, size=todo.size)
        x3 = rng.uniform(-1.0, 1.0, size=todo.size)
        x1 = -0.3 * np.sin(3.0 * x2) + 0.2 * x3 + rng.uniform(-0.025, 0.025, size=todo.size)
        ok = np.abs(x1) <= 1.0
        cl[0, todo[ok]] = x1[ok]
        cl[1, todo[ok]] = x2[ok]
        cl[2, todo[ok]] = x3[ok]
        todo = todo[~ok]
    perm = rng.permutation(Q)
    out = np.empty((3, Q), dtype=dtype)
    for k in range(3):      # row by row: the same values as gathering the stacked array
        out[k] = np.take(np.concatenate([uni[k], cl[k]]), perm)
    return out


# ----------------------------------------------------------------------------- fields
@dataclass
class FieldSpec:
    """A combustion-like scalar field: tanh fronts plus Gaussian blobs."""
    fronts: list = dc_field(default_factory=list)   # (normal(3), offset, width, curvature amp)
    gauss: list = dc_field(default_factory=list)    # (amp, width, centre(3))
    noise: float = 1e-4


def field_spec(seed: int, n_gauss: int, n_fronts: int = 1, randomize_fronts: bool = False,
               noise: float = 1e-4) -> FieldSpec:
    """Draw a field.  With ``randomize_fronts`` False the single front is the
    fixed surface x1 + 0.3 sin(3 x2) - 0.2 x3 = 0 with width 0.1."""
    rng = _rng(seed, 2)
    spec = FieldSpec(noise=noise)
    if not randomize_fronts:
        spec.fronts.append((np.array([1.0, 0.0, -0.2]), 0.0, 0.1, 0.3))
    else:
        for _ in range(n_fronts):
            nrm = rng.normal(size=3)
            nrm /= np.linalg.norm(nrm)
            spec.fronts.append((nrm, rng.uniform(-0.5, 0.5), rng.uniform(0.05, 0.2),
                                rng.uniform(0.0, 0.3)))
    for _ in range(n_gauss):
        spec.gauss.append((rng.uniform(0.5, 1.0), rng.uniform(0.1, 0.4),
                           rng.uniform(-1.0, 1.0, size=3)))
    return spec


def field_values(xyz: np.ndarray, spec: FieldSpec, seed: int, chunk: int = 1 << 22):
    """Return (u, u_clean): noisy samples and the noise-free field at ``xyz``."""
    Q = xyz.shape[1]
    clean = np.empty(Q)

    def one_chunk(s):
        x1, x2, x3 = (np.asarray(xyz[k, s:s + chunk], dtype=np.float64) for k in range(3))
        f = np.zeros_like(x1)
        for nrm, off, width, amp in spec.fronts:
            # fixed front: nrm=(1,0,-0.2), the curved term 0.3 sin(3 x2)
            f += np.tanh((nrm[0] * x1 + nrm[1] * x2 + nrm[2] * x3 + amp * np.sin(3.0 * x2) - off)
                         / width)
        for a, sig, c in spec.gauss:
            d2 = (x1 - c[0]) ** 2 + (x2 - c[1]) ** 2 + (x3 - c[2]) ** 2
            f += a * np.exp(-d2 / (2.0 * sig * sig))
        clean[s:s + chunk] = f

    starts = range(0, Q, chunk)
    if Q > chunk:       # chunks are independent: numpy releases the GIL, so threads share them
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(one_chunk, starts))
    else:
        for s in starts:
            one_chunk(s)
    noise = _rng(seed, 3).normal(size=Q) * spec.noise
    return clean + noise, clean


# ----------------------------------------------------------------------------- models
@dataclass
class Model:
    """A functional sparse Tucker model in host memory (eq. func_tuck, eq. sparse).

    ``colptr[k]``, ``rowidx[k]``, ``val[k]`` hold the CSC coefficient matrix of
    mode k: column j lists the degrees n and coefficients W^k_{n,j} of the
    orthonormal Legendre functions sqrt(2n+1) L_n.  ``alpha`` is the core in
    C order [j1][j2][j3].  ``lo``/``hi`` give the domain box mapped to [-1,1].
    """
    r: tuple
    p: tuple
    colptr: list
    rowidx: list
    val: list
    alpha: np.ndarray
    lo: np.ndarray = dc_field(default_factory=lambda: -np.ones(3))
    hi: np.ndarray = dc_field(default_factory=lambda: np.ones(3))
    wav: tuple | None = None            # (s, q): the multiwavelet space W_{s,q} of wavelet columns
    col_wavelet: list | None = None     # per mode, a bool per column: its rows index W_{s,q}

    @property
    def R(self) -> int:
        return int(self.r[0] * self.r[1] * self.r[2])

    def dense(self, k: int) -> np.ndarray:
        """Coefficient matrix of mode k as a dense (p_k+1) x r_k array."""
        W = np.zeros((self.p[k] + 1, self.r[k]))
        for j in range(self.r[k]):
            s, e = self.colptr[k][j], self.colptr[k][j + 1]
            W[self.rowidx[k][s:e], j] = self.val[k][s:e]
        return W

    def nnz(self) -> int:
        return int(sum(len(v) for v in self.val))

    def with_alpha(self, alpha: np.ndarray) -> "Model":
        return Model(self.r, self.p, self.colptr, self.rowidx, self.val,
                     np.asarray(alpha, dtype=np.float64).reshape(self.r), self.lo, self.hi,
                     self.wav, self.col_wavelet)


def random_model(r, p, seed: int, density: float = 0.6, decay: float = 1.0,
                 lo=None, hi=None, orthonormal: bool = False) -> Model:
    """A random model with ranks ``r`` and maximum degrees ``p``.

    Column j of mode k keeps max(1, round(density*(p_k+1))) randomly chosen
    degrees (always including one of degree <= j, the way low singular vectors
    are smooth); its coefficients are normal, scaled to unit 2-norm.  Core
    entries are normal with magnitude decaying like 1/(1+j1+j2+j3)^decay, the
    way a Tucker core sorted by singular value decays (Fig. 1).

    With ``orthonormal`` the coefficient columns of each mode are instead the
    first r_k columns of a random orthogonal matrix (all degrees stored), so the
    factor functions are orthonormal on [-1,1] like fitted singular vectors.
    """
    r = tuple(int(v) for v in r)
    p = tuple(int(v) for v in (p if np.ndim(p) else (p, p, p)))
    rng = _rng(seed, 4)
    colptr, rowidx, val = [], [], []
    for k in range(3):
        n = p[k] + 1
        if orthonormal:
            if r[k] > n:
                raise ValueError("orthonormal factors need r_k <= p_k + 1")
            Qm = np.linalg.qr(rng.normal(size=(n, n)))[0][:, :r[k]]
            colptr.append(np.arange(0, n * r[k] + 1, n, dtype=np.int32))
            rowidx.append(np.tile(np.arange(n, dtype=np.int32), r[k]))
            val.append(np.ascontiguousarray(Qm.T).reshape(-1))
            continue
        keep = max(1, min(n, int(round(density * n))))
        cp, ri, vv = [0], [], []
        for j in range(r[k]):
            low = int(rng.integers(0, min(j, n - 1) + 1))
            others = rng.permutation(np.setdiff1d(np.arange(n), [low]))[:keep - 1]
            rows = np.sort(np.concatenate([[low], others])).astype(np.int32)
            c = rng.normal(size=rows.size)
            c /= np.linalg.norm(c)
            ri.append(rows)
            vv.append(c)
            cp.append(cp[-1] + rows.size)
        colptr.append(np.asarray(cp, dtype=np.int32))
        rowidx.append(np.concatenate(ri).astype(np.int32))
        val.append(np.concatenate(vv).astype(np.float64))
    j1, j2, j3 = np.meshgrid(np.arange(r[0]), np.arange(r[1]), np.arange(r[2]), indexing="ij")
    alpha = rng.normal(size=r) / (1.0 + j1 + j2 + j3) ** decay
    lo = -np.ones(3) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.ones(3) if hi is None else np.asarray(hi, dtype=np.float64)
    return Model(r, p, colptr, rowidx, val, alpha, lo, hi)


def with_wavelet_columns(m: Model, wav=(3, 5), share: float = 0.5, seed: int = 0, density: float = 0.3) -> Model:
    """A copy of model m where a share of the columns of every mode (at least one, never all
    when r_k > 1) are replaced by random sparse unit-norm expansions in the multiwavelet
    space W_{s,q} (function indices 0 .. (q+1) 2^s - 1), the rest kept."""
    s_, q_ = int(wav[0]), int(wav[1])
    nw = (q_ + 1) * 2 ** s_
    rng = _rng(seed, 7)
    colptr, rowidx, val, flags = [], [], [], []
    for k in range(3):
        r = m.r[k]
        nwc = max(1, min(r - 1 if r > 1 else 1, int(round(share * r))))
        wcols = set(rng.choice(r, size=nwc, replace=False).tolist())
        cp, ri, vv, fl = [0], [], [], []
        for j in range(r):
            if j in wcols:
                keep = max(1, int(round(density * nw)))
                rows = np.sort(rng.choice(nw, size=keep, replace=False)).astype(np.int32)
                c = rng.normal(size=rows.size)
                c /= np.linalg.norm(c)
            else:
                s0, e0 = m.colptr[k][j], m.colptr[k][j + 1]
                rows = np.asarray(m.rowidx[k][s0:e0], dtype=np.int32)
                c = np.asarray(m.val[k][s0:e0], dtype=np.float64)
            ri.append(rows)
            vv.append(c)
            cp.append(cp[-1] + rows.size)
            fl.append(j in wcols)
        colptr.append(np.asarray(cp, dtype=np.int32))
        rowidx.append(np.concatenate(ri).astype(np.int32))
        val.append(np.concatenate(vv).astype(np.float64))
        flags.append(np.asarray(fl, dtype=bool))
    return Model(m.r, m.p, colptr, rowidx, val, m.alpha, m.lo, m.hi, (s_, q_), flags)


def row_indices(Q: int, m: int, seed: int) -> np.ndarray:
    """m distinct row indices of [0, Q), ascending (explicit sample sets for parity tests)."""
    rng = _rng(seed, 5)
    m = min(int(m), int(Q))
    return np.sort(rng.choice(int(Q), size=m, replace=False)).astype(np.int64)


# ----------------------------------------------------------------------------- workloads
@dataclass
class Workload:
    """One named workload (point count, field, ranks, degree, refit oversampling)."""
    name: str
    Q: int
    n_gauss: int
    grid: int
    sample_frac: float
    max_rank: int
    degree: int
    oversample: float
    eps: float
    clustered: float
    seed: int


WORKLOADS = {
    # 20,000 uniform points, 5 Gaussians, 5% onto 32^3, eps 1e-3, ranks <= 8, degree <= 15, m = 4R
    "fp64_small": Workload("fp64_small", 20_000, 5, 32, 0.05, 8, 15, 4.0, 1e-3, 0.0, 101),
    # 2^24 points (70% uniform, 30% in the front band), 20 Gaussians, 2% onto 128^3,
    # ranks <= 24, degree <= 31, m = 8R
    "fp32_16M": Workload("fp32_16M", 1 << 24, 20, 128, 0.02, 24, 31, 8.0, 1e-4, 0.3, 202),
    # 2^26 points, 256^3 grid, ranks fixed at 24, degree <= 63, m = 8R
    "precision_64M": Workload("precision_64M", 1 << 26, 20, 256, 0.02, 24, 63, 8.0, 0.0, 0.3, 303),
}


def log_uniform_int(rng: np.random.Generator, lo: float, hi: float, size=None):
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=size)).astype(np.int64)


def batch_instances(n_fields: int = 64, n_steps: int = 8, seed: int = 404,
                    q_lo: float = 1e5, q_hi: float = 2e6, r_lo: int = 4, r_hi: int = 24):
    """Instance table of the batching workload: fields x timesteps with uneven
    ranks (independently U{r_lo..r_hi} per mode) and log-uniform point counts."""
    rng = _rng(seed, 6)
    out = []
    for f in range(n_fields):
        for t in range(n_steps):
            r = tuple(int(v) for v in rng.integers(r_lo, r_hi + 1, size=3))
            Q = int(log_uniform_int(rng, q_lo, q_hi))
            out.append({"field": f, "step": t, "r": r, "Q": Q,
                        "seed": int(rng.integers(0, 2**62))})
    return out


# ----------------------------------------------------------------------------- order 4
# Four-way models and inputs, the SP4D-like case (three space axes and time): the same
# recipes with a fourth coordinate.
@dataclass
class Model4:
    """An order-4 functional sparse Tucker model (eq. func_tuck with d = 4): CSC coefficient
    matrices of the orthonormal Legendre functions per mode, the core alpha[j1][j2][j3][j4]
    in C order, and the box [lo_k, hi_k] of each coordinate."""
    r: tuple
    p: tuple
    colptr: list
    rowidx: list
    val: list
    alpha: np.ndarray
    lo: np.ndarray = dc_field(default_factory=lambda: -np.ones(4))
    hi: np.ndarray = dc_field(default_factory=lambda: np.ones(4))

    @property
    def R(self) -> int:
        return int(np.prod(self.r))

    def with_alpha(self, alpha: np.ndarray) -> "Model4":
        return Model4(self.r, self.p, self.colptr, self.rowidx, self.val,
                      np.asarray(alpha, dtype=np.float64).reshape(self.r), self.lo, self.hi)


def random_model4(r, p, seed: int, density: float = 0.6, orthonormal: bool = False, lo=None, hi=None) -> Model4:
    """A random order-4 model: the coefficient columns and core of random_model drawn for
    four modes (orthonormal columns when asked; core entries normal, decaying like
    1/(1 + j1 + j2 + j3 + j4))."""
    r = tuple(int(v) for v in r)
    p = tuple(int(v) for v in (p if np.ndim(p) else (p,) * 4))
    rng = _rng(seed, 8)
    colptr, rowidx, val = [], [], []
    for k in range(4):
        n = p[k] + 1
        if orthonormal:
            if r[k] > n:
                raise ValueError("orthonormal factors need r_k <= p_k + 1")
            Qm = np.linalg.qr(rng.normal(size=(n, n)))[0][:, :r[k]]
            colptr.append(np.arange(0, n * r[k] + 1, n, dtype=np.int32))
            rowidx.append(np.tile(np.arange(n, dtype=np.int32), r[k]))
            val.append(np.ascontiguousarray(Qm.T).reshape(-1))
            continue
        keep = max(1, min(n, int(round(density * n))))
        cp, ri, vv = [0], [], []
        for j in range(r[k]):
            low = int(rng.integers(0, min(j, n - 1) + 1))
            others = rng.permutation(np.setdiff1d(np.arange(n), [low]))[:keep - 1]
            rows = np.sort(np.concatenate([[low], others])).astype(np.int32)
            c = rng.normal(size=rows.size)
            c /= np.linalg.norm(c)
            ri.append(rows)
            vv.append(c)
            cp.append(cp[-1] + rows.size)
        colptr.append(np.asarray(cp, dtype=np.int32))
        rowidx.append(np.concatenate(ri).astype(np.int32))
        val.append(np.concatenate(vv).astype(np.float64))
    g = np.meshgrid(*[np.arange(v) for v in r], indexing="ij")
    alpha = rng.normal(size=r) / (1.0 + g[0] + g[1] + g[2] + g[3])
    lo = -np.ones(4) if lo is None else np.asarray(lo, dtype=np.float64)
    hi = np.ones(4) if hi is None else np.asarray(hi, dtype=np.float64)
    return Model4(r, p, colptr, rowidx, val, alpha, lo, hi)


def points4(Q: int, seed: int, clustered: float = 0.3, dtype=np.float64) -> np.ndarray:
    """Q points in [-1,1]^4 as a (4, Q) structure-of-arrays array: the three space axes of
    points() (uniform share and the band around the moving front) and a time coordinate t
    uniform in [-1, 1]; the band follows the front x1 = -0.3 sin(3 x2) + 0.2 x3 + 0.2 t."""
    Q = int(Q)
    rng = _rng(seed, 9)
    t = rng.uniform(-1.0, 1.0, size=Q)
    n_c = int(round(clustered * Q))
    n_u = Q - n_c
    uni = rng.uniform(-1.0, 1.0, size=(3, n_u))
    cl = np.empty((3, n_c))
    tc = t[n_u:]
    todo = np.arange(n_c)
    while todo.size:
        x2 = rng.uniform(-1.0, 1.0, size=todo.size)
        x3 = rng.uniform(-1.0, 1.0, size=todo.size)
        x1 = -0.3 * np.sin(3.0 * x2) + 0.2 * x3 + 0.2 * tc[todo] + rng.uniform(-0.025, 0.025, size=todo.size)
        ok = np.abs(x1) <= 1.0
        cl[0, todo[ok]] = x1[ok]
        cl[1, todo[ok]] = x2[ok]
        cl[2, todo[ok]] = x3[ok]
        todo = todo[~ok]
    perm = rng.permutation(Q)
    out = np.empty((4, Q), dtype=dtype)
    for k in range(3):
        out[k] = np.take(np.concatenate([uni[k], cl[k]]), perm)
    out[3] = np.take(t, perm)
    return out


def field_values4(xyzt: np.ndarray, spec: FieldSpec, seed: int):
    """Return (u, u_clean) of a moving field: the fronts of ``spec`` advected along x1 by
    0.2 t and its Gaussian blobs with amplitudes modulated by (1 + 0.3 sin(2 t))."""
    x1, x2, x3, t = (np.asarray(xyzt[k], dtype=np.float64) for k in range(4))
    f = np.zeros_like(x1)
    for nrm, off, width, amp in spec.fronts:
        f += np.tanh((nrm[0] * x1 + nrm[1] * x2 + nrm[2] * x3 + amp * np.sin(3.0 * x2) - 0.2 * t - off) / width)
    for a, sig, c in spec.gauss:
        d2 = (x1 - c[0]) ** 2 + (x2 - c[1]) ** 2 + (x3 - c[2]) ** 2
        f += a * (1.0 + 0.3 * np.sin(2.0 * t)) * np.exp(-d2 / (2.0 * sig * sig))
    noise = _rng(seed, 10).normal(size=x1.size) * spec.noise
    return f + noise, f
