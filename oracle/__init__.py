"""Plain FP64 CPU oracle for the functional sparse Tucker (FST) path.

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` are the only code
allowed to import this package.  The CUDA library and its Python binding never
import, link or call it, and share no code with it.

``fst_oracle.c`` holds the evaluation (Sec. 2, eq. func_tuck / eq. sparse), the
row sampler and the least-squares core refit (Sec. 5, eq. rand_core,
Algorithm 2); ``mixing.py`` holds Algorithm 2's sign flip and fast mixing of the
rows; ``fit.py`` holds the construction steps of Algorithm 1 (interpolation,
ST-HOSVD, sparse Legendre fit, choice between the Legendre and multiwavelet
spaces); ``wavelet.py`` holds the multiwavelet spaces and the evaluation and
refit of models whose factor functions use them; ``order4.py`` holds the
evaluation and refit of order-4 models (the SP4D case).  Parity status of each function
is stated in its docstring; every function here is pinned by a ``-m "not gpu"``
test against closed forms, library routines or brute force, except where a
docstring says "parity unpinned".
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "libfst_oracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile fst_oracle.c with gcc (OpenMP when the compiler supports it)."""
    src = _HERE / "fst_oracle.c"
    hdr = _HERE / "fst_oracle.h"
    if (not force and _LIB_PATH.exists()
            and _LIB_PATH.stat().st_mtime > max(src.stat().st_mtime, hdr.stat().st_mtime)):
        return _LIB_PATH
    _BUILD.mkdir(exist_ok=True)
    tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp")
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", str(src),
            "-o", str(tmp), "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [
        ("r", C.c_int32 * 3), ("p", C.c_int32 * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("colptr", C.c_void_p * 3), ("rowidx", C.c_void_p * 3), ("val", C.c_void_p * 3),
        ("alpha", C.c_void_p),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(_LIB_PATH))
        P, I32, I64, U64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
        sig = {
            "fst_oracle_legendre": (None, [D, I32, P]),
            "fst_oracle_factor_values": (None, [P, I32, D, P]),
            "fst_oracle_eval_point": (D, [P, D, D, D]),
            "fst_oracle_eval": (None, [P, P, I64, P, I32]),
            "fst_oracle_key": (U64, [U64, U64]),
            "fst_oracle_sample": (None, [U64, I64, I64, P]),
            "fst_oracle_design_row": (None, [P, D, D, D, P]),
            "fst_oracle_design_matrix": (None, [P, P, I64, P, I64, P]),
            "fst_oracle_normal_equations": (None, [P, P, P, I64, P, I64, P, P, P, I32]),
            "fst_oracle_cholesky": (I32, [P, I32, I32]),
            "fst_oracle_cholesky_solve": (None, [P, I32, P, P]),
            "fst_oracle_lsq_qr": (I32, [P, I64, I32, P, P]),
            "fst_oracle_refit": (I32, [P, P, P, I64, P, I64, P, I32]),
            "fst_oracle_normal_residual": (None, [P, P, P, I64, P, I64, P, P, I32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


class OracleModel:
    """ctypes view of a host model (anything with r, p, lo, hi, colptr, rowidx, val, alpha)."""

    def __init__(self, m):
        self.r = tuple(int(v) for v in m.r)
        self.p = tuple(int(v) for v in m.p)
        self._keep = []
        s = _Model()
        for k in range(3):
            s.r[k] = self.r[k]
            s.p[k] = self.p[k]
            s.lo[k] = float(m.lo[k])
            s.hi[k] = float(m.hi[k])
            cp = np.ascontiguousarray(m.colptr[k], dtype=np.int32)
            ri = np.ascontiguousarray(m.rowidx[k], dtype=np.int32)
            vv = np.ascontiguousarray(m.val[k], dtype=np.float64)
            if ri.size == 0:
                ri = np.zeros(1, np.int32)
                vv = np.zeros(1, np.float64)
            self._keep += [cp, ri, vv]
            s.colptr[k] = cp.ctypes.data
            s.rowidx[k] = ri.ctypes.data
            s.val[k] = vv.ctypes.data
        al = np.ascontiguousarray(np.asarray(m.alpha, dtype=np.float64).reshape(-1))
        self._keep.append(al)
        s.alpha = al.ctypes.data
        self.struct = s
        self.R = self.r[0] * self.r[1] * self.r[2]

    @property
    def ref(self):
        return C.byref(self.struct)


def legendre(t: float, p: int) -> np.ndarray:
    """L_0..L_p(t), Bonnet recurrence.  Pinned: closed forms at +-1 and 0, numpy legval,
    Gauss-Legendre orthogonality."""
    out = np.empty(p + 1)
    lib().fst_oracle_legendre(float(t), int(p), _ptr(out))
    return out


def factor_values(model, k: int, yk: float) -> np.ndarray:
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    out = np.empty(om.r[k])
    lib().fst_oracle_factor_values(om.ref, int(k), float(yk), _ptr(out))
    return out


def _wavelet_model(model) -> bool:
    """Models with columns in a multiwavelet space go to the numpy path of wavelet.py."""
    from . import wavelet
    return not isinstance(model, OracleModel) and wavelet.has_wavelets(model)


def eval_points(model, xyz: np.ndarray, nthreads: int = 1) -> np.ndarray:
    """u~ at the columns of xyz (3, n), eq. func_tuck by the plain triple sum.
    Pinned: rank-one cores vs numpy legval products, the full tensor-product
    expansion of Sec. 2, and the affine box map."""
    if _wavelet_model(model):
        from . import wavelet
        return wavelet.eval_points(model, xyz)
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    y = np.ascontiguousarray(xyz, dtype=np.float64)
    n = y.shape[1]
    out = np.empty(n)
    lib().fst_oracle_eval(om.ref, _ptr(y), n, _ptr(out), int(nthreads))
    return out


def key(seed: int, q: int) -> int:
    return int(lib().fst_oracle_key(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), C.c_uint64(q)))


def sample(seed: int, Q: int, m: int) -> np.ndarray:
    """The m rows of [0,Q) with the smallest splitmix64 keys, ascending.  Pinned by
    bijectivity of the finaliser, brute-force selection on tiny inputs, and
    uniformity statistics."""
    m = min(int(m), int(Q))
    out = np.empty(m, dtype=np.int64)
    lib().fst_oracle_sample(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(Q), m, _ptr(out))
    return out


def design_matrix(model, xyz: np.ndarray, idx: np.ndarray) -> np.ndarray:
    if _wavelet_model(model):
        from . import wavelet
        return wavelet.design_matrix(model, xyz, idx)
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    y = np.ascontiguousarray(xyz, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    A = np.empty((idx.size, om.R))
    lib().fst_oracle_design_matrix(om.ref, _ptr(y), y.shape[1], _ptr(idx), idx.size, _ptr(A))
    return A


def normal_equations(model, xyz, u, idx, nthreads: int = 1):
    if _wavelet_model(model):
        from . import wavelet
        A = wavelet.design_matrix(model, xyz, idx)
        b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
        return A.T @ A, A.T @ b, float(b @ b)
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    y = np.ascontiguousarray(xyz, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    G = np.empty((om.R, om.R))
    h = np.empty(om.R)
    btb = np.zeros(1)
    lib().fst_oracle_normal_equations(om.ref, _ptr(y), _ptr(u), y.shape[1], _ptr(idx), idx.size,
                                      _ptr(G), _ptr(h), _ptr(btb), int(nthreads))
    return G, h, float(btb[0])


def cholesky(G: np.ndarray, nthreads: int = 1):
    L = np.ascontiguousarray(G, dtype=np.float64).copy()
    rc = lib().fst_oracle_cholesky(_ptr(L), L.shape[0], int(nthreads))
    return L, int(rc)


def cholesky_solve(L: np.ndarray, h: np.ndarray) -> np.ndarray:
    L = np.ascontiguousarray(L, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    x = np.empty_like(h)
    lib().fst_oracle_cholesky_solve(_ptr(L), L.shape[0], _ptr(h), _ptr(x))
    return x


def lsq_qr(A: np.ndarray, b: np.ndarray):
    A = np.ascontiguousarray(A, dtype=np.float64).copy()
    b = np.ascontiguousarray(b, dtype=np.float64).copy()
    x = np.empty(A.shape[1])
    rc = lib().fst_oracle_lsq_qr(_ptr(A), A.shape[0], A.shape[1], _ptr(b), _ptr(x))
    return x, int(rc)


def refit(model, xyz, u, idx, nthreads: int = 1):
    """Core refit on rows idx (eq. rand_core): normal equations + Cholesky, QR fallback.
    Returns (alpha (r1, r2, r3), rc) with rc 0 = Cholesky, 1 = QR.  Pinned: normal-equation
    residual, m = Q against numpy lstsq, exact recovery, orthogonal-mixing invariance."""
    if _wavelet_model(model):
        from . import wavelet
        return wavelet.refit(model, xyz, u, idx), 0
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    y = np.ascontiguousarray(xyz, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    al = np.empty(om.R)
    rc = lib().fst_oracle_refit(om.ref, _ptr(y), _ptr(u), y.shape[1], _ptr(idx), idx.size,
                                _ptr(al), int(nthreads))
    return al.reshape(om.r), int(rc)


def normal_residual(model, xyz, u, idx, alpha, nthreads: int = 1) -> np.ndarray:
    if _wavelet_model(model):
        from . import wavelet
        A = wavelet.design_matrix(model, xyz, idx)
        b = np.asarray(u, dtype=np.float64)[np.asarray(idx, dtype=np.int64)]
        return A.T @ (A @ np.asarray(alpha, dtype=np.float64).reshape(-1) - b)
    om = model if isinstance(model, OracleModel) else OracleModel(model)
    y = np.ascontiguousarray(xyz, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
    g = np.empty(om.R)
    lib().fst_oracle_normal_residual(om.ref, _ptr(y), _ptr(u), y.shape[1], _ptr(idx), idx.size,
                                     _ptr(al), _ptr(g), int(nthreads))
    return g
