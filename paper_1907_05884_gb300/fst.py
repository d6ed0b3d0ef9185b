"""ctypes binding of libfst (include/fst.h): argument marshalling only.

Every step of evaluation, sampling and refit runs in libfst's CUDA kernels; this
module converts Python objects to the C ABI's plain pointers and sizes.  PyTorch
provides device memory and streams.  Importing this module loads the in-tree
``libfst.so`` and raises if it has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libfst.so"

FST_FP64, FST_FP32, FST_TF32, FST_BF16, FST_BF16X3 = 0, 1, 2, 3, 4
PREC = {"fp64": FST_FP64, "fp32": FST_FP32, "tf32": FST_TF32, "bf16": FST_BF16, "bf16x3": FST_BF16X3}
STATUS = {0: "FST_OK", -1: "FST_EINVAL", -2: "FST_ENOMEM", -3: "FST_ECUDA", -4: "FST_ENOTSPD",
          -5: "FST_ERANK", -6: "FST_ETIMEOUT", -7: "FST_EFORMAT", -8: "FST_ENOTCONV",
          -9: "FST_EUNSUPPORTED"}


class FstError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class ModelDesc(C.Structure):
    _fields_ = [
        ("r", C.c_int32 * 3), ("p", C.c_int32 * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("colptr", C.c_void_p * 3), ("rowidx", C.c_void_p * 3), ("val", C.c_void_p * 3),
        ("alpha", C.c_void_p),
    ]


class Model4Desc(C.Structure):
    _fields_ = [
        ("r", C.c_int32 * 4), ("p", C.c_int32 * 4),
        ("lo", C.c_double * 4), ("hi", C.c_double * 4),
        ("colptr", C.c_void_p * 4), ("rowidx", C.c_void_p * 4), ("val", C.c_void_p * 4),
        ("alpha", C.c_void_p),
    ]


class WaveletDesc(C.Structure):
    _fields_ = [("level", C.c_int32), ("degree", C.c_int32), ("col_wavelet", C.c_void_p * 3)]


class EvalItem(C.Structure):
    _fields_ = [("model", C.c_void_p), ("xyz", C.c_void_p), ("n", C.c_int64), ("out", C.c_void_p)]


class RefitOpts(C.Structure):
    _fields_ = [("max_refine", C.c_int32), ("refine_tol", C.c_double), ("fp64_cholesky", C.c_int32)]


class RefitReport(C.Structure):
    _fields_ = [("m", C.c_int64), ("refine_steps", C.c_int32), ("fallback_fp64", C.c_int32),
                ("fallback_bf16x3", C.c_int32), ("shifted_preconditioner", C.c_int32),
                ("first_rel_change", C.c_double), ("last_rel_update", C.c_double),
                ("ms_sample", C.c_double), ("ms_factors", C.c_double), ("ms_gram", C.c_double),
                ("ms_cholesky", C.c_double), ("ms_refine", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RefitItem(C.Structure):
    _fields_ = [("model", C.c_void_p), ("xyz", C.c_void_p), ("u", C.c_void_p), ("Q", C.c_int64),
                ("m", C.c_int64), ("seed", C.c_uint64)]


class FitParams(C.Structure):
    _fields_ = [("grid", C.c_int32 * 3), ("sample_frac", C.c_double), ("eps", C.c_double),
                ("max_rank", C.c_int32 * 3), ("max_degree", C.c_int32), ("fixed_rank", C.c_int32),
                ("oversample", C.c_double), ("seed", C.c_uint64), ("grid_values", C.c_void_p),
                ("wavelet", C.c_int32), ("wav_level", C.c_int32), ("wav_degree", C.c_int32)]


class FitReport(C.Structure):
    _fields_ = [("r", C.c_int32 * 3), ("r_hosvd", C.c_int32 * 3), ("nnz", C.c_int32 * 3),
                ("fill_sweeps", C.c_int32),
                ("eig_sweeps", C.c_int32 * 3), ("n_interp", C.c_int64), ("m", C.c_int64),
                ("compression_ratio", C.c_double), ("ms_interp", C.c_double), ("ms_hosvd", C.c_double),
                ("ms_sparse", C.c_double), ("ms_refit", C.c_double), ("refit", RefitReport),
                ("n_wavelet", C.c_int32 * 3)]

    def as_dict(self):
        d = {}
        for f, _ in self._fields_:
            v = getattr(self, f)
            d[f] = v.as_dict() if f == "refit" else (tuple(v) if f in ("r", "r_hosvd", "nnz", "eig_sweeps",
                                                                           "n_wavelet") else v)
        return d


class FitTrace(C.Structure):
    _fields_ = [("grid_values", C.c_void_p), ("eigvals", C.c_void_p * 3), ("W", C.c_void_p * 3),
                ("core_hosvd", C.c_void_p), ("col_nnz", C.c_void_p), ("col_loo", C.c_void_p),
                ("col_kept", C.c_void_p), ("col_wavelet", C.c_void_p), ("col_loo_alt", C.c_void_p)]


def _load():
    if not LIB_PATH.exists():
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1907_05884_gb300.build.build() "
                          "(libfst has no CPU fallback)")
    L = C.CDLL(str(LIB_PATH))
    P, I32, I64, U64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    sig = {
        "fst_model_create": (I32, [P, P]),
        "fst_model4_create": (I32, [P, P]),
        "fst_model4_free": (None, [P]),
        "fst_model4_read_core": (I32, [P, P]),
        "fst_eval4": (I32, [P, P, I64, P, P]),
        "fst_eval4_f64": (I32, [P, P, I64, P, P]),
        "fst_refit4": (I32, [P, P, P, I64, I64, U64, I32, P, P, P]),
        "fst_model_create_wavelet": (I32, [P, P, P]),
        "fst_model_read_wavelet": (I32, [P, P, P, P]),
        "fst_model_free": (None, [P]),
        "fst_model_shape": (I32, [P, P, P, P]),
        "fst_model_read": (I32, [P, P, P, P, P, P, P]),
        "fst_model_set_core": (I32, [P, P]),
        "fst_model_save": (I32, [P, C.c_char_p]),
        "fst_model_load": (I32, [C.c_char_p, P]),
        "fst_eval": (I32, [P, P, I64, P, I32, P]),
        "fst_eval_f64": (I32, [P, P, I64, P, P]),
        "fst_eval_prepare": (I32, [P, I32]),
        "fst_eval_batched": (I32, [P, I32, I32, P]),
        "fst_slice_points": (I32, [I32, C.c_double, P, P, I32, I32, P, P]),
        "fst_eval_plan_create": (I32, [P, I32, I32, P]),
        "fst_eval_plan_run": (I32, [P, P]),
        "fst_eval_plan_free": (None, [P]),
        "fst_eval_check": (I32, [P]),
        "fst_eval_autotune": (I32, [P, I32, I64, P, P, P, P]),
        "fst_eval_autotune_set": (I32, [P, I32, I32]),
        "fst_sample_rows": (I32, [U64, I64, I64, P, P]),
        "fst_sample_rows_static": (I32, [U64, I64, I64, P, P]),
        "fst_refit": (I32, [P, P, P, I64, P, I64, U64, I32, P, P, P]),
        "fst_refit_f64": (I32, [P, P, P, I64, P, I64, U64, P, P, P]),
        "fst_refit_batched": (I32, [P, I32, I32, P, I32, P]),
        "fst_refit_grouped": (I32, [P, I32, I32, P, P, P]),
        "fst_refit_mixed": (I32, [P, P, P, I64, I64, U64, U64, P, P]),
        "fst_normal_matrix": (I32, [P, P, P, I64, P, I64, I32, P, P, P]),
        "fst_fit": (I32, [P, P, I64, P, P, P, I32, P, P, P, P, P]),
        "fst_cholesky_f32": (I32, [P, I32, P]),
        "fst_set_wait_limit": (I32, [I64]),
        "fst_status_str": (C.c_char_p, [I32]),
        "fst_last_error": (C.c_char_p, []),
        "fst_build_info": (C.c_char_p, []),
        "fst_kernel_launches": (U64, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _check(st: int):
    if st != 0:
        raise FstError(st, lib.fst_last_error().decode(errors="replace"))


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dptr(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Model:
    """A device-resident FST model owned by libfst."""

    def __init__(self, host_model=None, _handle=None):
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
            return
        m = host_model
        d = ModelDesc()
        keep = []
        for k in range(3):
            d.r[k] = int(m.r[k])
            d.p[k] = int(m.p[k])
            d.lo[k] = float(m.lo[k])
            d.hi[k] = float(m.hi[k])
            cp = np.ascontiguousarray(m.colptr[k], dtype=np.int32)
            ri = np.ascontiguousarray(m.rowidx[k], dtype=np.int32)
            vv = np.ascontiguousarray(m.val[k], dtype=np.float64)
            if ri.size == 0:
                ri, vv = np.zeros(1, np.int32), np.zeros(1)
            keep += [cp, ri, vv]
            d.colptr[k], d.rowidx[k], d.val[k] = cp.ctypes.data, ri.ctypes.data, vv.ctypes.data
        al = np.ascontiguousarray(np.asarray(m.alpha, dtype=np.float64).reshape(-1))
        keep.append(al)
        d.alpha = al.ctypes.data
        cw = getattr(m, "col_wavelet", None)
        if cw is not None and getattr(m, "wav", None) is not None and any(np.any(c) for c in cw):
            w = WaveletDesc()
            w.level, w.degree = int(m.wav[0]), int(m.wav[1])
            for k in range(3):
                f = np.ascontiguousarray(np.asarray(cw[k], dtype=bool).astype(np.uint8))
                keep.append(f)
                w.col_wavelet[k] = f.ctypes.data
            _check(lib.fst_model_create_wavelet(C.byref(d), C.byref(w), C.byref(self._h)))
        else:
            _check(lib.fst_model_create(C.byref(d), C.byref(self._h)))

    @classmethod
    def load(cls, path: str) -> "Model":
        h = C.c_void_p()
        _check(lib.fst_model_load(str(path).encode(), C.byref(h)))
        return cls(_handle=h)

    def save(self, path: str):
        _check(lib.fst_model_save(self._h, str(path).encode()))

    def free(self):
        if self._h:
            lib.fst_model_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def shape(self):
        r, p, nnz = (C.c_int32 * 3)(), (C.c_int32 * 3)(), (C.c_int32 * 3)()
        _check(lib.fst_model_shape(self._h, r, p, nnz))
        return tuple(r), tuple(p), tuple(nnz)

    def read(self):
        """Host copy: dict with colptr, rowidx, val (lists per mode), alpha (r1,r2,r3), lo, hi."""
        r, p, nnz = self.shape()
        cps = [np.empty(r[k] + 1, np.int32) for k in range(3)]
        ris = [np.empty(max(nnz[k], 1), np.int32) for k in range(3)]
        vvs = [np.empty(max(nnz[k], 1), np.float64) for k in range(3)]
        al = np.empty(r[0] * r[1] * r[2])
        lo, hi = np.empty(3), np.empty(3)
        arr = lambda xs: (C.c_void_p * 3)(*[x.ctypes.data for x in xs])
        _check(lib.fst_model_read(self._h, arr(cps), arr(ris), arr(vvs), al.ctypes.data,
                                  lo.ctypes.data, hi.ctypes.data))
        level, degree = C.c_int32(), C.c_int32()
        flags = [np.zeros(r[k], np.uint8) for k in range(3)]
        _check(lib.fst_model_read_wavelet(self._h, C.byref(level), C.byref(degree), arr(flags)))
        wav = (level.value, degree.value) if level.value >= 0 else None
        return {"r": r, "p": p, "colptr": cps, "rowidx": [ris[k][:nnz[k]] for k in range(3)],
                "val": [vvs[k][:nnz[k]] for k in range(3)], "alpha": al.reshape(r), "lo": lo, "hi": hi,
                "wav": wav, "col_wavelet": [f.astype(bool) for f in flags] if wav else None}

    def host_model(self):
        """The model as a host synth.Model (the form the oracle and fst.Model take)."""
        from . import synth
        d = self.read()
        return synth.Model(d["r"], d["p"], d["colptr"], d["rowidx"], d["val"], d["alpha"], d["lo"], d["hi"],
                           d["wav"], d["col_wavelet"])

    def set_core(self, alpha):
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
        _check(lib.fst_model_set_core(self._h, al.ctypes.data))

    # ---------------------------------------------------------------- evaluation
    def eval(self, xyz, prec: str = "fp32", out=None, stream=None):
        """xyz: CUDA tensor (3, n) float32 (SoA); returns a CUDA float32 tensor (n,)."""
        import torch
        assert xyz.is_cuda and xyz.dtype == torch.float32 and xyz.is_contiguous() and xyz.shape[0] == 3
        n = xyz.shape[1]
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=xyz.device)
        _check(lib.fst_eval(self._h, _dptr(xyz), n, _dptr(out), PREC[prec], _stream(stream)))
        return out

    def prepare(self, prec: str):
        _check(lib.fst_eval_prepare(self._h, PREC[prec]))

    def autotune(self, prec: str, n_probe: int = 1 << 18, stream=None):
        """Measure this model's size class (fst_eval_autotune): returns
        {"ms_cuda_core_factors", "ms_tensor_core_factors", "choice"}."""
        a, b, c = C.c_float(), C.c_float(), C.c_int32()
        _check(lib.fst_eval_autotune(self._h, PREC[prec], int(n_probe), _stream(stream), C.byref(a), C.byref(b),
                                     C.byref(c)))
        return {"ms_cuda_core_factors": a.value, "ms_tensor_core_factors": b.value, "choice": c.value}

    def set_variant(self, prec: str, choice: int):
        """Record the evaluator variant of this model's size class by hand (-1 forgets it)."""
        _check(lib.fst_eval_autotune_set(self._h, PREC[prec], int(choice)))

    def eval_f64(self, xyz, out=None, stream=None):
        import torch
        assert xyz.is_cuda and xyz.dtype == torch.float64 and xyz.is_contiguous() and xyz.shape[0] == 3
        n = xyz.shape[1]
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=xyz.device)
        _check(lib.fst_eval_f64(self._h, _dptr(xyz), n, _dptr(out), _stream(stream)))
        return out

    # ---------------------------------------------------------------- refit
    def refit(self, xyz, u, m: int, seed: int = 0, prec: str = "fp32", idx=None,
              max_refine: int = 32, refine_tol: float = 0.0, fp64_cholesky: bool = False, stream=None):
        """Least-squares core refit over m sampled rows (or the rows in ``idx``).  xyz (3,Q) and u (Q,)
        are CUDA tensors, float32 (or float64 with prec='fp64').  Returns the report as a dict."""
        import torch
        Q = xyz.shape[1]
        opts = RefitOpts(int(max_refine), float(refine_tol), int(bool(fp64_cholesky)))
        rep = RefitReport()
        ip = C.c_void_p(0) if idx is None else _dptr(idx)
        if idx is not None:
            assert idx.is_cuda and idx.dtype == torch.int64
            m = idx.numel()
        if prec == "fp64":
            assert xyz.dtype == torch.float64 and u.dtype == torch.float64
            _check(lib.fst_refit_f64(self._h, _dptr(xyz), _dptr(u), Q, ip, int(m),
                                     C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), C.byref(opts), C.byref(rep),
                                     _stream(stream)))
        else:
            assert xyz.dtype == torch.float32 and u.dtype == torch.float32
            _check(lib.fst_refit(self._h, _dptr(xyz), _dptr(u), Q, ip, int(m),
                                 C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), PREC[prec], C.byref(opts),
                                 C.byref(rep), _stream(stream)))
        return rep.as_dict()


def refit_mixed(model, xyz, u, m: int, seed_signs: int, seed_rows: int, stream=None):
    """fst_refit_mixed: Algorithm 2 with the sign flip and Walsh-Hadamard mixing over all Q rows
    (FP64; xyz (3, Q) and u (Q,) float64 CUDA tensors).  Returns the report as a dict."""
    import torch
    assert xyz.is_cuda and xyz.dtype == torch.float64 and xyz.is_contiguous() and xyz.shape[0] == 3
    assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
    rep = RefitReport()
    _check(lib.fst_refit_mixed(model._h, _dptr(xyz), _dptr(u), xyz.shape[1], int(m),
                               C.c_uint64(seed_signs & 0xFFFFFFFFFFFFFFFF), C.c_uint64(seed_rows & 0xFFFFFFFFFFFFFFFF),
                               C.byref(rep), _stream(stream)))
    return rep.as_dict()


def refit_batched(models, xyzs, us, ms, seeds, prec: str = "bf16", streams: int = 4, max_refine: int = 32,
                  refine_tol: float = 0.0):
    """fst_refit_batched: refit every model on its own points concurrently on `streams` streams.
    Returns the reports (dicts)."""
    import torch
    n = len(models)
    arr = (RefitItem * max(n, 1))()
    for i, (M, x, u, m, sd) in enumerate(zip(models, xyzs, us, ms, seeds)):
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == 3
        assert u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
        arr[i] = RefitItem(M._h, x.data_ptr(), u.data_ptr(), x.shape[1], int(m), int(sd) & 0xFFFFFFFFFFFFFFFF)
    reps = (RefitReport * max(n, 1))()
    opts = RefitOpts(int(max_refine), float(refine_tol), 0)
    torch.cuda.synchronize()     # the library's streams do not wait on the caller's
    _check(lib.fst_refit_batched(arr, n, PREC[prec], C.byref(opts), int(streams), reps))
    return [reps[i].as_dict() for i in range(n)]


class Model4:
    """A device-resident order-4 model (fst_model4) built from a host synth.Model4."""

    def __init__(self, host_model):
        m = host_model
        d = Model4Desc()
        keep = []
        for k in range(4):
            d.r[k] = int(m.r[k])
            d.p[k] = int(m.p[k])
            d.lo[k] = float(m.lo[k])
            d.hi[k] = float(m.hi[k])
            cp = np.ascontiguousarray(m.colptr[k], dtype=np.int32)
            ri = np.ascontiguousarray(m.rowidx[k], dtype=np.int32)
            vv = np.ascontiguousarray(m.val[k], dtype=np.float64)
            if ri.size == 0:
                ri, vv = np.zeros(1, np.int32), np.zeros(1)
            keep += [cp, ri, vv]
            d.colptr[k], d.rowidx[k], d.val[k] = cp.ctypes.data, ri.ctypes.data, vv.ctypes.data
        al = np.ascontiguousarray(np.asarray(m.alpha, dtype=np.float64).reshape(-1))
        keep.append(al)
        d.alpha = al.ctypes.data
        self.r = tuple(int(v) for v in m.r)
        self._h = C.c_void_p()
        _check(lib.fst_model4_create(C.byref(d), C.byref(self._h)))

    def __del__(self):
        try:
            if self._h:
                lib.fst_model4_free(self._h)
                self._h = C.c_void_p()
        except Exception:
            pass

    def core(self):
        a = np.empty(int(np.prod(self.r)))
        _check(lib.fst_model4_read_core(self._h, a.ctypes.data))
        return a.reshape(self.r)

    def eval(self, x, out=None, stream=None):
        """f at the points x (4, n) CUDA tensor, float32 or float64 (the arithmetic follows)."""
        import torch
        assert x.is_cuda and x.is_contiguous() and x.shape[0] == 4
        n = x.shape[1]
        if out is None:
            out = torch.empty(n, device=x.device, dtype=x.dtype)
        fn = lib.fst_eval4_f64 if x.dtype == torch.float64 else lib.fst_eval4
        _check(fn(self._h, _dptr(x), n, _dptr(out), _stream(stream)))
        return out

    def refit(self, x, u, m: int, seed: int = 0, prec: str = "bf16x3", max_refine: int = 200,
              refine_tol: float = 0.0, stream=None):
        """Least-squares core refit over m sampled rows (x (4, Q), u (Q,) float32 CUDA tensors)."""
        import torch
        assert x.dtype == torch.float32 and u.dtype == torch.float32
        opts = RefitOpts(int(max_refine), float(refine_tol), 0)
        rep = RefitReport()
        _check(lib.fst_refit4(self._h, _dptr(x), _dptr(u), x.shape[1], int(m),
                              C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), PREC[prec], C.byref(opts), C.byref(rep),
                              _stream(stream)))
        return rep.as_dict()


def refit_grouped(models, xyzs, us, ms, seeds, prec: str = "bf16", max_refine: int = 32, refine_tol: float = 0.0,
                  fp64_cholesky: bool = False, stream=None):
    """fst_refit_grouped: refit every model on its own points, the factorisations and the
    conjugate gradients of all items in shared launches on one stream.  Returns the reports."""
    import torch
    n = len(models)
    arr = (RefitItem * max(n, 1))()
    for i, (M, x, u, m, sd) in enumerate(zip(models, xyzs, us, ms, seeds)):
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == 3
        assert u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
        arr[i] = RefitItem(M._h, x.data_ptr(), u.data_ptr(), x.shape[1], int(m), int(sd) & 0xFFFFFFFFFFFFFFFF)
    reps = (RefitReport * max(n, 1))()
    opts = RefitOpts(int(max_refine), float(refine_tol), int(bool(fp64_cholesky)))
    _check(lib.fst_refit_grouped(arr, n, PREC[prec], C.byref(opts), reps, _stream(stream)))
    return [reps[i].as_dict() for i in range(n)]


def fit(xyz, u, grid=(32, 32, 32), sample_frac: float = 0.05, eps: float = 1e-3, max_rank=(8, 8, 8),
        max_degree: int = 15, oversample: float = 4.0, seed: int = 1, fixed_rank: bool = False,
        prec: str = "fp32", lo=None, hi=None, grid_values=None, trace: bool = False,
        max_refine: int = 32, refine_tol: float = 0.0, wavelet=None, stream=None):
    """Algorithm 1 and the core refit (fst_fit).  xyz (3, Q) and u (Q,): CUDA float32 tensors.
    wavelet=(s, q) also fits every column in the multiwavelet space W_{s,q} and keeps the better.
    Returns (Model, report dict) or, with trace=True, (Model, report dict, trace dict)."""
    import torch
    assert xyz.is_cuda and xyz.dtype == torch.float32 and xyz.is_contiguous() and xyz.shape[0] == 3
    assert u.is_cuda and u.dtype == torch.float32 and u.is_contiguous()
    Q = xyz.shape[1]
    prm = FitParams()
    for k in range(3):
        prm.grid[k] = int(grid[k])
        prm.max_rank[k] = int(max_rank[k])
    prm.sample_frac, prm.eps, prm.max_degree = float(sample_frac), float(eps), int(max_degree)
    prm.fixed_rank, prm.oversample, prm.seed = int(bool(fixed_rank)), float(oversample), seed & 0xFFFFFFFFFFFFFFFF
    if wavelet is not None:
        prm.wavelet, prm.wav_level, prm.wav_degree = 1, int(wavelet[0]), int(wavelet[1])
    keep = []
    if grid_values is not None:
        gv = np.ascontiguousarray(np.asarray(grid_values, dtype=np.float64).reshape(-1))
        assert gv.size == int(np.prod(grid))
        keep.append(gv)
        prm.grid_values = gv.ctypes.data
    box = []
    for v in (lo, hi):
        if v is None:
            box.append(None)
        else:
            a = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
            keep.append(a)
            box.append(a.ctypes.data)
    opts = RefitOpts(int(max_refine), float(refine_tol), 0)
    rep = FitReport()
    tr, bufs = None, None
    if trace:
        G = [int(g) for g in grid]
        bufs = {"grid_values": np.zeros(G), "eigvals": [np.zeros(g) for g in G],
                "W": [np.zeros(g * int(mr)) for g, mr in zip(G, max_rank)],
                "core_hosvd": np.zeros(int(np.prod(max_rank))), "col_nnz": np.zeros(int(sum(max_rank)), np.int32),
                "col_loo": np.zeros(int(sum(max_rank))), "col_kept": np.zeros(int(sum(max_rank)), np.int32),
                "col_wavelet": np.zeros(int(sum(max_rank)), np.int32), "col_loo_alt": np.zeros(int(sum(max_rank)))}
        tr = FitTrace()
        tr.grid_values = bufs["grid_values"].ctypes.data
        for k in range(3):
            tr.eigvals[k] = bufs["eigvals"][k].ctypes.data
            tr.W[k] = bufs["W"][k].ctypes.data
        tr.core_hosvd = bufs["core_hosvd"].ctypes.data
        tr.col_nnz = bufs["col_nnz"].ctypes.data
        tr.col_loo = bufs["col_loo"].ctypes.data
        tr.col_kept = bufs["col_kept"].ctypes.data
        tr.col_wavelet = bufs["col_wavelet"].ctypes.data
        tr.col_loo_alt = bufs["col_loo_alt"].ctypes.data
    h = C.c_void_p()
    _check(lib.fst_fit(_dptr(xyz), _dptr(u), Q, box[0], box[1], C.byref(prm), PREC[prec], C.byref(opts),
                       C.byref(tr) if tr is not None else None, C.byref(rep), C.byref(h), _stream(stream)))
    model = Model(_handle=h)
    d = rep.as_dict()
    if not trace:
        return model, d
    r = d["r_hosvd"]
    ncol = sum(r)
    t = {"grid_values": bufs["grid_values"], "eigvals": bufs["eigvals"],
         "W": [bufs["W"][k][:G[k] * r[k]].reshape(G[k], r[k]) for k in range(3)],
         "core_hosvd": bufs["core_hosvd"][:r[0] * r[1] * r[2]].reshape(r),
         "col_nnz": bufs["col_nnz"][:ncol].copy(), "col_loo": bufs["col_loo"][:ncol].copy(),
         "col_kept": bufs["col_kept"][:ncol].copy(), "col_wavelet": bufs["col_wavelet"][:ncol].copy(),
         "col_loo_alt": bufs["col_loo_alt"][:ncol].copy()}
    return model, d, t


def cholesky_f32(G, stream=None):
    """In-place lower Cholesky factor of a CUDA float32 (R, R) SPD matrix (fst_cholesky_f32)."""
    import torch
    assert G.is_cuda and G.dtype == torch.float32 and G.is_contiguous() and G.dim() == 2
    assert G.shape[0] == G.shape[1]
    _check(lib.fst_cholesky_f32(_dptr(G), int(G.shape[0]), _stream(stream)))
    return G


def normal_matrix(model: "Model", xyz, u, idx, prec: str = "tf32", with_h: bool = True, stream=None):
    """G = A^T A (lower triangle valid) and h = A^T b over the rows idx, as CUDA tensors."""
    import torch
    r, _, _ = model.shape()
    R = r[0] * r[1] * r[2]
    G = torch.zeros((R, R), dtype=torch.float32, device=xyz.device)
    h = torch.zeros(R, dtype=torch.float64, device=xyz.device) if with_h else None
    _check(lib.fst_normal_matrix(model.handle, _dptr(xyz), _dptr(u), xyz.shape[1], _dptr(idx), idx.numel(),
                                 PREC[prec], _dptr(G), _dptr(h) if h is not None else C.c_void_p(0),
                                 _stream(stream)))
    return G, h


def sample_rows(seed: int, Q: int, m: int, device="cuda", stream=None):
    import torch
    m = min(int(m), int(Q))
    idx = torch.empty(m, dtype=torch.int64, device=device)
    _check(lib.fst_sample_rows(C.c_uint64(seed & 0xFFFFFFFFFFFFFFFF), int(Q), m, _dptr(idx),
                               _stream(stream)))
    return idx


def eval_batched(models, xyzs, outs=None, prec: str = "bf16x3", stream=None):
    """Evaluate model i at points xyzs[i] (CUDA (3, n_i) float32) for all i in one launch."""
    import torch
    if outs is None:
        outs = [torch.empty(x.shape[1], dtype=torch.float32, device=x.device) for x in xyzs]
    arr = (EvalItem * len(models))()
    for i, (m, x, o) in enumerate(zip(models, xyzs, outs)):
        assert x.is_cuda and x.dtype == torch.float32 and x.is_contiguous() and x.shape[0] == 3
        arr[i] = EvalItem(m.handle.value, x.data_ptr(), x.shape[1], o.data_ptr())
    _check(lib.fst_eval_batched(arr, len(models), PREC[prec], _stream(stream)))
    return outs


class EvalPlan:
    """A prepared batch: plan.run(stream) launches only (capturable in a CUDA graph)."""

    def __init__(self, models, xyzs, outs, prec: str = "bf16x3"):
        self._keep = (list(models), list(xyzs), list(outs))
        arr = (EvalItem * len(models))()
        for i, (m, x, o) in enumerate(zip(models, xyzs, outs)):
            arr[i] = EvalItem(m.handle.value, x.data_ptr(), x.shape[1], o.data_ptr())
        self._h = C.c_void_p()
        _check(lib.fst_eval_plan_create(arr, len(models), PREC[prec], C.byref(self._h)))

    def run(self, stream=None):
        _check(lib.fst_eval_plan_run(self._h, _stream(stream)))

    def free(self):
        if self._h:
            lib.fst_eval_plan_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def slice_points(axis: int, value: float, lo, hi, res0: int, res1: int, out=None, device="cuda", stream=None):
    """Points of the slice y_axis = value as a CUDA (3, res0*res1) float32 tensor."""
    import torch
    if out is None:
        out = torch.empty((3, res0 * res1), dtype=torch.float32, device=device)
    lo_a = (C.c_double * 3)(*[float(v) for v in lo])
    hi_a = (C.c_double * 3)(*[float(v) for v in hi])
    _check(lib.fst_slice_points(int(axis), float(value), lo_a, hi_a, int(res0), int(res1), _dptr(out),
                                _stream(stream)))
    return out


def eval_check(stream=None):
    _check(lib.fst_eval_check(_stream(stream)))


def set_wait_limit(cycles: int = 0):
    """fst_set_wait_limit: budget of the triangular solves' bounded waits (0: the default)."""
    _check(lib.fst_set_wait_limit(int(cycles)))


def kernel_launches() -> int:
    return int(lib.fst_kernel_launches())


def build_info() -> str:
    return lib.fst_build_info().decode()
