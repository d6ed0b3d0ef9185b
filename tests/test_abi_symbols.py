"""The C-ABI library loads on a machine without a GPU and exports every entry point that
include/fst.h declares; the header has plain C types only."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared():
    text = (ROOT / "include" / "fst.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fst_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libfst():
    from paper_1907_05884_gb300 import build
    return ctypes.CDLL(str(build.build()))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("fst_model_create", "fst_eval", "fst_eval_f64", "fst_refit", "fst_refit_f64",
                 "fst_sample_rows", "fst_model_save", "fst_model_load", "fst_status_str"):
        assert must in names


def test_every_declared_symbol_is_exported(libfst):
    missing = [n for n in _declared() if not hasattr(libfst, n)]
    assert not missing, missing


def test_header_has_no_torch_types():
    text = (ROOT / "include" / "fst.h").read_text()
    for bad in ("torch", "at::", "c10::", "#include <ATen", "PyObject"):
        assert bad not in text


def test_status_strings_without_gpu(libfst):
    libfst.fst_status_str.restype = ctypes.c_char_p
    assert libfst.fst_status_str(0) == b"ok"
    assert b"not positive definite" in libfst.fst_status_str(-4)


def test_binding_loads(libfst):
    from paper_1907_05884_gb300 import fst
    assert "sm_103a" in fst.build_info()
