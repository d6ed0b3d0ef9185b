"""Argument checks of the C ABI that happen before any device call, so they run on a machine
without a GPU: bad pointers and sizes come back as FST_EINVAL with a message, never a crash."""
import ctypes as C

import pytest

EINVAL = -1


@pytest.fixture(scope="module")
def lib():
    from paper_1907_05884_gb300 import build
    L = C.CDLL(str(build.build()))
    L.fst_last_error.restype = C.c_char_p
    return L


def _err(lib):
    return lib.fst_last_error().decode()


def test_refit_mixed_rejects_null_and_sizes(lib):
    f = lib.fst_refit_mixed
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int64, C.c_uint64, C.c_uint64, C.c_void_p,
                  C.c_void_p]
    assert f(None, None, None, 100, 10, 1, 2, None, None) == EINVAL
    assert "NULL" in _err(lib)


def test_refit_batched_checks_items_and_streams(lib):
    f = lib.fst_refit_batched
    f.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p]
    # an empty batch is a no-op, with or without items
    assert f(None, 0, 3, None, 4, None) == 0
    # items missing, a bad precision, a bad stream count
    assert f(None, 2, 3, None, 4, None) == EINVAL
    items = (C.c_uint8 * 256)()
    assert f(items, 1, 0, None, 4, None) == EINVAL        # FP64 is not a batched-refit precision
    assert f(items, 1, 3, None, 0, None) == EINVAL
    assert f(items, 1, 3, None, 65, None) == EINVAL
    assert "streams" in _err(lib)


def test_sample_rows_rejects_negative_sizes(lib):
    f = lib.fst_sample_rows
    f.argtypes = [C.c_uint64, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p]
    assert f(1, -5, 3, None, None) == EINVAL
    assert f(1, 10, -3, None, None) == EINVAL
    # nothing to draw is a no-op
    assert f(1, 0, 0, None, None) == 0


def test_refit_rejects_null_model(lib):
    f = lib.fst_refit
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_uint64, C.c_int32,
                  C.c_void_p, C.c_void_p, C.c_void_p]
    assert f(None, None, None, 100, None, 10, 0, 3, None, None, None) == EINVAL
