"""fst_sample_rows_static, the sampler variant for callers that cannot allocate device
memory (an in-situ hook inside a simulation whose pool owns the device memory, or a
latency-bound loop that cannot absorb cudaMalloc's implicit synchronisation).

It is called here through the C ABI and must return exactly the rows of the
allocating fst_sample_rows, on two calls in a row (a large call, then a smaller one
with another seed, so stale state from the first call would show), and reject row
counts beyond its fixed scratch with FST_EINVAL.  This file is collected last.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def _static_rows(F, seed, Q, m):
    import torch
    idx = torch.full((m,), -1, dtype=torch.int64, device="cuda")
    st = F.lib.fst_sample_rows_static(C.c_uint64(seed), Q, m, F._dptr(idx), F._stream())
    F._check(st)
    torch.cuda.synchronize()
    return idx


def test_static_sampler_matches_allocating_sampler_twice(F):
    import torch
    for seed, Q, m in [(0xA11CE, 3_000_017, 110_592), (42, 70_001, 999)]:
        got = _static_rows(F, seed, Q, m)
        ref = F.sample_rows(seed, Q, m)
        torch.cuda.synchronize()
        assert torch.equal(got, ref)


def test_static_sampler_rejects_rows_beyond_its_scratch(F):
    import torch
    idx = torch.empty(16, dtype=torch.int64, device="cuda")
    st = F.lib.fst_sample_rows_static(C.c_uint64(1), (1 << 29) + 1, 16, F._dptr(idx), F._stream())
    assert st == -1
    assert b"at most" in F.lib.fst_last_error()
