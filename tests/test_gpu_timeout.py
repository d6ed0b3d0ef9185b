"""The expiry path of the bounded device waits: with the triangular solves' wait budget cut to
a few clock cycles (fst_set_wait_limit), a refit's solve blocks give up on values their
predecessors have not published, the refit reports FST_ETIMEOUT and leaves the model as it
was, and the next refit with the default budget succeeds in the same process."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import cuda_tensor

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


def test_solve_wait_expiry_reports_timeout(F, oracle_lib):
    import torch
    # R = 4,096: 64 block rows in each triangular solve, so later rows wait on earlier ones
    model = synth.random_model((16, 16, 16), (23, 23, 23), seed=61, orthonormal=True)
    Q = 60000
    xyz = synth.points(Q, seed=62).astype(np.float32)
    u, _ = synth.field_values(xyz, synth.field_spec(63, 4), seed=64)
    xt, ut = cuda_tensor(xyz, torch.float32), cuda_tensor(u.astype(np.float32), torch.float32)
    mm = 4 * model.R
    M = F.Model(model)
    try:
        F.set_wait_limit(2)
        with pytest.raises(F.FstError) as e:
            M.refit(xt, ut, mm, seed=65, prec="bf16")
        assert e.value.status == -6, e.value
    finally:
        F.set_wait_limit(0)
    assert np.array_equal(M.read()["alpha"], model.alpha)     # the failed refit changed nothing
    # the context is usable: the same refit with the default budget solves the normal equations
    rep = M.refit(xt, ut, mm, seed=65, prec="bf16")
    idx = oracle_lib.sample(65, Q, mm)
    alpha = M.read()["alpha"].reshape(-1)
    x64, u64 = xyz.astype(np.float64), u.astype(np.float32).astype(np.float64)
    g = oracle_lib.normal_residual(model, x64, u64, idx, alpha, nthreads=oracle_lib.default_threads())
    h = oracle_lib.normal_residual(model, x64, u64, idx, np.zeros(model.R), nthreads=oracle_lib.default_threads())
    assert np.linalg.norm(g) < 1e-5 * np.linalg.norm(h), rep
    with pytest.raises(F.FstError):
        F.set_wait_limit(-1)
