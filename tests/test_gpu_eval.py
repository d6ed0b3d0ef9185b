"""Parity of the CUDA evaluation (fst_eval / fst_eval_f64) with the FP64 oracle
(Sec. 2, eq. func_tuck; Sec. 6, reconstruction by basis evaluation)."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import rel_l2, cuda_tensor

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available()
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst
    return fst


CASES = [
    # ranks, degrees, density, n
    ((1, 1, 1), (0, 0, 0), 1.0, 1),
    ((1, 1, 1), (5, 3, 7), 1.0, 127),
    ((3, 4, 5), (7, 6, 8), 0.6, 128),
    ((8, 8, 8), (15, 15, 15), 0.5, 129),
    ((5, 9, 2), (11, 4, 13), 0.7, 1009),
    ((16, 12, 20), (31, 31, 31), 0.5, 4099),
    ((24, 24, 24), (31, 31, 31), 0.6, 3001),
    ((32, 7, 32), (63, 20, 63), 0.3, 2048),
]


@pytest.mark.parametrize("r,p,dens,n", CASES)
def test_eval_fp64_and_fp32_match_oracle(F, oracle_lib, r, p, dens, n):
    import torch
    m = synth.random_model(r, p, seed=sum(r) * 7 + n, density=dens)
    xyz = synth.points(n, seed=n + 1)
    ref = oracle_lib.eval_points(m, xyz, nthreads=4)
    M = F.Model(m)
    got64 = M.eval_f64(cuda_tensor(xyz, torch.float64)).cpu().numpy()
    assert rel_l2(got64, ref) < TOL_FP64
    got32 = M.eval(cuda_tensor(xyz, torch.float32)).cpu().numpy()
    ref32 = oracle_lib.eval_points(m, xyz.astype(np.float32).astype(np.float64), nthreads=4)
    assert rel_l2(got32, ref32) < TOL_FP32


def test_eval_box_and_extrapolation(F, oracle_lib):
    import torch
    lo, hi = np.array([0.0, -2.0, 10.0]), np.array([1.0, 2.0, 10.5])
    m = synth.random_model((4, 5, 3), (9, 6, 7), seed=5, lo=lo, hi=hi)
    t = synth.points(777, seed=6) * 1.1          # 10% outside the box: polynomial extrapolation
    y = lo[:, None] + (t + 1) / 2 * (hi - lo)[:, None]
    ref = oracle_lib.eval_points(m, y)
    got = F.Model(m).eval_f64(cuda_tensor(y, torch.float64)).cpu().numpy()
    assert rel_l2(got, ref) < TOL_FP64


def test_eval_empty_and_errors(F):
    import torch
    m = synth.random_model((2, 2, 2), (3, 3, 3), seed=1)
    M = F.Model(m)
    x = torch.empty((3, 0), device="cuda", dtype=torch.float32)
    assert M.eval(x).numel() == 0
    host = torch.zeros((3, 4), dtype=torch.float32)
    with pytest.raises(F.FstError) as e:
        F._check(F.lib.fst_eval(M.handle, F._dptr(host), 4, F._dptr(host), F.FST_FP32, F._stream()))
    assert e.value.status == -1


def test_model_validation_and_roundtrip(F, tmp_path):
    m = synth.random_model((3, 2, 4), (5, 9, 2), seed=9, density=0.5)
    M = F.Model(m)
    path = tmp_path / "m.fstm"
    M.save(str(path))
    M2 = F.Model.load(str(path))
    a, b = M.read(), M2.read()
    for k in range(3):
        assert np.array_equal(a["colptr"][k], b["colptr"][k])
        assert np.array_equal(a["rowidx"][k], b["rowidx"][k])
        assert np.array_equal(a["val"][k], b["val"][k])
        assert np.array_equal(a["colptr"][k], m.colptr[k])
    assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["alpha"], m.alpha)
    bad = synth.random_model((3, 2, 4), (5, 9, 2), seed=9)
    bad.rowidx[0] = bad.rowidx[0].copy()
    bad.rowidx[0][0] = 99                          # degree above p
    with pytest.raises(F.FstError) as e:
        F.Model(bad)
    assert e.value.status == -1
    (tmp_path / "junk.fstm").write_bytes(b"NOPE" + bytes(20))
    with pytest.raises(F.FstError) as e:
        F.Model.load(str(tmp_path / "junk.fstm"))
    assert e.value.status == -7


def test_eval_full_size_sampled(F, oracle_lib):
    """2^24 points, ranks 24^3, degree 31 (the 16M-point FP32 workload), evaluated in one
    launch; 4096 sampled outputs compared with the oracle."""
    import torch
    n = 1 << 24
    m = synth.random_model((24, 24, 24), (31, 31, 31), seed=202, density=0.6)
    xyz = synth.points(n, seed=203, clustered=0.3, dtype=np.float32)
    M = F.Model(m)
    got = M.eval(cuda_tensor(xyz, torch.float32)).cpu().numpy()
    sel = np.random.default_rng(0).choice(n, 4096, replace=False)
    ref = oracle_lib.eval_points(m, xyz[:, sel].astype(np.float64), nthreads=8)
    assert rel_l2(got[sel], ref) < TOL_FP32
