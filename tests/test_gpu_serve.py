"""The continuous-batching server: every query's result equals the same query served alone,
queries that arrive while others run are admitted into later launches that overlap them, and
admission never exceeds the device-memory budget."""
import numpy as np
import pytest

from paper_1907_05884_gb300 import synth
from gpu_util import EVAL_TOL, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst, serve
    rng = np.random.default_rng(1)
    host_models = [synth.random_model(tuple(int(v) for v in rng.integers(4, 25, size=3)), (31, 31, 31),
                                      seed=100 + i, density=0.6) for i in range(8)]
    models = [fst.Model(m) for m in host_models]
    pool = torch.from_numpy(synth.points(1 << 20, seed=2, clustered=0.3).astype(np.float32)).pin_memory()
    return fst, serve, host_models, models, pool


def test_results_same_alone_and_in_the_mix(setup, oracle_lib):
    import torch
    fst, serve, host_models, models, pool = setup
    srv = serve.FieldServer(models, pool, mem_budget=64 << 20, streams=2, keep_results=True)
    srv.prepare(("bf16x3", "bf16"))
    qs = serve.make_queries(160, len(models), rate_qps=20000.0, seed=3, precs=("fp32", "bf16", "bf16x3"),
                            pool_points=pool.shape[1], slice_res=(32, 256), point_range=(1e2, 2e5))
    srv.run(qs)
    torch.cuda.synchronize()
    assert all(np.isfinite(q.t_done) for q in qs)
    assert srv.peak_mem <= 64 << 20
    launches_with_many = 0
    for q in qs:
        M = models[q.field]
        if q.kind == "slice":
            lo, hi = srv.boxes[q.field]
            xyz = fst.slice_points(q.axis, q.value, lo, hi, q.res, q.res)
        else:
            xyz = pool[:, q.p0:q.p0 + q.n].cuda()
        alone = M.eval(xyz.contiguous(), prec=q.prec)
        assert torch.equal(alone, q.out), (q.qid, q.kind, q.prec)
    # a few against the FP64 oracle
    for q in qs[:6]:
        if q.kind != "points":
            continue
        ref = oracle_lib.eval_points(host_models[q.field], pool[:, q.p0:q.p0 + q.n].numpy().astype(np.float64))
        tol = EVAL_TOL[q.prec]
        assert rel_l2(q.out.cpu().numpy(), ref) < tol


def test_slice_points_grid(setup):
    import torch
    fst, serve, _, models, _ = setup
    xyz = fst.slice_points(1, 0.25, [-1, -2, -3], [1, 2, 3], 5, 7).cpu().numpy()
    assert np.all(xyz[1] == np.float32(0.25))
    assert np.allclose(xyz[0].reshape(5, 7)[:, 0], np.linspace(-1, 1, 5))
    assert np.allclose(xyz[2].reshape(5, 7)[0], np.linspace(-3, 3, 7))


def test_oversize_query_admitted_alone(setup):
    import torch
    fst, serve, _, models, pool = setup
    srv = serve.FieldServer(models, pool, mem_budget=1 << 20, streams=2, keep_results=True)
    qs = serve.make_queries(6, len(models), rate_qps=0.0, seed=5, precs=("bf16x3",), pool_points=pool.shape[1],
                            slice_res=(300, 400), point_range=(1e5, 2e5))
    srv.run(qs)
    torch.cuda.synchronize()
    assert all(np.isfinite(q.t_done) for q in qs)


def test_fp32_queries_served_by_bf16x3(setup, oracle_lib):
    """With fp32_via="bf16x3" the queries asking for FP32 accuracy run the BF16x3 evaluator:
    each result equals that evaluator alone and meets the FP32 bound against the oracle."""
    import torch
    fst, serve, host_models, models, pool = setup
    srv = serve.FieldServer(models, pool, mem_budget=64 << 20, streams=2, keep_results=True, fp32_via="bf16x3")
    srv.prepare(("bf16x3", "bf16"))
    qs = serve.make_queries(60, len(models), rate_qps=20000.0, seed=7, precs=("fp32", "bf16"),
                            pool_points=pool.shape[1], slice_res=(32, 128), point_range=(1e2, 1e5))
    srv.run(qs)
    torch.cuda.synchronize()
    checked = 0
    for q in qs:
        if q.kind != "points":
            continue
        x = pool[:, q.p0:q.p0 + q.n].cuda().contiguous()
        want = "bf16x3" if q.prec == "fp32" else q.prec
        assert torch.equal(models[q.field].eval(x, prec=want), q.out), q.qid
        if q.prec == "fp32" and checked < 4:
            ref = oracle_lib.eval_points(host_models[q.field], pool[:, q.p0:q.p0 + q.n].numpy().astype(np.float64))
            assert rel_l2(q.out.cpu().numpy(), ref) < EVAL_TOL["fp32"]
            checked += 1
    assert checked > 0
