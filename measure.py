"""Run one libfst entry point on seeded synthetic inputs, for timing and profiling (the
commands the summaries under profiles/ were made with).

    python measure.py gram  --prec bf16   --m 16384
    python measure.py eval  --prec bf16x3 --n 4194304
    python measure.py refit --prec bf16   --n 1048576
    python measure.py chol  --m 110592

The model has ranks 24^3 and Legendre degree 31 with orthonormal factor functions (unless
--ranks/--degree say otherwise); each call is repeated --reps times and timed with CUDA events.
"""
from __future__ import annotations

import argparse
import sys
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parent))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["gram", "eval", "refit", "sample", "batch", "serve", "fit", "chol",
                                     "refit-batch", "mixed", "order4"])
    ap.add_argument("--grid", type=int, default=64)
    ap.add_argument("--frac", type=float, default=0.05)
    ap.add_argument("--eps", type=float, default=1e-3)
    ap.add_argument("--queries", type=int, default=2000)
    ap.add_argument("--q-lo", type=float, default=1e5)
    ap.add_argument("--q-hi", type=float, default=2e6)
    ap.add_argument("--instances", type=int, default=512)
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--ranks", type=int, nargs=3, default=[24, 24, 24])
    ap.add_argument("--degree", type=int, default=31)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--streams", type=int, nargs="*", default=[1, 2, 4, 8])
    ap.add_argument("--grouped-only", action="store_true", help="refit-batch: time fst_refit_grouped alone")
    ap.add_argument("--variant", type=int, default=-1,
                    help="evaluator variant (0: factor values on the CUDA cores, 1: on the tensor cores); "
                         "default: autotuned")
    args = ap.parse_args()

    import torch
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst, synth

    if args.what == "batch":
        return batch(args)
    if args.what == "refit-batch":
        return refit_batch(args)
    if args.what == "mixed":
        return mixed(args)
    if args.what == "serve":
        return serve_loads(args)
    if args.what == "fit":
        return fit(args)
    if args.what == "order4":
        return order4(args)
    model = synth.random_model(tuple(args.ranks), (args.degree,) * 3, seed=4, orthonormal=True)
    M = fst.Model(model)
    Q = max(args.n, 2 * args.m)
    xyz = torch.from_numpy(synth.points(Q, seed=5, clustered=0.3).astype(np.float32)).cuda()
    u_np, _ = synth.field_values(xyz.cpu().numpy(), synth.field_spec(6, 20), seed=7)
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    out = torch.empty(Q, device="cuda")
    idx = fst.sample_rows(8, Q, args.m)
    if args.what == "eval" and args.prec != "fp32":
        if args.variant >= 0:
            M.set_variant(args.prec, args.variant)
        M.prepare(args.prec)
    for r in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        extra = ""
        if args.what == "gram":
            fst.normal_matrix(M, xyz, u, idx, prec=args.prec, with_h=False)
        elif args.what == "eval":
            M.eval(xyz[:, :args.n].contiguous() if Q != args.n else xyz, prec=args.prec, out=out[:args.n])
        elif args.what == "chol":
            # G = A^T A of the sampled rows (BF16 Gram), then the FP32 factorisation alone
            G, _ = fst.normal_matrix(M, xyz, u, idx, prec="bf16", with_h=False)
            torch.cuda.synchronize()
            e0.record()
            fst.cholesky_f32(G)
        elif args.what == "refit":
            rep = M.refit(xyz, u, args.m, seed=9, prec=args.prec)
            extra = f" {rep}"
        else:
            fst.sample_rows(10 + r, Q, args.m)
        e1.record()
        torch.cuda.synchronize()
        print(f"{args.what} prec={args.prec} m={args.m} n={args.n} ms={e0.elapsed_time(e1):.3f}{extra}", flush=True)


def batch(args):
    """Batched-evaluation workload: instances (fields x timesteps) with ranks U{4..24} per mode
    and point counts log-uniform in [1e5, 2e6]; one fst_eval_batched launch against one
    fst_eval launch per instance."""
    import torch
    from paper_1907_05884_gb300 import fst, synth
    table = synth.batch_instances(n_fields=max(1, args.instances // 8), n_steps=8, q_lo=args.q_lo,
                                  q_hi=args.q_hi)[:args.instances]
    models, xs, outs = [], [], []
    for k, inst in enumerate(table):
        m = synth.random_model(inst["r"], (args.degree,) * 3, seed=inst["seed"] % (1 << 31), density=0.6)
        models.append(fst.Model(m))
        x = torch.rand((3, inst["Q"]), device="cuda", generator=None) * 2 - 1
        xs.append(x.contiguous())
        outs.append(torch.empty(inst["Q"], device="cuda"))
        models[-1].prepare(args.prec)
    total = sum(x.shape[1] for x in xs)
    plan = fst.EvalPlan(models, xs, outs, prec=args.prec)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.run()
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(graph):
        plan.run()
    for Mi, x, o in zip(models, xs, outs):       # single-instance work lists built before timing
        Mi.eval(x, prec=args.prec, out=o)
    torch.cuda.synchronize()
    for r in range(args.reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        plan.run()
        ev[1].record()
        graph.replay()
        ev[2].record()
        for Mi, x, o in zip(models, xs, outs):
            Mi.eval(x, prec=args.prec, out=o)
        ev[3].record()
        torch.cuda.synchronize()
        tp, tg, ts = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])
        print(f"batch instances={len(models)} points={total} prec={args.prec} "
              f"plan_ms={tp:.3f} ({total / tp / 1e3:.1f} Mpoints/s) graph_ms={tg:.3f} "
              f"({total / tg / 1e3:.1f} Mpoints/s) per_instance_ms={ts:.3f} ({total / ts / 1e3:.1f} Mpoints/s)",
              flush=True)


def refit_batch(args):
    """Batched refits over the batching workload's instances (ranks U{4..24} per mode, point
    counts log-uniform in [--q-lo, --q-hi], m = 8R rows each): one fst_refit_batched call on S
    streams and one fst_refit_grouped call against one fst_refit per instance, one after
    another."""
    import time
    import torch
    from paper_1907_05884_gb300 import fst, synth
    table = synth.batch_instances(n_fields=max(1, args.instances // 8), n_steps=8, q_lo=args.q_lo,
                                  q_hi=args.q_hi)[:args.instances]
    models, xs, us, ms, seeds = [], [], [], [], []
    g = torch.Generator(device="cuda")
    g.manual_seed(11)
    for inst in table:
        m = synth.random_model(inst["r"], (args.degree,) * 3, seed=inst["seed"] % (1 << 31), density=0.6,
                               orthonormal=True)
        models.append(fst.Model(m))
        x = torch.rand((3, inst["Q"]), device="cuda", generator=g) * 2 - 1
        xs.append(x.contiguous())
        # a smooth synthetic field of the coordinates
        us.append((torch.exp(-2 * (x * x).sum(0)) + 0.3 * torch.sin(3 * x[0]) * x[1]).contiguous())
        ms.append(min(8 * m.R, inst["Q"]))
        seeds.append(inst["seed"])
    rows = sum(ms)
    torch.cuda.synchronize()
    for r in range(args.reps):
        line = f"refit-batch instances={len(models)} rows={rows} prec={args.prec}"
        if not args.grouped_only:
            # wall-clock on both sides: the batched call runs on several streams of its own
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            reps = [Mi.refit(x, u, mm, seed=sd, prec=args.prec)
                    for Mi, x, u, mm, sd in zip(models, xs, us, ms, seeds)]
            torch.cuda.synchronize()
            seq = (time.perf_counter() - h0) * 1e3
            phases = {k: sum(rp[k] for rp in reps) for k in ("ms_sample", "ms_factors", "ms_gram", "ms_cholesky",
                                                              "ms_refine")}
            line += f" sequential_ms={seq:.2f} " + " ".join(f"{k}={v:.1f}" for k, v in phases.items())
        for S in ([] if args.grouped_only else args.streams):
            torch.cuda.synchronize()
            h0 = time.perf_counter()
            fst.refit_batched(models, xs, us, ms, seeds, prec=args.prec, streams=S)
            torch.cuda.synchronize()
            line += f" streams{S}_ms={(time.perf_counter() - h0) * 1e3:.2f}"
        torch.cuda.synchronize()
        h0 = time.perf_counter()
        greps = fst.refit_grouped(models, xs, us, ms, seeds, prec=args.prec)
        torch.cuda.synchronize()
        line += (f" grouped_ms={(time.perf_counter() - h0) * 1e3:.2f} grouped_rows_gram_ms={greps[0]['ms_gram']:.1f}"
                 f" grouped_cholesky_ms={greps[0]['ms_cholesky']:.1f} grouped_refine_ms={greps[0]['ms_refine']:.1f}"
                 f" grouped_steps_max={max(rp['refine_steps'] for rp in greps)}")
        print(line, flush=True)


def order4(args):
    """Order-4 models at the paper's SP4D ranks 30 x 38 x 5 x 11 (R = 62,700; degrees 40, 40,
    15, 20, orthonormal factor functions): evaluation at --n points in FP32 and FP64, and the
    core refit on m = 4R rows of 2^19 points (values of the model itself)."""
    import torch
    from paper_1907_05884_gb300 import fst, synth
    m = synth.random_model4((30, 38, 5, 11), (40, 40, 15, 20), seed=77, orthonormal=True)
    M = fst.Model4(m)
    x = torch.from_numpy(synth.points4(args.n, seed=78).astype(np.float32)).cuda()
    x64 = x.double()
    for r in range(args.reps):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record()
        M.eval(x)
        e[1].record()
        M.eval(x64)
        e[2].record()
        torch.cuda.synchronize()
        t32, t64 = e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])
        print(f"order4 eval n={args.n} R={m.R} fp32_ms={t32:.3f} ({args.n / t32 / 1e3:.1f} Mpoints/s, "
              f"{2 * m.R * args.n / t32 / 1e9:.1f} TFLOP/s of contraction) fp64_ms={t64:.3f}", flush=True)
    Q = 1 << 19
    xr = synth.points4(Q, seed=79)
    u = M.eval(torch.from_numpy(xr).cuda()).float().contiguous()
    xr32 = torch.from_numpy(xr.astype(np.float32)).cuda()
    for r in range(args.reps):
        M0 = fst.Model4(m.with_alpha(np.zeros(m.r)))
        torch.cuda.synchronize()
        rep = M0.refit(xr32, u, 4 * m.R, seed=80, prec=args.prec, max_refine=200)
        err = np.linalg.norm(M0.core() - m.alpha) / np.linalg.norm(m.alpha)
        print(f"order4 refit R={m.R} m={4 * m.R} prec={args.prec} {rep} core_rel_l2={err:.3e}", flush=True)


def mixed(args):
    """Algorithm 2 with and without its mixing step (Sec. 5; configuration-1 scale): --n points
    (default 20,000; 90 % clustered in the band, so plain uniform sampling over-weights it) of a
    sum of Gaussians, an orthonormal model of ranks --ranks (default 8^3) and degree --degree
    (default 15).  For each m: the refit on m rows with mixing (fst_refit_mixed) and without
    (fst_refit_f64 on m uniformly sampled points), and the change of the core when m grows by
    R / 4 (the self-convergence of Fig. 5), each timed with CUDA events."""
    import json
    import torch
    from paper_1907_05884_gb300 import fst, synth
    Q = args.n if args.n != (1 << 22) else 20000
    ranks = tuple(args.ranks) if tuple(args.ranks) != (24, 24, 24) else (8, 8, 8)
    deg = args.degree if args.degree != 31 else 15
    model = synth.random_model(ranks, (deg,) * 3, seed=51, density=0.8, orthonormal=True)
    xyz_np = synth.points(Q, seed=52, clustered=0.9)
    u_np, _ = synth.field_values(xyz_np, synth.field_spec(53, 5), seed=54)
    xyz = torch.from_numpy(xyz_np).cuda()
    u = torch.from_numpy(u_np).cuda()
    R = model.R
    M = fst.Model(model)
    N = 1
    while N < Q:
        N *= 2
    for mult in (1.25, 1.5, 2.0, 3.0, 4.0, 6.0, 8.0):
        m1 = int(mult * R)
        m2 = m1 + R // 4
        if m2 > min(Q, N):
            break
        line = {"what": "mixed", "Q": Q, "N": N, "R": R, "m": m1}
        for name, call in (("mixed", lambda mm: fst.refit_mixed(M, xyz, u, mm, 61, 62)),
                           ("plain", lambda mm: M.refit(xyz, u, mm, seed=62, prec="fp64"))):
            cores = []
            for mm in (m1, m2):
                M.set_core(model.alpha)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                call(mm)
                e1.record()
                torch.cuda.synchronize()
                if mm == m1:
                    line[f"{name}_ms"] = e0.elapsed_time(e1)
                cores.append(M.read()["alpha"].ravel())
            line[f"{name}_self_change"] = float(np.linalg.norm(cores[1] - cores[0]) / np.linalg.norm(cores[1]))
        print(json.dumps(line), flush=True)


def fit(args):
    """Construction workload: --n scattered points (70% uniform, 30% in a band) of a sum of
    20 Gaussians plus noise; grid --grid^3, rank caps --ranks, degree --degree, a --frac
    subset interpolated, refit on ceil(8 R) rows in --prec."""
    import json
    import torch
    from paper_1907_05884_gb300 import fst, synth
    xyz_np = synth.points(args.n, seed=5, clustered=0.3).astype(np.float32)
    u_np, _ = synth.field_values(xyz_np.astype(np.float64), synth.field_spec(6, 20), seed=7)
    xyz = torch.from_numpy(xyz_np).cuda()
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    for r in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        M, rep = fst.fit(xyz, u, grid=(args.grid,) * 3, sample_frac=args.frac, eps=args.eps,
                         max_rank=tuple(args.ranks), max_degree=args.degree, oversample=8.0, seed=11 + r,
                         prec=args.prec)
        e1.record()
        torch.cuda.synchronize()
        ref = u[:1 << 20]
        pred = M.eval(xyz[:, :1 << 20].contiguous(), prec="fp32")
        rel = float(torch.linalg.norm(pred - ref) / torch.linalg.norm(ref))
        print(json.dumps({"fit_ms": e0.elapsed_time(e1), "rel_l2_first_1M": rel, **{
            k: v for k, v in rep.items() if k != "refit"}, "refit": {k: rep["refit"][k] for k in (
                "refine_steps", "ms_gram", "ms_cholesky", "ms_refine", "fallback_bf16x3", "shifted_preconditioner",
                "fallback_fp64")}}), flush=True)


def serve_loads(args):
    """Serving workload: 64 resident fields (ranks <= 24, degree 31); Poisson queries, half
    slices (side 512..2048), half point sets (1e3..1e7 points); precision 50/50 FP32/BF16.
    Saturation throughput from a closed run, then offered loads of 25/50/75/90% of it."""
    import json
    import torch
    from paper_1907_05884_gb300 import fst, serve, synth
    rng = np.random.default_rng(11)
    models = [fst.Model(synth.random_model(tuple(int(v) for v in rng.integers(4, 25, size=3)),
                                           (args.degree,) * 3, seed=200 + i, density=0.6)) for i in range(64)]
    pool = torch.from_numpy(synth.points(10_000_000, seed=12, clustered=0.3).astype(np.float32)).pin_memory()
    for via in ("fp32", "bf16x3"):
        # FP32-accuracy queries on the CUDA cores, or on the tensor cores in BF16x3 (same bound)
        srv = serve.FieldServer(models, pool, mem_budget=8 << 30, streams=2, fp32_via=via)
        srv.prepare(("bf16", "bf16x3"))
        closed = serve.make_queries(min(args.queries, 400), 64, rate_qps=0.0, seed=13)
        srv.run(closed[:50])
        sat = serve.latency_stats(srv.run(closed))
        print(json.dumps({"fp32_via": via, "load": "closed", **sat}), flush=True)
        mean_pts = np.mean([q.npoints() for q in closed])
        for frac in (0.25, 0.5, 0.75, 0.9):
            rate = frac * sat["Mpoints_s"] * 1e6 / mean_pts
            qs = serve.make_queries(args.queries, 64, rate_qps=rate, seed=14 + int(frac * 100))
            st = serve.latency_stats(srv.run(qs))
            print(json.dumps({"fp32_via": via, "load": frac, "rate_qps": rate, **st}), flush=True)


if __name__ == "__main__":
    main()
