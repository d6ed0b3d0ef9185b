"""Accuracy and timing of configurations 1-3 against the FP64 oracle (test infrastructure: it
runs the library on the GPU and compares with `oracle/`).

    python tests/measure_configs.py precision --reps 3   # 2^26 points, degree 63, every precision
    python tests/measure_configs.py plain --reps 3       # FP64 small model; plain FP32 vs tensor cores

Prints one JSON line per measurement.
"""
from __future__ import annotations

import argparse
import sys
from pathlib import Path

import numpy as np

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))


def _peaks():
    import json
    from pathlib import Path
    p = Path(__file__).resolve().parents[1] / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        # burst figure: each evaluation and Gram is timed alone, a few milliseconds at a time
        return d.get("bf16_tflops", d.get("bf16_tflops_sustained")), "measured"
    return 1900.0, "fallback"


def _timed(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def precision(args):
    """Precision workload: --n points (default 2^26), ranks 24^3, degree 63 (orthonormal
    synthetic model); evaluation in FP32 / TF32 / BF16 / BF16x3 with rel-L2 against the FP64
    oracle on the first 2^20 points, and the refit on m = 8R rows with TF32 / BF16 / BF16x3
    Gram assembly (normal-equation residual against the oracle on those rows)."""
    import json
    import torch
    import oracle
    from paper_1907_05884_gb300 import fst, synth
    oracle.build()
    nth = oracle.default_threads()
    Q = args.n
    deg = args.degree
    ranks = tuple(args.ranks)
    model = synth.random_model(ranks, (deg,) * 3, seed=31, orthonormal=True)
    xyz_np = synth.points(Q, seed=33, clustered=0.3, dtype=np.float32)
    u_np, _ = synth.field_values(xyz_np, synth.field_spec(34, 20), seed=35)
    M = fst.Model(model)
    xyz = torch.from_numpy(xyz_np).cuda()
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    out = torch.empty(Q, device="cuda")
    R = model.R
    sub = 1 << 20
    ref = oracle.eval_points(model, xyz_np[:, :sub].astype(np.float64), nthreads=nth)
    bf16_peak, kind = _peaks()
    tc_peak = {"tf32": bf16_peak * 0.5, "bf16": bf16_peak, "bf16x3": bf16_peak / 3}
    for prec in ("fp32", "tf32", "bf16", "bf16x3"):
        if prec != "fp32":
            M.prepare(prec)
        ms = _timed(lambda: M.eval(xyz, prec=prec, out=out), args.reps)
        rel = float(np.linalg.norm(out[:sub].cpu().numpy() - ref) / np.linalg.norm(ref))
        line = {"config": "precision", "what": "eval", "prec": prec, "Q": Q, "ranks": ranks, "degree": deg,
                "ms": ms, "Mpoints_s": Q / ms / 1e3, "rel_l2_first_2^20_vs_oracle": rel}
        if prec != "fp32":
            line["contraction_roofline_frac"] = 2 * R * Q / (ms / 1e3) / 1e12 / tc_peak[prec]
            line["peak"] = f"{kind} bf16 burst {bf16_peak} TFLOP/s x {tc_peak[prec] / bf16_peak:.3f}"
        print(json.dumps(line), flush=True)
    m = 8 * R
    for prec in ("tf32", "bf16", "bf16x3"):
        M.set_core(model.alpha)
        rep = M.refit(xyz, u, m, seed=77, prec=prec)
        idx = oracle.sample(77, Q, m)
        cur = M.read()["alpha"].reshape(-1)
        x64 = xyz_np.astype(np.float64)
        g = oracle.normal_residual(model, x64, u_np.astype(np.float64), idx, cur, nthreads=nth)
        h = oracle.normal_residual(model, x64, u_np.astype(np.float64), idx, np.zeros(R), nthreads=nth)
        print(json.dumps({"config": "precision", "what": "refit", "prec": prec, "m": m, "R": R,
                          "ms": sum(rep[k] for k in ("ms_sample", "ms_factors", "ms_gram", "ms_cholesky",
                                                     "ms_refine")),
                          "ms_gram": rep["ms_gram"], "ms_cholesky": rep["ms_cholesky"],
                          "ms_refine": rep["ms_refine"], "refine_steps": rep["refine_steps"],
                          "gram_tflops": m * R * (R + 1) / (rep["ms_gram"] / 1e3) / 1e12,
                          "normal_residual_rel_vs_oracle": float(np.linalg.norm(g) / np.linalg.norm(h)),
                          "fallbacks": [rep["fallback_bf16x3"], rep["shifted_preconditioner"],
                                        rep["fallback_fp64"]]}), flush=True)


def plain(args):
    """Plain forms.  Config 1: 20,000 uniform points, 5 Gaussians, fst_fit in FP64 (grid 32^3,
    5% interpolated, eps 1e-3, ranks <= 8, degree <= 15, m = 4R) and FP64 evaluation at all
    points against the oracle.  Config 2: 2^24 points, ranks 24^3, degree 31: evaluation and
    refit on the CUDA cores in FP32 beside the BF16 / BF16x3 tensor-core forms."""
    import json
    import torch
    import oracle
    from paper_1907_05884_gb300 import fst, synth
    oracle.build()
    nth = oracle.default_threads()
    # config 1
    Q = 20000
    xyz_np = synth.points(Q, seed=41, clustered=0.0, dtype=np.float32)
    u_np, clean = synth.field_values(xyz_np, synth.field_spec(42, 5), seed=43)
    xyz = torch.from_numpy(xyz_np).cuda()
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    M, rep = fst.fit(xyz, u, grid=(32, 32, 32), sample_frac=0.05, eps=1e-3, max_rank=(8, 8, 8), max_degree=15,
                     oversample=4.0, seed=44, prec="fp64")
    e1.record()
    torch.cuda.synchronize()
    fit_ms = e0.elapsed_time(e1)
    x64 = torch.from_numpy(xyz_np.astype(np.float64)).cuda()
    ev = _timed(lambda: M.eval_f64(x64), args.reps)
    got = M.eval_f64(x64).cpu().numpy()
    d = M.read()
    om = synth.Model(d["r"], d["p"], d["colptr"], d["rowidx"], d["val"], d["alpha"], d["lo"], d["hi"])
    ref = oracle.eval_points(om, xyz_np.astype(np.float64), nthreads=nth)
    print(json.dumps({"config": "plain_fp64", "Q": Q, "fit_ms": fit_ms, "ranks": rep["r"], "nnz": rep["nnz"],
                      "m": rep["m"], "eval_ms": ev,
                      "rel_l2_eval_vs_oracle": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)),
                      "rel_l2_vs_noise_free_field": float(np.linalg.norm(got - clean) / np.linalg.norm(clean)),
                      "compression_ratio": rep["compression_ratio"]}), flush=True)
    # config 2
    Q = 1 << 24
    model = synth.random_model((24, 24, 24), (31,) * 3, seed=4, orthonormal=True)
    xyz_np = synth.points(Q, seed=45, clustered=0.3, dtype=np.float32)
    u_np, _ = synth.field_values(xyz_np, synth.field_spec(46, 20), seed=47)
    M = fst.Model(model)
    xyz = torch.from_numpy(xyz_np).cuda()
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    out = torch.empty(Q, device="cuda")
    sub = 1 << 18
    for prec in ("fp32", "bf16x3", "bf16"):
        M.set_core(model.alpha)
        rep = M.refit(xyz, u, 8 * model.R, seed=48, prec=prec)
        if prec != "fp32":
            M.prepare(prec)
        ms = _timed(lambda: M.eval(xyz, prec=prec, out=out), args.reps)
        d = M.read()
        om = synth.Model(d["r"], d["p"], d["colptr"], d["rowidx"], d["val"], d["alpha"], d["lo"], d["hi"])
        ref = oracle.eval_points(om, xyz_np[:, :sub].astype(np.float64), nthreads=nth)
        rel = float(np.linalg.norm(out[:sub].cpu().numpy() - ref) / np.linalg.norm(ref))
        print(json.dumps({"config": "plain_fp32_vs_tensor", "prec": prec, "Q": Q, "eval_ms": ms,
                          "eval_Mpoints_s": Q / ms / 1e3, "rel_l2_eval_first_2^18_vs_oracle": rel,
                          "refit_ms": sum(rep[k] for k in ("ms_sample", "ms_factors", "ms_gram", "ms_cholesky",
                                                           "ms_refine")),
                          "refit_gram_ms": rep["ms_gram"], "refit_cholesky_ms": rep["ms_cholesky"],
                          "refit_pcg_ms": rep["ms_refine"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["precision", "plain"])
    ap.add_argument("--n", type=int, default=1 << 26)
    ap.add_argument("--ranks", type=int, nargs=3, default=[24, 24, 24])
    ap.add_argument("--degree", type=int, default=63)
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args()
    from paper_1907_05884_gb300 import build
    build.build()
    return precision(args) if args.what == "precision" else plain(args)


if __name__ == "__main__":
    main()
