#!/usr/bin/env python
"""Benchmark of the FST hot path on GB300.

One step = the randomized least-squares refit of the core on m = 8R rows sampled
from the Q data points (Sec. 5, eq. rand_core, Algorithm 2 with uniform sampling),
followed by the evaluation of the refitted model at all Q points (Sec. 6,
reconstruction by evaluating the basis functions).

Workloads (``--workload``):
  precision_64M (default): Q = 2^26 unstructured points (70% uniform, 30% in a band
      around a curved tanh front), ranks 24^3, Legendre degree <= 63, m = 8R = 110,592;
      accuracy against the FP64 oracle on the first 2^20 points;
  fp32_16M: Q = 2^24 points, degree <= 31, otherwise the same.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead,
on a bounded sample of the same workload, extrapolated to the same unit.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "Mpoints/s fst_eval + LS refit ms on 1 GB300 at stated rel-L2 vs FP64 oracle"
UNIT = "Mpoints/s"
RANKS = (24, 24, 24)
OVERSAMPLE = 8
WORKLOADS = {
    "precision_64M": {"Q": 1 << 26, "degree": 63, "seed": 303},
    "fp32_16M": {"Q": 1 << 24, "degree": 31, "seed": 2024},
}
ACCURACY_POINTS = 1 << 20       # rel-L2 of the evaluation against the oracle on the first 2^20 points


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="fst", choices=["fst", "reference"])
    ap.add_argument("--prec", default="bf16",
                    help="normal-matrix (Gram) precision of the refit: fp32, tf32, bf16, bf16x3; the PCG "
                         "refinement with FP64-accumulated residuals makes the core independent of it")
    ap.add_argument("--eval-prec", default="bf16x3", help="evaluation precision: fp32, tf32, bf16, bf16x3")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="precision_64M", choices=sorted(WORKLOADS))
    ap.add_argument("--Q", type=int, default=0, help="point count (default: the workload's)")
    a = ap.parse_args()
    w = WORKLOADS[a.workload]
    a.Q = a.Q or w["Q"]
    a.degree = w["degree"]
    a.seed = w["seed"]
    return a


# ----------------------------------------------------------------------------- workload
def make_workload(Q: int, seed: int, degree: int):
    from paper_1907_05884_gb300 import synth
    xyz = synth.points(Q, seed=seed + 1, clustered=0.3, dtype=np.float32)
    u, _ = synth.field_values(xyz, synth.field_spec(seed + 2, 20), seed=seed + 3)
    model = synth.random_model(RANKS, (degree,) * 3, seed=seed + 4, orthonormal=True)
    return xyz, u.astype(np.float32), model


def workload_config(name, Q, R, m, degree, prec, eval_prec):
    return {"workload": f"{name}: Q={Q} unstructured points in [-1,1]^3 (70% uniform, 30% in a 0.05 band "
                        f"around a tanh front), 20 Gaussians + 1e-4 noise, ranks {RANKS}, degree <= {degree}, "
                        f"refit on m = {OVERSAMPLE}R = {m} sampled rows, then evaluation at all Q points",
            "Q": Q, "ranks": list(RANKS), "R": R, "degree": degree, "m": m, "refit_prec": prec,
            "eval_prec": eval_prec, "model": "seeded synthetic model with orthonormal factor functions",
            "l2": "inputs larger than L2: xyz + u = 16 B/point = %.0f MB per step" % (16 * Q / 1e6)}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str | None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_index is not None:
            cmd += ["-i", gpu_index]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except (FileNotFoundError, PermissionError):
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [l.split(",") for l in Path(self.f.name).read_text().splitlines() if l.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_index_for_smi():
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    lr = int(os.environ.get("LOCAL_RANK", "0"))
    if vis:
        parts = [x for x in vis.split(",") if x.strip()]
        if lr < len(parts):
            return parts[lr].strip()
    return str(lr)


# ----------------------------------------------------------------------------- peaks
GRAM_PK_BF16_TRAFFIC = 13.94e9 + 0.3565e9
# DRAM bytes of one evaluation launch, keyed by (precision, points, degree), from one ncu
# capture of the current kernel (a smaller case scaled by the point count where stated)
EVAL_TRAFFIC = {
    # eval_pipe_kernel<BF16X3, 24, 24>: 201.70 MB read + 47.05 MB written at 2^24 points, degree 63
    # (ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum on the current kernel), scaled by
    # the point count (the traffic is the streamed coordinates and values at both sizes)
    ("bf16x3", 1 << 26, 63): 4 * (201.70e6 + 47.05e6),
}


def measured_peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    """FP32 FMA pipe: 128 lanes per SM, 2 flops per FMA."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# ----------------------------------------------------------------------------- oracle timing
def oracle_sample_timing(model, xyz, u, Q, m, nthreads, n_eval=8192, m_rows=16, R_chol=768):
    """Time the oracle on a bounded sample of the step and extrapolate to the full step:
    evaluation on ``n_eval`` points (per-point rate x Q), the normal equations of ``m_rows``
    sampled rows at the full R (per-row rate x m), and a Cholesky factorisation at
    ``R_chol`` (x (R / R_chol)^3).  Returns (seconds per full step, parts, description)."""
    import oracle
    R = model.R
    xs = np.ascontiguousarray(xyz[:, :n_eval].astype(np.float64))
    t0 = time.perf_counter()
    oracle.eval_points(model, xs, nthreads=nthreads)
    t_eval = (time.perf_counter() - t0) / n_eval * Q
    idx = np.arange(m_rows, dtype=np.int64)
    x64 = np.ascontiguousarray(xyz[:, :m_rows].astype(np.float64))
    u64 = np.ascontiguousarray(u[:m_rows].astype(np.float64))
    t0 = time.perf_counter()
    oracle.normal_equations(model, x64, u64, idx, nthreads=nthreads)
    t_gram = (time.perf_counter() - t0) / m_rows * m
    rng = np.random.default_rng(0)
    B = rng.normal(size=(R_chol + 8, R_chol))
    G = B.T @ B
    t0 = time.perf_counter()
    oracle.cholesky(G, nthreads=nthreads)
    t_chol = (time.perf_counter() - t0) * (R / R_chol) ** 3
    total = t_eval + t_gram + t_chol
    desc = (f"oracle eval on {n_eval} points scaled to Q={Q}; oracle normal equations on {m_rows} rows at "
            f"R={R} scaled to m={m}; oracle Cholesky at R={R_chol} scaled by (R/{R_chol})^3; {nthreads} threads")
    return total, {"eval_s": t_eval, "gram_s": t_gram, "cholesky_s": t_chol}, desc


# samples of the CPU baseline: all host cores, and one thread (about 10-20 s of CPU work each)
CPU_SAMPLE_ALL = {"n_eval": 65536, "m_rows": 256, "R_chol": 2048}
CPU_SAMPLE_ONE = {"n_eval": 8192, "m_rows": 32, "R_chol": 1536}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    Q = args.Q
    xyz, u, model = make_workload(1 << 16, seed=args.seed, degree=args.degree)
    R = model.R
    m = OVERSAMPLE * R
    nthreads = oracle.default_threads()
    times = []
    sample = {"n_eval": 4096, "m_rows": 16, "R_chol": 1024}
    for it in range(args.warmup + args.steps):
        t, parts, desc = oracle_sample_timing(model, xyz, u, Q, m, nthreads, **sample)
        if it >= args.warmup:
            times.append(t)
    t = statistics.median(times)
    value = Q / t / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, Q, R, m, args.degree, "fp64", "fp64"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle", "sample": desc,
                             "parts_s": parts},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1907_05884_gb300 import build as fbuild
    fbuild.build()
    from paper_1907_05884_gb300 import fst

    Q = args.Q
    from paper_1907_05884_gb300 import shard
    xyz, u, model = make_workload(Q, seed=shard.rank_seed(args.seed, rank), degree=args.degree)
    R = model.R
    m = OVERSAMPLE * R
    M = fst.Model(model)
    stream = torch.cuda.current_stream()
    xyz_d = torch.from_numpy(xyz).cuda()
    u_d = torch.from_numpy(u).cuda()
    out_d = torch.empty(Q, dtype=torch.float32, device="cuda")

    def barrier():
        if world > 1:
            dist.barrier()

    reports = []
    eval_ms = []

    def step(i, timed_eval=False):
        rep = M.refit(xyz_d, u_d, m, seed=1000 + i, prec=args.prec)
        if args.eval_prec != "fp32":
            M.prepare(args.eval_prec)        # the refitted core as tensor-core operand tiles
        if timed_eval:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        M.eval(xyz_d, prec=args.eval_prec, out=out_d)
        if timed_eval:
            e1.record(stream)
            return rep, (e0, e1)
        return rep, None

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()

    # device-resident timing
    launches0 = fst.kernel_launches()
    clocks = ClockSampler(gpu_index_for_smi()) if rank == 0 else None
    barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    evs = []
    for i in range(args.steps):
        rep, ev = step(args.warmup + i, timed_eval=True)
        reports.append(rep)
        evs.append(ev)
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop() if clocks else None
    launches = fst.kernel_launches() - launches0
    ms = t0.elapsed_time(t1)
    eval_ms = [a.elapsed_time(b) for a, b in evs]
    ms = shard.job_time_ms(ms, world, device="cuda")
    ms_step = ms / args.steps
    value = shard.job_throughput(Q, world, args.steps, ms)

    # end to end through the public API with host buffers (pinned), copies inside the region:
    # every step copies its inputs in and its result out, on a copy stream with two device
    # buffer sets, so step i+1's inputs and step i-1's result move while step i computes
    xyz_h = torch.from_numpy(xyz).pin_memory()
    u_h = torch.from_numpy(u).pin_memory()
    outs_h = [torch.empty(Q, dtype=torch.float32).pin_memory() for _ in range(2)]
    sets = [(xyz_d, u_d, out_d), (torch.empty_like(xyz_d), torch.empty_like(u_d), torch.empty_like(out_d))]
    copy = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)

    def copy_in(k):
        with torch.cuda.stream(copy):
            sets[k][0].copy_(xyz_h, non_blocking=True)
            sets[k][1].copy_(u_h, non_blocking=True)
            ev_in[k].record(copy)

    copy.wait_event(e0)
    copy_in(0)
    for i in range(args.steps):
        k, nk = i % 2, (i + 1) % 2
        if i + 1 < args.steps:
            if i >= 1:
                copy.wait_event(ev_done[nk])      # step i-1 has finished reading set nk
            copy_in(nk)
        stream.wait_event(ev_in[k])
        if i >= 2:
            stream.wait_event(ev_out[k])          # step i-2's result has left set k
        xk, uk, ok = sets[k]
        M.refit(xk, uk, m, seed=5000 + i, prec=args.prec)
        if args.eval_prec != "fp32":
            M.prepare(args.eval_prec)
        M.eval(xk, prec=args.eval_prec, out=ok)
        ev_done[k].record(stream)
        copy.wait_event(ev_done[k])
        with torch.cuda.stream(copy):
            outs_h[k].copy_(ok, non_blocking=True)
            ev_out[k].record(copy)
    stream.wait_stream(copy)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = shard.job_time_ms(e0.elapsed_time(e1), world, device="cuda")
    e2e_value = shard.job_throughput(Q, world, args.steps, e2e_ms)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return 0

    peaks, peak_kind = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sm_max = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
    gram_ms = statistics.mean(r["ms_gram"] for r in reports)
    chol_ms = statistics.mean(r["ms_cholesky"] for r in reports)
    refine_ms = statistics.mean(r["ms_refine"] for r in reports)
    refit_ms = statistics.mean(r["ms_sample"] + r["ms_factors"] + r["ms_gram"] + r["ms_cholesky"] + r["ms_refine"]
                               for r in reports)
    ev_ms = statistics.mean(eval_ms)
    nnz = sum(len(v) for v in model.val)
    gram_flops = m * R * (R + 1)                      # lower triangle of A^T A, 2 flops per product
    eval_tc_flops = 2 * R * Q                         # T = U1 C_(1): 2 r1 r2 r3 flops per point
    # CUDA-core work a point: the Khatri-Rao epilogue (2 (r2 r3 + r2)) and the Legendre
    # recurrence of the three modes (~5 flops a degree), plus the sparse factor values
    # (2 nnz) where they are not on the tensor cores (the FP32 form)
    eval_alu_flops_pt = 2 * (RANKS[1] * RANKS[2] + RANKS[1]) + 5 * 3 * args.degree
    if args.eval_prec == "fp32":
        eval_alu_flops_pt += 2 * nnz
    alu_peak = fp32_alu_peak_tflops(sm_max, sms)
    # tensor peaks: the measured cuBLAS BF16 burst figure (each kernel is timed alone, a few
    # milliseconds at a time, inside steps of well under a second of timed work);
    # TF32 = BF16 x 0.5 (nominal dense ratio); BF16x3 runs three BF16 products per term
    bf16_peak = peaks.get("bf16_tflops", peaks.get("bf16_tflops_sustained"))
    ratio = {"tf32": 0.5, "bf16": 1.0, "bf16x3": 1 / 3}
    tc_peak = {k: bf16_peak * v for k, v in ratio.items()}
    if args.prec == "fp32":
        roof_gram = {"kernel": "gram_simt (A^T A over sampled Khatri-Rao rows, CUDA cores)", "bound": "alu",
                     "achieved": gram_flops / (gram_ms / 1e3) / 1e12, "peak": alu_peak, "unit": "TFLOP/s",
                     "peak_source": f"FP32 ALU: {sms} SMs x 128 FMA/clk x 2 x {sm_max:.0f} MHz"}
    else:
        roof_gram = {"kernel": f"pack_kr + gram_pk_kernel<{args.prec}> (A^T A from the packed Khatri-Rao "
                               "operand, tcgen05; time of the whole Gram phase)",
                     "bound": "tensor", "achieved": gram_flops / (gram_ms / 1e3) / 1e12,
                     "peak": tc_peak[args.prec], "unit": "TFLOP/s",
                     "peak_source": f"{peak_kind} bf16_tflops (burst) {bf16_peak} x {ratio[args.prec]:.3f}"}
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one gram_pk_kernel<BF16>
    # launch at R = 13,824, m = 110,592 from one ncu capture of the current kernel
    roof_gram["traffic"] = GRAM_PK_BF16_TRAFFIC if (args.prec == "bf16" and R == 13824 and m == 110592) else None
    roof_gram["frac"] = roof_gram["achieved"] / roof_gram["peak"]
    roof_gram["ms"] = gram_ms
    # the evaluation's core contraction T = U1 C_(1): 2R flops a point over the evaluation
    # kernel's CUDA-event time; bytes: 12 B of coordinates in, 4 B of value out a point
    if args.eval_prec == "fp32":
        roof_eval = {"kernel": "eval_simt_kernel (FP32, CUDA cores)", "bound": "alu",
                     "achieved": eval_alu_flops_pt * Q / (ev_ms / 1e3) / 1e12, "peak": alu_peak}
    else:
        roof_eval = {"kernel": f"eval_pipe_kernel<{args.eval_prec}> (Legendre basis on the CUDA cores, factor "
                               "step and core contraction on tcgen05, Khatri-Rao epilogue from tensor memory)",
                     "bound": "tensor", "achieved": eval_tc_flops / (ev_ms / 1e3) / 1e12,
                     "peak": tc_peak[args.eval_prec],
                     "peak_source": f"{peak_kind} bf16_tflops (burst) {bf16_peak} x {ratio[args.eval_prec]:.3f}"}
    roof_eval.update({"unit": "TFLOP/s", "ms": ev_ms, "traffic": EVAL_TRAFFIC.get((args.eval_prec, Q, args.degree)),
                      "algorithmic_bytes": 16 * Q, "hbm_GBps": 16 * Q / (ev_ms / 1e3) / 1e9,
                      "hbm_peak_GBps": peaks["hbm_gbs"],
                      "alu_TFLOPs": eval_alu_flops_pt * Q / (ev_ms / 1e3) / 1e12, "alu_peak": alu_peak})
    roof_eval["frac"] = roof_eval["achieved"] / roof_eval["peak"]
    # the headline roofline is the core contraction of the evaluation, the largest kernel of
    # the step at this workload and the one the contraction target is stated for
    dominant = roof_eval
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec if args.prec == args.eval_prec else f"{args.prec}+{args.eval_prec}",
            "data": "synthetic",
            "config": workload_config(args.workload, Q, R, m, args.degree, args.prec, args.eval_prec),
            "refit_ms": refit_ms, "refit_gram_ms": gram_ms, "refit_cholesky_ms": chol_ms,
            "refit_pcg_ms": refine_ms,
            "refit_pcg_steps": statistics.mean(r["refine_steps"] for r in reports),
            "refit_fallback_fp64": max(r["fallback_fp64"] for r in reports),
            "refit_fallback_bf16x3": max(r["fallback_bf16x3"] for r in reports),
            "refit_shifted_preconditioner": max(r["shifted_preconditioner"] for r in reports),
            "eval_ms": ev_ms, "eval_Mpoints_s": Q / ev_ms / 1e3,
            "roofline": {k: v for k, v in dominant.items()},
            "rooflines": {"eval": roof_eval, "gram": roof_gram},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": xyz.nbytes + u.nbytes,
                    "d2h_bytes_per_step": 4 * Q},
            "gpu_launches": launches, "clocks": clk, "peaks": peak_kind}

    if world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        nthreads = oracle.default_threads()
        t_cpu, parts, desc = oracle_sample_timing(model, xyz, u, Q, m, nthreads, **CPU_SAMPLE_ALL)
        t_one, parts1, desc1 = oracle_sample_timing(model, xyz, u, Q, m, 1, **CPU_SAMPLE_ONE)
        line["cpu_baseline"] = {"value": Q / t_cpu / 1e6, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                                "sample": desc, "parts_s": parts,
                                "single_thread": {"value": Q / t_one / 1e6, "cores": 1, "sample": desc1,
                                                  "parts_s": parts1},
                                "cpu": platform_cpu()}
        # accuracy stated against the FP64 oracle: evaluation of the refitted model on the first
        # 2^20 points, and the normal-equation residual of the last refit (FP64, exact design)
        from paper_1907_05884_gb300 import synth
        cur = M.read()
        om = synth.Model(model.r, model.p, model.colptr, model.rowidx, model.val, cur["alpha"])
        na = min(ACCURACY_POINTS, Q)
        ref = oracle.eval_points(om, xyz[:, :na].astype(np.float64), nthreads=nthreads)
        got = sets[(args.steps - 1) % 2][2][:na].cpu().numpy()   # the last step's evaluation
        line["rel_l2_eval_vs_oracle"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        line["rel_l2_eval_points"] = na
        idx = oracle.sample(5000 + args.steps - 1, Q, m)   # rows of the last refit (e2e loop)
        x64 = xyz.astype(np.float64)
        u64 = u.astype(np.float64)
        g = oracle.normal_residual(om, x64, u64, idx, cur["alpha"], nthreads=nthreads)
        h = oracle.normal_residual(om, x64, u64, idx, np.zeros(R), nthreads=nthreads)
        line["refit_normal_residual_rel"] = float(np.linalg.norm(g) / np.linalg.norm(h))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


ARM_PARTS = {"0xd4f": "Arm Neoverse-V2", "0xd40": "Arm Neoverse-V1", "0xd0c": "Arm Neoverse-N1"}


def platform_cpu() -> str:
    try:
        for l in Path("/proc/cpuinfo").read_text().splitlines():
            if l.lower().startswith(("model name", "cpu part")):
                v = l.split(":", 1)[1].strip()
                return ARM_PARTS.get(v.lower(), v)
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


if __name__ == "__main__":
    sys.exit(main())
