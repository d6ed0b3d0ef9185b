"""Run one libfst entry point on seeded synthetic inputs, for timing and profiling.

    python -m paper_1907_05884_gb300.drive gram  --prec bf16   --m 16384
    python -m paper_1907_05884_gb300.drive eval  --prec bf16x3 --n 4194304
    python -m paper_1907_05884_gb300.drive refit --prec bf16   --n 1048576
    python -m paper_1907_05884_gb300.drive chol  --prec fp32

The model has ranks 24^3 and Legendre degree 31 with orthonormal factor functions (unless
--ranks/--degree say otherwise); each call is repeated --reps times and timed with CUDA events.
"""
from __future__ import annotations

import argparse

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["gram", "eval", "refit", "sample"])
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--m", type=int, default=16384)
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--ranks", type=int, nargs=3, default=[24, 24, 24])
    ap.add_argument("--degree", type=int, default=31)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()

    import torch
    from paper_1907_05884_gb300 import build
    build.build()
    from paper_1907_05884_gb300 import fst, synth

    model = synth.random_model(tuple(args.ranks), (args.degree,) * 3, seed=4, orthonormal=True)
    M = fst.Model(model)
    Q = max(args.n, 2 * args.m)
    xyz = torch.from_numpy(synth.points(Q, seed=5, clustered=0.3).astype(np.float32)).cuda()
    u_np, _ = synth.field_values(xyz.cpu().numpy(), synth.field_spec(6, 20), seed=7)
    u = torch.from_numpy(u_np.astype(np.float32)).cuda()
    out = torch.empty(Q, device="cuda")
    idx = fst.sample_rows(8, Q, args.m)
    if args.what == "eval" and args.prec != "fp32":
        M.prepare(args.prec)
    for r in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        extra = ""
        if args.what == "gram":
            fst.normal_matrix(M, xyz, u, idx, prec=args.prec, with_h=False)
        elif args.what == "eval":
            M.eval(xyz[:, :args.n].contiguous() if Q != args.n else xyz, prec=args.prec, out=out[:args.n])
        elif args.what == "refit":
            rep = M.refit(xyz, u, args.m, seed=9, prec=args.prec)
            extra = f" {rep}"
        else:
            fst.sample_rows(10 + r, Q, args.m)
        e1.record()
        torch.cuda.synchronize()
        print(f"{args.what} prec={args.prec} m={args.m} n={args.n} ms={e0.elapsed_time(e1):.3f}{extra}", flush=True)


if __name__ == "__main__":
    main()
