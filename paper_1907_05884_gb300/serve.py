"""Continuous-batching visualisation server over resident FST models.

Compressed fields stay resident on the device (their tensor-core core tiles prepared once).
Queries are either an axis-aligned slice (points generated on the device by fst_slice_points)
or an unstructured point set (copied from pinned host memory).  The serving loop:

  * admits arrived queries in arrival order while the device memory they need (16 bytes per
    point: coordinates and result) fits the budget -- a query larger than the whole budget is
    admitted alone when nothing else is in flight;
  * packs every admitted query of one precision into one fst_eval_batched call (one
    persistent launch per size class of ranks) on the next free stream, so queries that
    arrive while others run join the next launch instead of waiting for the GPU to drain;
  * retires a batch when its CUDA event completes, releasing its memory and stamping each
    query's latency (completion minus arrival).

All device work runs in libfst; this module only schedules.  Each query's result is the
same whether it is served alone or in a mix (fst_eval_batched equals fst_eval bit for bit).
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Query:
    qid: int
    field: int                      # index of the resident model
    kind: str                       # "slice" or "points"
    prec: str                       # "bf16x3", "bf16", "tf32" or "fp32"
    arrival: float = 0.0            # seconds from the start of the run
    # slice
    axis: int = 0
    value: float = 0.0
    res: int = 0
    # point set: rows [p0, p0+n) of the server's host point pool
    p0: int = 0
    n: int = 0
    # filled by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    out: object = None

    def npoints(self) -> int:
        return self.res * self.res if self.kind == "slice" else self.n


@dataclass
class _Batch:
    queries: list
    event: object
    stream: object
    nbytes: int
    bufs: list = field(default_factory=list)


class FieldServer:
    def __init__(self, models, point_pool, mem_budget: int = 2 << 30, streams: int = 2,
                 keep_results: bool = False, fp32_via: str = "fp32"):
        """fp32_via: the evaluator that serves queries asking for FP32 accuracy -- "fp32" (CUDA
        cores) or "bf16x3" (tensor cores, the same 1e-5 accuracy bound at several times the
        throughput)."""
        import torch
        from paper_1907_05884_gb300 import fst
        self.fst = fst
        self.torch = torch
        self.models = list(models)
        self.pool = point_pool                        # pinned host tensor (3, P) float32
        self.budget = int(mem_budget)
        self.streams = [torch.cuda.Stream() for _ in range(streams)]
        self.keep = keep_results
        assert fp32_via in ("fp32", "bf16x3")
        self.fp32_via = fp32_via
        self.mem_used = 0
        self.peak_mem = 0
        self.inflight: list[_Batch] = []
        self.boxes = []
        for M in self.models:
            d = M.read()
            self.boxes.append((d["lo"], d["hi"]))

    def prepare(self, precs=("bf16x3", "bf16", "tf32")):
        for M in self.models:
            for p in precs:
                M.prepare(p)

    # ------------------------------------------------------------------ one scheduling step
    def _retire(self, now_fn):
        keep = []
        for b in self.inflight:
            if b.event.query():
                t = now_fn()
                for q in b.queries:
                    q.t_done = t
                    if not self.keep:
                        q.out = None
                self.mem_used -= b.nbytes
            else:
                keep.append(b)
        self.inflight = keep

    def _launch(self, batch_q, now_fn):
        torch, fst = self.torch, self.fst
        busy = {id(b.stream) for b in self.inflight}
        stream = next(s for s in self.streams if id(s) not in busy)
        nbytes = sum(16 * q.npoints() for q in batch_q)
        self.mem_used += nbytes
        self.peak_mem = max(self.peak_mem, self.mem_used)
        bufs = []
        groups = collections.defaultdict(list)
        with torch.cuda.stream(stream):
            for q in batch_q:
                n = q.npoints()
                if q.kind == "slice":
                    lo, hi = self.boxes[q.field]
                    xyz = fst.slice_points(q.axis, q.value, lo, hi, q.res, q.res, stream=stream)
                else:
                    xyz = torch.empty((3, n), dtype=torch.float32, device="cuda")
                    xyz.copy_(self.pool[:, q.p0:q.p0 + n], non_blocking=True)
                out = torch.empty(n, dtype=torch.float32, device="cuda")
                q.out = out
                q.t_admit = now_fn()
                bufs += [xyz, out]
                prec = self.fp32_via if q.prec == "fp32" else q.prec
                groups[prec].append((self.models[q.field], xyz, out))
            for prec, items in groups.items():
                fst.eval_batched([m for m, _, _ in items], [x for _, x, _ in items], [o for _, _, o in items],
                                 prec=prec, stream=stream)
            ev = torch.cuda.Event()
            ev.record(stream)
        for t in bufs:
            t.record_stream(stream)
        self.inflight.append(_Batch(batch_q, ev, stream, nbytes, bufs))

    def run(self, queries, max_batch_points: int = 1 << 25, idle_sleep: float = 2e-5):
        """Serve `queries` (arrival times in seconds from now); returns them with latencies."""
        pending = collections.deque(sorted(queries, key=lambda q: q.arrival))
        waiting = collections.deque()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0
        while pending or waiting or self.inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                waiting.append(pending.popleft())
            self._retire(now)
            launched = False
            if waiting and len(self.inflight) < len(self.streams):
                batch, pts, need = [], 0, 0
                while waiting:
                    q = waiting[0]
                    b = 16 * q.npoints()
                    alone_ok = not self.inflight and not batch          # oversize: alone only
                    if (self.mem_used + need + b <= self.budget or alone_ok) and \
                            (pts + q.npoints() <= max_batch_points or not batch):
                        batch.append(waiting.popleft())
                        pts += q.npoints()
                        need += b
                        if alone_ok and b > self.budget:
                            break
                    else:
                        break
                if batch:
                    self._launch(batch, now)
                    launched = True
            if not launched:
                if self.inflight and (not waiting or len(self.inflight) >= len(self.streams)):
                    # nothing to admit until something completes or arrives
                    next_arr = pending[0].arrival - now() if pending else 1.0
                    if next_arr > 0:
                        time.sleep(min(idle_sleep, next_arr))
                elif pending and not waiting:
                    dt = pending[0].arrival - now()
                    if dt > 0:
                        time.sleep(min(dt, 1e-3))
        return list(queries)


def make_queries(n: int, n_fields: int, rate_qps: float, seed: int, precs=("fp32", "bf16"),
                 pool_points: int = 10_000_000, slice_res=(512, 2048), point_range=(1e3, 1e7)):
    """Poisson arrivals at `rate_qps`; half slices (random axis and offset, side log-uniform),
    half point sets (log-uniform size, rows of the host point pool); precision 50/50."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate_qps) if rate_qps > 0 else 0.0
        q = Query(qid=i, field=int(rng.integers(n_fields)), kind="slice" if rng.random() < 0.5 else "points",
                  prec=precs[int(rng.integers(len(precs)))], arrival=t)
        if q.kind == "slice":
            q.axis = int(rng.integers(3))
            q.value = float(rng.uniform(-1, 1))
            q.res = int(np.exp(rng.uniform(np.log(slice_res[0]), np.log(slice_res[1]))))
        else:
            q.n = int(np.exp(rng.uniform(np.log(point_range[0]), np.log(point_range[1]))))
            q.n = min(q.n, pool_points)
            q.p0 = int(rng.integers(0, pool_points - q.n + 1))
        out.append(q)
    return out


def latency_stats(queries):
    lat = np.array([q.t_done - q.arrival for q in queries])
    pts = sum(q.npoints() for q in queries)
    span = max(q.t_done for q in queries) - min(q.arrival for q in queries)
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "Mpoints_s": pts / span / 1e6, "queries": len(queries)}
