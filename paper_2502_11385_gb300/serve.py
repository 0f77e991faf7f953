"""Serving form: a request loop over the statevector engine.

The paper's CutQC Evaluator runs many subcircuit instances through a pool of
32 worker processes sized by trial (Listing 4, Sec. IV-A).  Here one process
serves a stream of circuit requests of mixed width on one GPU:

- admission: a request is admitted when its resident bytes (state + float64
  probability vector) fit in the HBM budget next to the requests already on
  the GPU (first come, first served; a request that does not fit waits);
- continuous batching: small requests (below `large_qubits`) that are admitted
  while a batch is running join the next batch; each batch is one sv_batch
  (multi-state launches in one CUDA graph) whose arena comes from the caching
  allocator, so no device-wide synchronisation happens;
- large requests run on worker threads with their own CUDA streams, so their
  kernels overlap with the batches on the device;
- every request's plan depends on that request only, so its result is the
  same alone and in the mix.

Latency = time its probabilities are on the host - arrival time.
"""
from __future__ import annotations

import argparse
import json
import math
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np

from . import sv
from . import workloads as W


@dataclass
class Result:
    rid: int
    n: int
    dtype: str
    arrival: float
    start: float = 0.0
    finish: float = 0.0
    status: int = 0
    probs: np.ndarray | None = None
    path: str = ""

    @property
    def latency(self):
        return self.finish - self.arrival


def need_bytes(n: int, dtype: str) -> int:
    return sv.state_bytes(n, dtype) + (8 << n) + (1 << 16)


def summarize(results, wall):
    lat = np.array([r.latency for r in results])
    ok = sum(1 for r in results if r.status == 0)
    return {"requests": len(results), "ok": ok, "wall_s": round(wall, 4),
            "circuits_per_s": round(len(results) / wall, 3) if wall > 0 else None,
            "p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3) if len(lat) else None,
            "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3) if len(lat) else None,
            "mean_ms": round(float(lat.mean()) * 1e3, 3) if len(lat) else None}


class Server:
    def __init__(self, budget_bytes=None, reserve_bytes=2 << 30, large_qubits=24, large_workers=2,
                 max_batch=256, opts=None, keep_outputs=True):
        import torch
        self.torch = torch
        torch.cuda.init()
        free, _total = torch.cuda.mem_get_info()
        self.budget = int(budget_bytes) if budget_bytes else int(free - reserve_bytes)
        self.large_qubits = large_qubits
        self.large_workers = large_workers
        self.max_batch = max_batch
        self.opts = opts
        self.keep_outputs = keep_outputs
        self.cv = threading.Condition()
        self.resident = 0
        self.peak_resident = 0
        self.small, self.large = deque(), deque()
        self.done_admitting = False
        self.batches = 0
        self.batch_sizes = []
        self.error = None

    # -- admission ---------------------------------------------------------
    def _admit(self, req, res, t0):
        need = need_bytes(req.n, req.dtype)
        if need > self.budget:
            res.status = sv.SV_ERR_OOM
            res.finish = time.perf_counter() - t0
            return
        with self.cv:
            while self.resident + need > self.budget and self.error is None:
                self.cv.wait(0.05)
            self.resident += need
            self.peak_resident = max(self.peak_resident, self.resident)
            (self.small if req.n < self.large_qubits else self.large).append((req, res))
            self.cv.notify_all()

    def _release(self, req):
        with self.cv:
            self.resident -= need_bytes(req.n, req.dtype)
            self.cv.notify_all()

    # -- workers -------------------------------------------------------------
    def _small_worker(self, t0):
        torch = self.torch
        try:
            while True:
                with self.cv:
                    while not self.small and not (self.done_admitting and not self.small):
                        self.cv.wait(0.05)
                    if not self.small and self.done_admitting:
                        return
                    take = [self.small.popleft() for _ in range(min(self.max_batch, len(self.small)))]
                start = time.perf_counter() - t0
                outs = [torch.empty(1 << q.n, dtype=torch.float64, device="cuda") for q, _ in take]
                items = [(q.n, q.dtype, q.gates, o) for (q, _), o in zip(take, outs)]
                arena = torch.empty(sv.batch_arena_bytes(items, self.opts) + 256, dtype=torch.uint8, device="cuda")
                off = (-arena.data_ptr()) % 256
                with sv.Batch(items, self.opts, arena=arena[off:]) as b:
                    b.execute()
                    status = b.status
                host = [o.cpu().numpy() for o in outs] if self.keep_outputs else [None] * len(outs)
                fin = time.perf_counter() - t0
                self.batches += 1
                self.batch_sizes.append(len(take))
                for (q, r), st, h in zip(take, status, host):
                    r.start, r.finish, r.status, r.probs, r.path = start, fin, st, h, "batch"
                    self._release(q)
                del arena, outs
        except Exception as e:  # surfaced by run()
            self.error = e

    def _large_worker(self, t0):
        torch = self.torch
        stream = torch.cuda.Stream()
        handle = None
        try:
            while True:
                with self.cv:
                    while not self.large and not self.done_admitting:
                        self.cv.wait(0.05)
                    if not self.large:
                        return
                    q, r = self.large.popleft()
                r.start = time.perf_counter() - t0
                ctype = torch.complex128 if q.dtype == "c128" else torch.complex64
                buf = torch.empty(1 << q.n, dtype=ctype, device="cuda")
                p = torch.empty(1 << q.n, dtype=torch.float64, device="cuda")
                if handle is None:
                    handle = sv.State.from_tensor(buf, q.n, q.dtype, stream=stream.cuda_stream)
                else:
                    handle.rebind(buf, q.n, q.dtype)
                try:
                    handle.reset(0)
                    handle.apply_circuit(q.gates, self.opts)
                    handle.probabilities(p)
                    r.status = 0
                except sv.SvError as e:
                    r.status = e.code
                r.probs = p.cpu().numpy() if self.keep_outputs else None
                r.finish = time.perf_counter() - t0
                r.path = "large"
                del buf, p
                self._release(q)
        except Exception as e:
            self.error = e
        finally:
            if handle is not None:
                handle.close()

    # -- driver --------------------------------------------------------------
    def run(self, requests, time_scale=1.0):
        """Serves `requests` (workloads.Request, arrival-ordered) in real time;
        arrival times are multiplied by time_scale.  Returns (results, stats)."""
        torch = self.torch
        results = [Result(q.rid, q.n, q.dtype, q.arrival * time_scale) for q in requests]
        self.done_admitting = False
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        workers = [threading.Thread(target=self._small_worker, args=(t0,), daemon=True)]
        workers += [threading.Thread(target=self._large_worker, args=(t0,), daemon=True)
                    for _ in range(self.large_workers)]
        for w in workers:
            w.start()
        for q, r in zip(requests, results):
            now = time.perf_counter() - t0
            if r.arrival > now:
                time.sleep(r.arrival - now)
            self._admit(q, r, t0)
            if self.error:
                break
        with self.cv:
            self.done_admitting = True
            self.cv.notify_all()
        for w in workers:
            w.join()
        if self.error:
            raise self.error
        wall = max(r.finish for r in results) - min(r.arrival for r in results)
        st = summarize(results, wall)
        st.update({"batches": self.batches, "mean_batch": round(float(np.mean(self.batch_sizes)), 2)
                   if self.batch_sizes else 0, "peak_resident_gib": round(self.peak_resident / 2 ** 30, 3),
                   "budget_gib": round(self.budget / 2 ** 30, 2)})
        return results, st


def run_serial(requests, opts=None, time_scale=1.0, keep_outputs=True, large_qubits=24):
    """The plain single-circuit path, one request at a time in arrival order.
    Also records each request's tile-pass GPU time (CUDA events), split
    between requests below and from `large_qubits` on: with the small ones
    fully hidden, no schedule can serve the stream faster than
    requests / (GPU time of the large ones)."""
    import torch
    results = [Result(q.rid, q.n, q.dtype, q.arrival * time_scale) for q in requests]
    stream = torch.cuda.Stream()
    handle = None
    o = opts if opts is not None else sv.run_opts()
    topts = sv.run_opts(max_fuse_k=o.max_fuse_k, tile_qubits=o.tile_qubits, arith=o.arith,
                        debug_checks=o.debug_checks, timing=1)
    gpu_ms = {"small": 0.0, "large": 0.0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for q, r in zip(requests, results):
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        r.start = time.perf_counter() - t0
        ctype = torch.complex128 if q.dtype == "c128" else torch.complex64
        buf = torch.empty(1 << q.n, dtype=ctype, device="cuda")
        p = torch.empty(1 << q.n, dtype=torch.float64, device="cuda")
        if handle is None:
            handle = sv.State.from_tensor(buf, q.n, q.dtype, stream=stream.cuda_stream)
        else:
            handle.rebind(buf, q.n, q.dtype)
        handle.reset(0)
        handle.apply_circuit(q.gates, topts)
        gpu_ms["large" if q.n >= large_qubits else "small"] += handle.stats()["kernel_ms"]
        handle.probabilities(p)
        r.probs = p.cpu().numpy() if keep_outputs else None
        r.finish = time.perf_counter() - t0
        r.path = "serial"
    if handle is not None:
        handle.close()
    wall = max(r.finish for r in results) - min(r.arrival for r in results)
    st = summarize(results, wall)
    st["tile_pass_gpu_s"] = {k: round(v / 1e3, 3) for k, v in gpu_ms.items()}
    if gpu_ms["large"] > 0:
        st["throughput_bound_small_hidden"] = round(len(results) / (gpu_ms["large"] / 1e3), 3)
    return results, st


def mean_service_time(requests, opts=None):
    """Mean time of the plain path per request (no waiting between requests)."""
    timed = [W.Request(q.rid, 0.0, q.n, q.dtype, q.family, q.depth, q.gates) for q in requests]
    _, st = run_serial(timed, opts, keep_outputs=False)
    return st["wall_s"] / max(1, len(requests))


def main():
    ap = argparse.ArgumentParser(description="serving form: Poisson stream, continuous batching")
    ap.add_argument("--count", type=int, default=2000)
    ap.add_argument("--rho", type=float, nargs="+", default=[0.7, 2.0])
    ap.add_argument("--wmin", type=int, default=10)
    ap.add_argument("--wmax", type=int, default=30)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--warm", type=int, default=100)
    ap.add_argument("--large-qubits", type=int, default=24)
    args = ap.parse_args()
    opts = sv.run_opts()
    probe = W.serving_stream(args.warm, 1.0, seed=args.seed + 1000, wmin=args.wmin, wmax=args.wmax)
    mean_service_time(probe[:5], opts)  # warm-up
    sbar = mean_service_time(probe, opts)
    out = {"mean_service_s": round(sbar, 5), "runs": []}
    for rho in args.rho:
        reqs = W.serving_stream(args.count, rho / sbar, seed=args.seed, wmin=args.wmin, wmax=args.wmax)
        srv = Server(large_qubits=args.large_qubits, opts=opts, keep_outputs=False)
        _, st = srv.run(reqs)
        _, ss = run_serial(reqs, opts, keep_outputs=False)
        out["runs"].append({"rho": rho, "rate_per_s": round(rho / sbar, 3), "served": st, "serial": ss})
    print(json.dumps(out))


if __name__ == "__main__":
    main()
