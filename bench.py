#!/usr/bin/env python
"""Benchmark of the statevector hot path on GB300.

One step = the whole path over one circuit: validate + plan (fusion, tile
passes) + initialise |0..0> + every tile pass + probabilities.  Workload: 30
qubits, complex128 (16 GiB state), GHZ prefix then a seeded depth-20 random
brickwork (920 gates), fusion width chosen by the planner's cost model.

Prints one JSON line.  `value` is statevector HBM GB/s: bytes the step's
kernels must move (init write, 2 x state per tile pass, probability pass
read + write) divided by the step time, with the state and output resident
in HBM.  `e2e` is the same through host buffers (probabilities copied to
pinned host memory inside the timed region).  `--impl reference` times the
CPU oracle instead (a bounded sample of the same circuit on the host cores).
With --gpus N > 1 (torchrun) every rank runs an independent replica.  The
default line also carries short measurements of the batching form (`batch`)
and of the serving form (`serve`), taken after the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP64_NOMINAL_TFLOPS = 1.25      # GB300 FP64 (CUDA cores), nominal
FP32_FMA_PER_CLK_SM = 128       # FP32 lanes per SM
SMS = 152
FAMILIES = ("adder", "aqft", "bv", "hwea", "supremacy")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=30)
    ap.add_argument("--depth", type=int, default=20)
    ap.add_argument("--dtype", default="c128", choices=["c128", "c64"])
    ap.add_argument("--arith", type=int, default=0,
                    help="0 auto, 1 native FP64, 2 double-float, 3 tensor cores (tcgen05), 4 tensor cores (mma.sync)")
    ap.add_argument("--fuse", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--form", default="full", choices=["full", "batch", "serve"],
                    help="full: one circuit (default); batch: the 91 cut-subcircuit variants of the "
                         "40-qubit brickwork; serve: a Poisson request stream")
    ap.add_argument("--circuit", default="ghz_brickwork",
                    choices=["ghz_brickwork", "brickwork", "qaoa"] + list(FAMILIES),
                    help="full form: GHZ + brickwork depth --depth seed 2 (default); brickwork depth --depth "
                         "seed 1 (12 q, depth 10, --fuse 1: the unfused 175-gate circuit); QAOA p = 2 seed 3 "
                         "on a random 3-regular graph; the paper's families (Sec. V-B): Cuccaro adder, AQFT "
                         "(degree 5), Bernstein-Vazirani, hardware-efficient ansatz (--depth layers), 2-D "
                         "random circuit (--depth cycles)")
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-wmax", type=int, default=30)
    ap.add_argument("--serve-sample", type=int, default=300,
                    help="requests of the serving sample added to the default line")
    ap.add_argument("--analytic-model", action="store_true",
                    help="plan with the analytic cost model instead of the tables measured on this GPU")
    ap.add_argument("--no-forms", action="store_true",
                    help="leave the batching and serving measurements out of the default line")
    return ap.parse_args()


def reduce_max(x: float, dist=None, device="cpu") -> float:
    """Max of a per-rank number over all ranks (identity without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(bytes_per_rank_step: float, world: int, ms_per_step: float) -> float:
    """Whole-job GB/s: every rank runs an independent replica of the step, the
    job's step time is the slowest rank's."""
    return world * bytes_per_rank_step / (ms_per_step / 1e3) / 1e9


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def code_of(text):
    """C/C++ source without comments and whitespace (string literals kept)."""
    import re
    pat = re.compile(r'"(?:\\.|[^"\\])*"|//[^\n]*|/\*.*?\*/', re.S)
    text = pat.sub(lambda m: m.group(0) if m.group(0).startswith('"') else " ", text)
    return "".join(text.split())


def kernel_hash():
    """Hash of the kernel code (comments and whitespace ignored), recorded
    beside each ncu traffic figure so that a figure is used only for the code
    it was taken from."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "device_types.hpp"):
        with open(os.path.join(ROOT, "paper_2502_11385_gb300", "csrc", f)) as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()[:16]


def ncu_traffic(workload_key, per_launch_scale):
    """DRAM bytes (read + write) per tile-pass launch from the committed ncu
    summaries: a line `traffic-record: key=<workload> bytes=<per launch>
    kernel_hash=<hash>` in profiles/*.md.  None when there is no record or the
    kernel source changed since the capture."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as f:
            for line in f:
                if not line.startswith("traffic-record:"):
                    continue
                kv = dict(tok.split("=", 1) for tok in line.split()[1:] if "=" in tok)
                if kv.get("key") == workload_key and kv.get("kernel_hash") == kernel_hash():
                    return float(kv["bytes"]) * per_launch_scale
    return None


def cpu_baseline(n, gates, seconds, state_bytes_c128):
    """The oracle (as it stands) on the host cores: applies a sample of the
    circuit's gates, spread evenly over the whole list (so the GHZ prefix and
    the U3 / CZ body appear in their proportions), one by one to a 2^n
    complex128 state until `seconds` have passed; each gate is one read +
    write sweep of the state.  Returns the sweep rate and the circuit time it
    implies (every gate at the sampled mean time)."""
    import numpy as np
    import oracle
    avail = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    m = n
    while m > 20 and (1 << m) * 16 * 1.5 > avail:
        m -= 1
    usable = [g for g in gates if g["q0"] < m and g["q1"] < m]
    psi = np.zeros(1 << m, dtype=np.complex128)
    psi[0] = 1
    oracle.apply(m, psi, usable[:1])  # first touch of the state's pages, untimed
    # stride through the list; the stride is set from the first gate's time
    t0 = time.perf_counter()
    oracle.apply(m, psi, usable[1:2])
    per_gate = max(1e-6, time.perf_counter() - t0)
    want = max(2, min(len(usable), int(seconds / per_gate)))
    stride = max(1, len(usable) // want)
    sample = usable[::stride]
    done, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and done < len(sample):
        oracle.apply(m, psi, sample[done:done + 1])
        done += 1
    dt = time.perf_counter() - t0
    sweep_gbs = done * 2 * (1 << m) * 16 / dt / 1e9
    full_s = len(gates) * (dt / done) * (1 << (n - m))
    return {"value": round(sweep_gbs, 3), "unit": "GB/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} of the {len(gates)} gates of the {n}-qubit circuit (every {stride}th, in order, "
                      f"all gate kinds) applied gate by gate to a {m}-qubit complex128 state in {dt:.1f} s; "
                      f"GB/s = gates x 2 x state bytes / time",
            "circuit_s_extrapolated": round(full_s, 1)}


def family_gates(name, n, depth, W):
    """The paper's benchmark families (Sec. V-B) as full-circuit runs on n
    qubits, from the generators in workloads.py, with fixed inputs."""
    mask = (1 << n) - 1
    if name == "adder":  # Cuccaro ripple-carry adder, m-bit registers, 2m + 2 qubits
        m = (n - 2) // 2
        a, b = 0x2A5B3C1D & ((1 << m) - 1), 0x15D3A2C7 & ((1 << m) - 1)
        return W.cuccaro_adder(m, a, b), f"{2 * m + 2}q Cuccaro adder (m={m}, a={a:#x}, b={b:#x})"
    if name == "aqft":  # approximate QFT of a basis state, controlled phases up to distance 5
        j = 0x2345677 & mask
        return W.aqft(n, 5, j), f"{n}q AQFT degree 5 of |{j:#x}>"
    if name == "bv":
        secret = 0x2CB8F0FA & ((1 << (n - 1)) - 1)
        return W.bernstein_vazirani(n, secret), f"{n}q Bernstein-Vazirani, secret {secret:#x}"
    if name == "hwea":
        return W.hwea(n, depth, 6), f"{n}q hardware-efficient ansatz, {depth} layers, seed 6"
    if name == "supremacy":
        rows = max(r for r in range(1, int(n ** 0.5) + 1) if n % r == 0)
        return W.supremacy(rows, n // rows, depth, 7), \
            f"{n}q 2-D random circuit on a {rows}x{n // rows} grid, {depth} cycles, seed 7"
    raise ValueError(name)


def workload_gates(args, W):
    """The full form's circuit and its name (the same for both arms)."""
    n = args.n
    if args.circuit == "qaoa":
        gates = W.workload_qaoa(n, 2, 3)[0]
        name = f"{n}q QAOA p=2 seed 3 on a random 3-regular graph ({len(gates)} gates)"
    elif args.circuit == "brickwork":
        gates = W.brickwork(n, args.depth, 1)
        name = f"{n}q brickwork depth {args.depth} seed 1 ({len(gates)} gates)"
    elif args.circuit in FAMILIES:
        gates, name = family_gates(args.circuit, n, args.depth, W)
        name = f"{name} ({len(gates)} gates)"
    else:
        gates = W.workload_ghz_brickwork(n, args.depth, 2)
        name = f"{n}q GHZ + brickwork depth {args.depth} seed 2 ({len(gates)} gates)"
    return gates, name


def run_reference(args):
    """The oracle arm: each step applies a bounded, evenly spread sample of the
    circuit's gates (cpu_baseline) on the host cores.  `value` is in the GPU
    arm's unit: the bytes the GPU path's step moves divided by the oracle's
    circuit time extrapolated from the sample, so that the two arms' values
    compare circuit times; the oracle's own sweep rate is reported beside it."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2502_11385_gb300 import workloads as W
    gates, wl_name = workload_gates(args, W)
    per_step = max(1.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    sweeps, circ_s, step_ms = [], [], []
    last = None
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_baseline(args.n, gates, per_step, 0)
        if i >= args.warmup:
            step_ms.append((time.perf_counter() - t0) * 1e3)
            sweeps.append(r["value"])
            circ_s.append(r["circuit_s_extrapolated"])
        last = r
    circuit_s = statistics.mean(circ_s)
    # the GPU arm's step bytes for this workload: init + 2 x state per pass +
    # probability read and write; its pass count comes from the plan
    state_bytes = (1 << args.n) * 16
    passes = None
    try:
        import __graft_entry__
        __graft_entry__.build_library()
        from paper_2502_11385_gb300 import sv
        passes = sv.Plan(args.n, "c128", gates, sv.run_opts(max_fuse_k=args.fuse, tile_qubits=args.tile,
                                                            arith=args.arith)).summary()["n_passes"]
    except Exception:  # no library on this host: count one pass per gate
        passes = len(gates)
    step_bytes = state_bytes * (1 + 2 * passes + 1) + (1 << args.n) * 8
    v = step_bytes / circuit_s / 1e9
    out = {"impl": "reference", "metric": "statevector HBM GB/s vs peak at 30q c128", "value": round(v, 3),
           "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(statistics.mean(step_ms), 1),
           "step": "a bounded sample of the circuit's gates (see cpu_baseline.sample), not the whole circuit",
           "circuit_s_extrapolated": round(circuit_s, 1),
           "value_basis": f"GPU-arm step bytes ({passes} passes) / extrapolated oracle circuit time",
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{wl_name}, complex128", "n_qubits": args.n, "state_dtype": "c128",
                      "arith": "oracle: complex128 gate by gate on the host cores"},
           "cpu_baseline": {"kind": "oracle", "cores": last["cores"], "sample": last["sample"], "value": round(v, 3),
                            "unit": "GB/s", "sweep_gbs": round(statistics.mean(sweeps), 3)},
           "e2e": {"value": round(v, 3), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch_form(args):
    """Batched form: all 4^3 downstream (22 q) and 3^3 upstream (21 q) variants
    of the 40-qubit cuttable brickwork (depth 12, seed 4) in one prepared batch
    (CUDA-graph replay), against looping the single-circuit path over the same
    variants on the same GPU.  Both write every variant's probabilities to
    device memory; results are compared bitwise."""
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv, workloads as W
    cc = W.workload_cut40()
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    out = {"form": "batch", "metric": "cut-subcircuit variants/s", "unit": "variants/s",
           "config": {"workload": "40q cuttable brickwork depth 12 seed 4, 3 cuts: 27 x 21q + 64 x 22q variants"},
           "results": []}
    for dtype in ("c128", "c64"):
        outs = [torch.empty(1 << cc.width_a, dtype=torch.float64, device="cuda") for _ in ups]
        outs += [torch.empty(1 << cc.width_b, dtype=torch.float64, device="cuda") for _ in downs]
        gl = ups + downs
        widths = [cc.width_a] * len(ups) + [cc.width_b] * len(downs)
        items = [(w, dtype, g, o) for w, g, o in zip(widths, gl, outs)]
        t0 = time.perf_counter()
        b = sv.Batch(items)
        build_ms = (time.perf_counter() - t0) * 1e3
        for _ in range(args.warmup):
            b.execute()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            b.execute()
        torch.cuda.synchronize()
        batch_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        ref = [o.clone() for o in outs]
        info = b.stats()
        b.close()
        # loop of the single-circuit path
        ctype = torch.complex128 if dtype == "c128" else torch.complex64
        bufs = {w: torch.empty(1 << w, dtype=ctype, device="cuda") for w in set(widths)}
        stream = torch.cuda.Stream()
        h = sv.State.from_tensor(bufs[cc.width_a], cc.width_a, dtype, stream=stream.cuda_stream)

        def loop():
            for w, g, o in zip(widths, gl, outs):
                h.rebind(bufs[w], w, dtype)
                h.reset(0)
                h.apply_circuit(g)
                h.probabilities(o)
        for _ in range(max(1, args.warmup // 2)):
            loop()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            loop()
        torch.cuda.synchronize()
        loop_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        same = all(torch.equal(a, c) for a, c in zip(ref, outs))
        h.close()
        del bufs
        # shared work: upstream body once, downstream by linearity (1 + 2^K bodies)
        up_o = [torch.empty_like(o) for o in outs[:len(ups)]]
        dn_o = [torch.empty_like(o) for o in outs[len(ups):]]
        sv.cut_variants(cc, dtype, up_o, dn_o)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.cut_variants(cc, dtype, up_o, dn_o)
        torch.cuda.synchronize()
        shared_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        shared_err = max((a - c).abs().max().item() for a, c in zip(ref, up_o + dn_o))
        # reconstruction (Eqs. 3.2-3.7) on the GPU: the marginal over 12 upstream
        # and 12 downstream qubits (2^24 outputs; the 2^40 joint does not fit)
        cut_q = list(cc.cut_qubits)
        keep_a = sum(1 << q for q in [q for q in range(cc.width_a) if q not in cut_q][:12])
        keep_b = (1 << 12) - 1
        rec = torch.empty(1 << 24, dtype=torch.float64, device="cuda")
        sv.cut_reconstruct(up_o, dn_o, cc.width_a, cut_q, cc.width_b, keep_a, keep_b, out=rec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.cut_reconstruct(up_o, dn_o, cc.width_a, cut_q, cc.width_b, keep_a, keep_b, out=rec)
        torch.cuda.synchronize()
        rec_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        rec_norm_err = abs(rec.sum().item() - 1.0)
        del up_o, dn_o, rec
        nv = len(items)
        out["results"].append({"dtype": dtype, "variants": nv, "batched_ms": round(batch_ms, 3),
                               "loop_ms": round(loop_ms, 3), "batched_variants_per_s": round(nv / batch_ms * 1e3, 2),
                               "loop_variants_per_s": round(nv / loop_ms * 1e3, 2),
                               "speedup": round(loop_ms / batch_ms, 3), "bitwise_equal": same,
                               "shared_work_ms": round(shared_ms, 3),
                               "shared_work_variants_per_s": round(nv / shared_ms * 1e3, 2),
                               "shared_work_speedup_vs_loop": round(loop_ms / shared_ms, 3),
                               "shared_work_max_abs_dp": shared_err,
                               "reconstruction": {"outputs": "2^24 (12 upstream + 12 downstream qubits)",
                                                  "terms": 4 ** len(cut_q), "ms": round(rec_ms, 3),
                                                  "abs_sum_minus_1": rec_norm_err},
                               "graph_launches": info["n_launches"], "arena_gib": round(info["arena_bytes"] / 2**30, 3),
                               "batch_build_ms": round(build_ms, 1)})
        torch.cuda.empty_cache()
    print(json.dumps(out), flush=True)


def batch_summary(steps):
    """The batching form in brief, for the default line: the 91 cut-subcircuit
    variants of the 40-qubit brickwork (27 x 21 q + 64 x 22 q) as one prepared
    batch (CUDA-graph replay) against looping the single-circuit path over the
    same variants; wall time per sweep of all variants, both writing device
    outputs; results compared bitwise."""
    import torch
    from paper_2502_11385_gb300 import sv, workloads as W
    cc = W.workload_cut40()
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    gl = ups + downs
    widths = [cc.width_a] * len(ups) + [cc.width_b] * len(downs)
    res = {"workload": "40q cuttable brickwork depth 12 seed 4, 3 cuts: 27 x 21q + 64 x 22q variants",
           "unit": "variants/s"}
    for dtype in ("c128", "c64"):
        outs = [torch.empty(1 << w, dtype=torch.float64, device="cuda") for w in widths]
        b = sv.Batch([(w, dtype, g, o) for w, g, o in zip(widths, gl, outs)])
        b.execute()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            b.execute()
        batch_ms = (time.perf_counter() - t0) * 1e3 / steps
        ref = [o.clone() for o in outs]
        b.close()
        ctype = torch.complex128 if dtype == "c128" else torch.complex64
        bufs = {w: torch.empty(1 << w, dtype=ctype, device="cuda") for w in set(widths)}
        stream = torch.cuda.Stream()
        h = sv.State.from_tensor(bufs[cc.width_a], cc.width_a, dtype, stream=stream.cuda_stream)

        def loop():
            for w, g, o in zip(widths, gl, outs):
                h.rebind(bufs[w], w, dtype)
                h.reset(0)
                h.apply_circuit(g)
                h.probabilities(o)
        loop()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            loop()
        torch.cuda.synchronize()
        loop_ms = (time.perf_counter() - t0) * 1e3 / steps
        same = all(torch.equal(a, c) for a, c in zip(ref, outs))
        h.close()
        nv = len(gl)
        res[dtype] = {"batched_variants_per_s": round(nv / batch_ms * 1e3, 1),
                      "looped_variants_per_s": round(nv / loop_ms * 1e3, 1),
                      "speedup": round(loop_ms / batch_ms, 3), "bitwise_equal": same, "sweeps": steps}
        if dtype == "c128":
            # reconstruction (Eqs. 3.2-3.7) of the marginal over 12 upstream and 12
            # downstream qubits (2^24 outputs; the 2^40 joint does not fit)
            cut_q = list(cc.cut_qubits)
            keep_a = sum(1 << q for q in [q for q in range(cc.width_a) if q not in cut_q][:12])
            rec = torch.empty(1 << 24, dtype=torch.float64, device="cuda")
            up_o, dn_o = outs[:len(ups)], outs[len(ups):]
            sv.cut_reconstruct(up_o, dn_o, cc.width_a, cut_q, cc.width_b, keep_a, (1 << 12) - 1, out=rec)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                sv.cut_reconstruct(up_o, dn_o, cc.width_a, cut_q, cc.width_b, keep_a, (1 << 12) - 1, out=rec)
            torch.cuda.synchronize()
            rec_ms = (time.perf_counter() - t0) * 1e3 / steps
            rec_bytes = (len(ups) * (1 << cc.width_a) + len(downs) * (1 << cc.width_b) + (1 << 24)) * 8
            peak = load_peaks()[0]["hbm_gbs"]
            res["reconstruction"] = {"outputs": "2^24 (12 upstream + 12 downstream qubits)",
                                     "terms": 4 ** len(cut_q), "ms": round(rec_ms, 3),
                                     "algorithmic_bytes": rec_bytes,
                                     "gbs": round(rec_bytes / rec_ms / 1e6, 1),
                                     "frac_of_hbm": round(rec_bytes / rec_ms / 1e6 / peak, 4),
                                     "abs_sum_minus_1": abs(rec.sum().item() - 1.0)}
            del rec
        del bufs, outs, ref
        torch.cuda.empty_cache()
    return res


def serve_summary(count):
    """The serving form in brief, for the default line: a Poisson stream of
    `count` requests (width log-uniform 10-30, depth 5-40, brickwork / QAOA,
    complex64 / complex128, seed 5) at offered loads rho = 0.7 and 2.0 of the
    serial path's measured mean service time, served (admission by bytes,
    continuous batching) and run serially; circuits/s and p50 / p99 latency."""
    from paper_2502_11385_gb300 import serve, sv, workloads as W
    opts = sv.run_opts()
    probe = W.serving_stream(60, 1.0, seed=1005, wmin=10, wmax=30)
    serve.mean_service_time(probe[:10], opts)
    sbar = serve.mean_service_time(probe, opts)
    res = {"workload": f"Poisson stream of {count} requests, width log-uniform 10-30, depth 5-40, "
                       f"brickwork/QAOA 50/50, c64/c128 50/50, seed 5", "mean_service_ms": round(sbar * 1e3, 2)}
    for rho in (0.7, 2.0):
        reqs = W.serving_stream(count, rho / sbar, seed=5, wmin=10, wmax=30)
        _, st = serve.Server(opts=opts, keep_outputs=False).run(reqs)
        _, ss = serve.run_serial(reqs, opts, keep_outputs=False)
        res[f"rho_{rho}"] = {"served": {k: st[k] for k in ("circuits_per_s", "p50_ms", "p99_ms", "mean_batch")},
                             "serial": {k: ss[k] for k in ("circuits_per_s", "p50_ms", "p99_ms",
                                                           "tile_pass_gpu_s", "throughput_bound_small_hidden")},
                             "throughput_ratio": round(st["circuits_per_s"] / ss["circuits_per_s"], 3)}
    return res


def dtype_summary(gates, n, dtype, steps):
    """The same circuit in another dtype, for the default line: tile-pass
    kernel time per circuit (CUDA events on the handle's stream) and the tile
    pass's HBM roofline fraction."""
    import torch
    from paper_2502_11385_gb300 import sv
    ct = torch.complex64 if dtype == "c64" else torch.complex128
    buf = torch.empty(1 << n, dtype=ct, device="cuda")
    stream = torch.cuda.Stream()
    st = sv.State.from_tensor(buf, n, dtype, stream=stream.cuda_stream)
    opts = sv.run_opts(timing=1)
    ks = []
    for i in range(steps + 2):
        st.reset(0)
        st.apply_circuit(gates, opts)
        if i >= 2:
            ks.append(st.stats())
    st.close()
    del buf
    torch.cuda.empty_cache()
    s0 = ks[-1]
    kern_ms = statistics.mean(k["kernel_ms"] for k in ks)
    amp = 8 if dtype == "c64" else 16
    launch_gbs = 2 * (amp << n) / (kern_ms / s0["n_launches"] / 1e3) / 1e9
    peak = load_peaks()[0]["hbm_gbs"]
    return {"kernel_ms_per_circuit": round(kern_ms, 2), "passes": s0["n_passes"], "blocks": s0["n_blocks"],
            "fuse_k": s0["fuse_k"], "tile_pass_gbs": round(launch_gbs, 1),
            "frac_of_measured_hbm": round(launch_gbs / peak, 4)}


def precision_summary(n=32):
    """The precision form (QAOA p = 2 on a seeded 3-regular graph): the
    circuit in complex128 and in complex64, their kernel times, and the
    complex64 result's max |delta a| and probability L1 distance from the
    complex128 one (both probability vectors computed in float64)."""
    import torch
    from paper_2502_11385_gb300 import sv, workloads as W
    free = torch.cuda.mem_get_info()[0]
    if free < (1 << n) * (16 + 8 + 8 + 8) * 1.1:
        return {"skipped": f"needs {(1 << n) * 40 / 2**30:.0f} GiB of free device memory"}
    g = W.workload_qaoa(n, 2, 3)[0]
    res = {"workload": f"{n}q QAOA p=2 seed 3 on a random 3-regular graph ({len(g)} gates)"}
    bufs = {}
    for dtype, ct in (("c128", torch.complex128), ("c64", torch.complex64)):
        buf = torch.empty(1 << n, dtype=ct, device="cuda")
        st = sv.State.from_tensor(buf, n, dtype)
        st.reset(0)
        st.apply_circuit(g, sv.run_opts(timing=1))
        res[f"{dtype}_kernel_ms"] = round(st.stats()["kernel_ms"], 1)
        res[f"{dtype}_norm_minus_1"] = abs(st.norm() - 1.0)
        st.close()
        bufs[dtype] = buf
    a, b = bufs["c128"], bufs["c64"]
    chunk, mx, l1 = 1 << 26, 0.0, 0.0
    for i in range(0, 1 << n, chunk):
        x, y = a[i:i + chunk], b[i:i + chunk].to(torch.complex128)
        mx = max(mx, (x - y).abs().max().item())
        l1 += ((x.real ** 2 + x.imag ** 2) - (y.real ** 2 + y.imag ** 2)).abs().sum().item()
    res["c64_vs_c128_max_abs_da"] = mx
    res["c64_vs_c128_prob_l1"] = l1
    del bufs, a, b
    torch.cuda.empty_cache()
    return res


def run_serve_form(args):
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import serve, sv, workloads as W
    opts = sv.run_opts()
    probe = W.serving_stream(100, 1.0, seed=1005, wmin=10, wmax=args.serve_wmax)
    serve.mean_service_time(probe[:10], opts)
    sbar = serve.mean_service_time(probe, opts)
    out = {"form": "serve", "metric": "circuits/s, p50/p99 latency", "mean_service_s": round(sbar, 5),
           "config": {"workload": f"Poisson stream of {args.serve_count} requests, width log-uniform 10-"
                                  f"{args.serve_wmax}, depth 5-40, brickwork/QAOA 50/50, c64/c128 50/50, seed 5"},
           "runs": []}
    for rho in (0.7, 2.0):
        reqs = W.serving_stream(args.serve_count, rho / sbar, seed=5, wmin=10, wmax=args.serve_wmax)
        srv = serve.Server(opts=opts, keep_outputs=False)
        _, st = srv.run(reqs)
        _, ss = serve.run_serial(reqs, opts, keep_outputs=False)
        out["runs"].append({"rho": rho, "rate_per_s": round(rho / sbar, 3), "served": st, "serial": ss})
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.form == "batch":
        run_batch_form(args)
        return
    if args.form == "serve":
        run_serve_form(args)
        return
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv, workloads as W

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    n, dt = args.n, args.dtype
    gates, wl_name = workload_gates(args, W)
    # the measured autotuner: this GPU's cost tables (cached JSON, measured on
    # first use) steer the planner's choice of fusion width and variant
    tuned = {}
    if not args.analytic_model:
        from paper_2502_11385_gb300 import tune
        tuned = tune.ensure()
    ctype = torch.complex128 if dt == "c128" else torch.complex64
    amp_bytes = 16 if dt == "c128" else 8
    state_bytes = (1 << n) * amp_bytes
    stream = torch.cuda.Stream()
    buf = torch.empty(1 << n, dtype=ctype, device="cuda")
    st = sv.State.from_tensor(buf, n, dt, stream=stream.cuda_stream)
    probs = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    opts = sv.run_opts(max_fuse_k=args.fuse, tile_qubits=args.tile, arith=args.arith, timing=1)

    stats_acc = []

    def step(out):
        st.reset(0)
        st.apply_circuit(gates, opts)
        stats_acc.append(st.stats())
        st.probabilities(out)

    for _ in range(args.warmup):
        step(probs)
    stats_acc.clear()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step(probs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    ms = reduce_max(ms, dist, "cuda")

    s0 = stats_acc[-1]
    passes = s0["n_passes"]
    step_bytes = state_bytes * (1 + 2 * passes + 1) + (1 << n) * 8
    value = job_throughput(step_bytes, world, ms)
    launches_per_step = 1 + s0["n_launches"] + 1

    # e2e: probabilities copied into pinned host memory every step
    host_p = torch.empty(1 << n, dtype=torch.float64, pin_memory=True)
    host_np = host_p.numpy()

    def e2e_step():
        st.reset(0)
        st.apply_circuit(gates, opts)
        st.probabilities(host_np)

    e2e_step()  # untimed: first use of the pinned buffer on this path
    torch.cuda.synchronize()
    barrier()
    e2e_steps = max(1, min(args.steps, 3))
    e2e_step_ms = []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ts = time.perf_counter()
        e2e_step()
        e2e_step_ms.append(round((time.perf_counter() - ts) * 1e3, 1))
    torch.cuda.synchronize()
    e2e_ms = reduce_max((time.perf_counter() - t0) * 1e3 / e2e_steps, dist, "cuda")
    e2e_val = job_throughput(step_bytes, world, e2e_ms)

    peaks, peak_src = load_peaks()
    kern_ms = statistics.mean(s["kernel_ms"] for s in stats_acc)
    avg_launch_ms = kern_ms / max(1, s0["n_launches"])
    arith = s0["arith"]
    # algorithmic bytes of one tile-pass launch: one read + one write of the state
    hbm_achieved = 2 * state_bytes / (avg_launch_ms / 1e3) / 1e9
    # ALU work the plan's arithmetic needs, counted as in the planner's model
    # (FP64 lane ops for native complex128; FP32 for complex64 FMAs and double-float)
    alu_ops = s0["alu_ops"]
    if dt == "c128" and arith == 1:
        alu_peak = FP64_NOMINAL_TFLOPS * 1e12 / 2          # FP64 lane ops (FMA = 1) per second
        alu_name = "FP64 nominal 1.25 TFLOP/s = 0.625 T lane-ops/s"
    else:
        alu_peak = SMS * FP32_FMA_PER_CLK_SM * peaks.get("sm_max_mhz", 2070.0) * 1e6
        alu_name = "FP32 152 SM x 128 lanes x max clock (lane-ops/s)"
    alu_achieved = alu_ops / (kern_ms / 1e3)
    tensor_peak = peaks.get("bf16_tflops", 1900.0)
    tc = arith in (3, 4) and s0["tensor_flops"] > 0
    if tc or hbm_achieved / peaks["hbm_gbs"] >= alu_achieved / alu_peak:
        # the pass's algorithmic work is its HBM traffic: the tensor-core
        # arithmetic (digit or triple-split products) is this design's means,
        # not the method's work, and is reported beside it
        roof = {"bound": "hbm", "achieved": round(hbm_achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(hbm_achieved / peaks["hbm_gbs"], 4), "peak_source": f"{peak_src} hbm_gbs",
                "bytes_per_launch": 2 * state_bytes}
    else:
        roof = {"bound": "alu", "achieved": round(alu_achieved / 1e12, 3), "peak": round(alu_peak / 1e12, 3),
                "unit": "T lane-ops/s", "frac": round(alu_achieved / alu_peak, 4), "peak_source": alu_name}
    if tc:
        tf = s0["tensor_flops"] / (kern_ms / 1e3) / 1e12
        roof["design_mma"] = {"what": ("16-bit MMA flops of the complex128 digit products (28 digit pairs)"
                                       if dt == "c128" else "bfloat16 MMA flops of the complex64 triple split "
                                                            "(6 part pairs)"),
                              "tflops": round(tf, 2), "peak": tensor_peak, "frac": round(tf / tensor_peak, 4)}
    wl_key = f"tile_pass_{n}q_{dt}"
    roof["kernel"] = "k_tile_pass"
    roof["launch_ms"] = round(avg_launch_ms, 3)
    roof["traffic"] = ncu_traffic(wl_key, 1.0)
    # the circuit's lower bound: its passes at the HBM peak, or its algorithmic
    # flops (the fused blocks' complex products, FMA = 2) at the tensor peak,
    # whichever is slower; the design's own MMA work is a separate figure
    hbm_bound_ms = passes * 2 * state_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    alg_bound_ms = s0["flops"] / (tensor_peak * 1e12) * 1e3
    bound_ms = max(hbm_bound_ms, alg_bound_ms)
    circuit_bound = {"passes": passes, "hbm_bound_ms": round(hbm_bound_ms, 2),
                     "algorithmic_flops": s0["flops"], "algorithmic_tensor_bound_ms": round(alg_bound_ms, 2),
                     "bound_ms": round(bound_ms, 2), "kernel_ms_per_circuit": round(kern_ms, 2),
                     "frac_of_bound": round(bound_ms / kern_ms, 4)}
    if tc:
        circuit_bound["design_mma_bound_ms"] = round(s0["tensor_flops"] / (tensor_peak * 1e12) * 1e3, 2)
    if dt == "c128":
        arith_name = {1: "native FP64", 2: "double-float (float pairs on the FP32 units)",
                      3: "Q56 fixed point, 7 balanced 8-bit digits as fp16 on tcgen05.mma, exact float32 level "
                         "sums re-assembled in int64 (absolute error < 2^-50 per block product)",
                      4: "Q62 fixed point, 8-bit digits on mma.sync"}.get(arith, "double-float")
        dtype_name = {1: "f64", 2: "f32x2", 3: "int64", 4: "int64"}.get(arith, "f32x2")
    else:
        arith_name = ("float32 components split into 3 bfloat16 parts on tcgen05.mma, float32 accumulation"
                      if arith == 3 else "float32 FMAs")
        dtype_name = "f32"
    fusion = f"k<={s0['fuse_k']} (cost-model choice among k=1..{4 if (dt == 'c128' and tc) else 5}" + \
             ("; tcgen05 digit blocks have at most 4 qubits)" if (dt == "c128" and tc) else ")")
    if args.fuse:
        fusion = f"k<={args.fuse} (fixed)"

    out = {"metric": "statevector HBM GB/s vs peak at 30q c128", "value": round(value, 2), "unit": "GB/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": dtype_name, "data": "synthetic",
           "config": {"workload": f"{wl_name}, complex{128 if dt == 'c128' else 64}",
                      "fusion": fusion, "n_qubits": n, "state_dtype": dt,
                      "storage": "complex128 (2 x float64)" if dt == "c128" else "complex64 (2 x float32)",
                      "arith": arith_name,
                      "fuse_k": s0["fuse_k"], "tile_qubits": s0["tile_qubits"], "passes": passes,
                      "blocks": s0["n_blocks"], "l2": f"state {state_bytes >> 30} GiB > L2, no flush needed",
                      "planner": ("cost tables measured on this GPU (sv_calibrate, cached)" if tuned
                                  else "analytic cost model"),
                      "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
           "frac_of_measured_hbm": round(value / peaks["hbm_gbs"], 4),
           "frac_of_8tbs": round(value / 8000.0, 4),
           "gate_equivalent_gbs": round(world * len(gates) * 2 * state_bytes / (ms / 1e3) / 1e9, 1),
           # the metric counts the passes the plan needs, so a plan with fewer
           # passes reads lower at equal speed: the circuit time against its
           # lower bound (pass bytes at the HBM peak, algorithmic flops at the
           # tensor peak)
           "circuit_bound": circuit_bound,
           "roofline": roof,
           "e2e": {"value": round(e2e_val, 2), "unit": "GB/s", "ms_per_step": round(e2e_ms, 3),
                   "h2d_bytes_per_step": int(s0["upload_bytes"]), "d2h_bytes_per_step": (1 << n) * 8,
                   "step_ms": e2e_step_ms, "warmup": 1},
           "gpu_launches": launches_per_step * args.steps,
           "clocks": clk}
    st.close()
    del buf, probs, host_p
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_forms:
        # the other dtype, the precision form and the batching and serving
        # forms, measured after the timed region
        other = "c64" if dt == "c128" else "c128"
        out[other] = dtype_summary(gates, n, other, max(2, min(args.steps, 5)))
        out["precision"] = precision_summary()
        out["batch"] = batch_summary(max(2, min(args.steps, 5)))
        out["serve"] = serve_summary(args.serve_sample)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(n, gates, args.cpu_seconds, state_bytes)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
