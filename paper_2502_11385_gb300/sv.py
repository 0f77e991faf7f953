"""ctypes binding of libsv (include/sv.h, include/sv_plan.h).

Argument marshalling only: every step of the statevector path runs in the
library's sm_103a kernels.  Importing this module loads the library and fails
loudly when it has not been built; there is no CPU fallback.

Names follow the C-ABI: ``create``, ``apply_circuit``, ``probabilities``,
``marginal_probabilities``, ``amplitudes``, ``norm``, ``batch_run`` ...
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .workloads import GATE_DTYPE

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsv.so")

SV_OK, SV_ERR_ARG, SV_ERR_QUBIT, SV_ERR_OOM, SV_ERR_SIZE, SV_ERR_CUDA, SV_ERR_TIMEOUT, SV_ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7
C64, C128 = 0, 1
ARITH_AUTO, ARITH_NATIVE, ARITH_DF64, ARITH_TC, ARITH_TC_SYNC = 0, 1, 2, 3, 4
# block classes of a plan (sv_plan.h)
BLOCK_DENSE, BLOCK_DIAG, BLOCK_PERM, BLOCK_KRON = 0, 1, 2, 3
DTYPES = {"c64": C64, "c128": C128, C64: C64, C128: C128}
NP_DTYPE = {C64: np.complex64, C128: np.complex128}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libsv is not built ({LIB_PATH} missing): run __graft_entry__.build() "
                      "or python paper_2502_11385_gb300/build.py; there is no CPU fallback")
_lib = ctypes.CDLL(LIB_PATH)


class RunOpts(ctypes.Structure):
    _fields_ = [("max_fuse_k", ctypes.c_int32), ("tile_qubits", ctypes.c_int32),
                ("arith", ctypes.c_int32), ("debug_checks", ctypes.c_int32), ("timing", ctypes.c_int32)]


class ApplyStats(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("n_passes", ctypes.c_int32), ("fuse_k", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32), ("arith", ctypes.c_int32), ("n_launches", ctypes.c_int32),
                ("flops", ctypes.c_double), ("hbm_bytes", ctypes.c_double), ("plan_ms", ctypes.c_double),
                ("kernel_ms", ctypes.c_double), ("max_kernel_ms", ctypes.c_double),
                ("upload_bytes", ctypes.c_double), ("alu_ops", ctypes.c_double),
                ("tensor_flops", ctypes.c_double)]


class BatchItem(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int32), ("dt", ctypes.c_int32), ("gates", ctypes.c_void_p),
                ("n_gates", ctypes.c_size_t), ("probs_out", ctypes.c_void_p), ("probs_on_device", ctypes.c_int32)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int32), ("n_launches", ctypes.c_int32),
                ("arena_bytes", ctypes.c_double), ("last_ms", ctypes.c_double)]


class PlanSummary(ctypes.Structure):
    _fields_ = [("n_blocks", ctypes.c_int32), ("n_passes", ctypes.c_int32), ("fuse_k", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32), ("flops", ctypes.c_double), ("model_ms", ctypes.c_double)]


class Costs(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_int32), ("arith", ctypes.c_int32), ("n_qubits", ctypes.c_int32),
                ("tile_qubits", ctypes.c_int32), ("pass_ps", ctypes.c_double), ("dense_ps", ctypes.c_double * 6),
                ("diag_ps", ctypes.c_double), ("sign_ps", ctypes.c_double), ("perm_ps", ctypes.c_double * 6)]


_vp, _sz, _i32, _u64, _dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
_SIGS = {
    "sv_state_bytes": ([_i32, _i32], _sz),
    "sv_create": ([_i32, _i32, ctypes.POINTER(_vp)], _i32),
    "sv_create_on": ([_vp, _sz, _i32, _i32, _vp, ctypes.POINTER(_vp)], _i32),
    "sv_destroy": ([_vp], None),
    "sv_num_qubits": ([_vp], _i32),
    "sv_dtype_of": ([_vp], _i32),
    "sv_device_ptr": ([_vp], _vp),
    "sv_reset": ([_vp, _u64], _i32),
    "sv_apply_circuit": ([_vp, _vp, _sz, ctypes.POINTER(RunOpts)], _i32),
    "sv_probabilities": ([_vp, _dp, _sz, _i32], _i32),
    "sv_marginal_probabilities": ([_vp, _u64, _dp, _sz, _i32], _i32),
    "sv_marginal_probabilities_noalloc": ([_vp, _i32, _i32, _u64, _dp, _sz, _i32, _vp], _i32),
    "sv_amplitudes": ([_vp, _vp, _sz, _i32], _i32),
    "sv_set_amplitudes": ([_vp, _vp, _sz, _i32], _i32),
    "sv_norm": ([_vp, ctypes.POINTER(ctypes.c_double)], _i32),
    "sv_last_stats": ([_vp, ctypes.POINTER(ApplyStats)], _i32),
    "sv_batch_run": ([ctypes.POINTER(BatchItem), _sz, ctypes.POINTER(RunOpts), ctypes.POINTER(ctypes.c_int)], _i32),
    "sv_batch_create": ([ctypes.POINTER(BatchItem), _sz, ctypes.POINTER(RunOpts), ctypes.POINTER(ctypes.c_int),
                         ctypes.POINTER(_vp)], _i32),
    "sv_batch_execute": ([_vp], _i32),
    "sv_batch_arena_bytes": ([ctypes.POINTER(BatchItem), _sz, ctypes.POINTER(RunOpts), ctypes.POINTER(_sz)], _i32),
    "sv_batch_create_in": ([ctypes.POINTER(BatchItem), _sz, ctypes.POINTER(RunOpts), ctypes.POINTER(ctypes.c_int),
                            _vp, _sz, ctypes.POINTER(_vp)], _i32),
    "sv_rebind": ([_vp, _vp, _sz, _i32, _i32], _i32),
    "sv_batch_destroy": ([_vp], None),
    "sv_batch_stats": ([_vp, ctypes.POINTER(BatchInfo)], _i32),
    "sv_cut_reconstruct": ([ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32, _i32, ctypes.POINTER(ctypes.c_int32),
                            _i32, _u64, _u64, _dp, _sz, _i32], _i32),
    "sv_cut_variants": ([_i32, _vp, _sz, _i32, ctypes.POINTER(ctypes.c_int32), _vp, _sz, _i32,
                         ctypes.POINTER(ctypes.c_int32), _i32, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i32,
                         ctypes.POINTER(RunOpts)], _i32),
    "sv_status_str": ([_i32], ctypes.c_char_p),
    "sv_version": ([], ctypes.c_char_p),
    "sv_plan_build": ([_i32, _i32, _vp, _sz, ctypes.POINTER(RunOpts), ctypes.POINTER(_vp)], _i32),
    "sv_plan_free": ([_vp], None),
    "sv_plan_summary_get": ([_vp, ctypes.POINTER(PlanSummary)], _i32),
    "sv_plan_block": ([_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32),
                       ctypes.POINTER(_i32), ctypes.POINTER(_i32), _sz, ctypes.POINTER(ctypes.c_double), _sz], _i32),
    "sv_plan_pass": ([_vp, _i32, ctypes.POINTER(_u64), ctypes.POINTER(_i32), ctypes.POINTER(_i32), _sz], _i32),
    "sv_plan_check": ([_vp, _vp, _sz], _i32),
    "sv_calibrate": ([_i32, _i32, ctypes.POINTER(Costs)], _i32),
    "sv_set_costs": ([_i32, _i32, ctypes.POINTER(Costs)], _i32),
}
for _name, (_args, _res) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _res

EXPORTED = tuple(_SIGS)


class SvError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__(f"{what}: {status_str(code)} ({code})")


def status_str(code: int) -> str:
    return _lib.sv_status_str(code).decode()


def version() -> str:
    return _lib.sv_version().decode()


def _check(code, what):
    if code != SV_OK:
        raise SvError(code, what)


_COST_KEYS = ("pass_ps", "dense_ps", "diag_ps", "sign_ps", "perm_ps")


def calibrate(dtype, arith=ARITH_AUTO) -> dict:
    """Measures the tile-pass cost table on the current device (sv_calibrate):
    picoseconds per amplitude of a pass, of dense / permutation blocks of
    k = 1..5 qubits and of diagonal blocks.  The returned dict carries the
    resolved arithmetic it was measured for."""
    c = Costs()
    _check(_lib.sv_calibrate(DTYPES[dtype], int(arith), ctypes.byref(c)), "sv_calibrate")
    return {"dt": c.dt, "arith": c.arith, "n_qubits": c.n_qubits, "tile_qubits": c.tile_qubits,
            "pass_ps": c.pass_ps, "dense_ps": list(c.dense_ps), "diag_ps": c.diag_ps, "sign_ps": c.sign_ps,
            "perm_ps": list(c.perm_ps)}


def set_costs(dtype, arith: int, costs) -> None:
    """Installs a measured cost table for (dtype, resolved arith) in the
    planner (sv_set_costs); costs=None returns that pair to the analytic
    model."""
    if costs is None:
        _check(_lib.sv_set_costs(DTYPES[dtype], int(arith), None), "sv_set_costs")
        return
    c = Costs()
    c.dt, c.arith = DTYPES[dtype], int(arith)
    c.n_qubits, c.tile_qubits = int(costs.get("n_qubits", 0)), int(costs.get("tile_qubits", 0))
    c.pass_ps, c.diag_ps, c.sign_ps = float(costs["pass_ps"]), float(costs["diag_ps"]), float(costs["sign_ps"])
    for i in range(6):
        c.dense_ps[i] = float(costs["dense_ps"][i])
        c.perm_ps[i] = float(costs["perm_ps"][i])
    _check(_lib.sv_set_costs(c.dt, c.arith, ctypes.byref(c)), "sv_set_costs")


def state_bytes(n: int, dtype) -> int:
    return int(_lib.sv_state_bytes(n, DTYPES[dtype]))


def as_gates(gates) -> np.ndarray:
    g = np.ascontiguousarray(gates)
    if g.dtype != GATE_DTYPE:
        raise TypeError("gates must be a numpy array with workloads.GATE_DTYPE")
    return g


def run_opts(max_fuse_k=0, tile_qubits=0, arith=ARITH_AUTO, debug_checks=0, timing=0):
    return RunOpts(max_fuse_k, tile_qubits, arith, debug_checks, timing)


def _opts_ptr(opts):
    if opts is None:
        return None
    if isinstance(opts, dict):
        opts = RunOpts(**opts)
    return ctypes.byref(opts)


def _ptr_of(buf):
    """(pointer, is_device, bytes) for a contiguous numpy array or torch tensor."""
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("buffer must be C-contiguous")
        return buf.ctypes.data, 0, buf.nbytes
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr(), 1 if buf.is_cuda else 0, buf.numel() * buf.element_size()
    raise TypeError(type(buf))


def _f64_len(buf, nbytes):
    itemsize = buf.itemsize if isinstance(buf, np.ndarray) else buf.element_size()
    if itemsize != 8:
        raise TypeError("probability buffers hold float64")
    return nbytes // 8


class State:
    """An n-qubit statevector in device memory (sv_state)."""

    def __init__(self, n: int, dtype="c128", _handle=None, _keep=None):
        self.n = n
        self.dt = DTYPES[dtype]
        self._keep = _keep
        if _handle is None:
            h = _vp()
            _check(_lib.sv_create(n, self.dt, ctypes.byref(h)), "sv_create")
            _handle = h
        self._h = _handle

    @classmethod
    def from_tensor(cls, tensor, n: int, dtype, stream=None):
        """Wraps a caller-owned CUDA tensor (kept alive by the State)."""
        dt = DTYPES[dtype]
        h = _vp()
        st = _vp(stream) if stream is not None else None
        _check(_lib.sv_create_on(tensor.data_ptr(), tensor.numel() * tensor.element_size(), n, dt, st,
                                 ctypes.byref(h)), "sv_create_on")
        return cls(n, dt, _handle=h, _keep=tensor)

    def rebind(self, tensor, n: int, dtype):
        """Points a from_tensor() handle at another caller-owned CUDA tensor."""
        dt = DTYPES[dtype]
        _check(_lib.sv_rebind(self._h, tensor.data_ptr(), tensor.numel() * tensor.element_size(), n, dt),
               "sv_rebind")
        self.n, self.dt, self._keep = n, dt, tensor
        return self

    def close(self):
        if getattr(self, "_h", None):
            _lib.sv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def dim(self):
        return 1 << self.n

    @property
    def device_ptr(self) -> int:
        return int(_lib.sv_device_ptr(self._h) or 0)

    def reset(self, basis: int = 0):
        _check(_lib.sv_reset(self._h, basis), "sv_reset")

    def apply_circuit(self, gates, opts=None):
        g = as_gates(gates)
        _check(_lib.sv_apply_circuit(self._h, g.ctypes.data if len(g) else None, len(g), _opts_ptr(opts)),
               "sv_apply_circuit")
        return self

    def stats(self) -> dict:
        s = ApplyStats()
        _check(_lib.sv_last_stats(self._h, ctypes.byref(s)), "sv_last_stats")
        return {f: getattr(s, f) for f, _ in ApplyStats._fields_}

    def probabilities(self, out=None):
        if out is None:
            out = np.empty(self.dim, dtype=np.float64)
        p, dev, nb = _ptr_of(out)
        _check(_lib.sv_probabilities(self._h, p, _f64_len(out, nb), dev), "sv_probabilities")
        return out

    def marginal_probabilities(self, qubit_mask: int, out=None):
        nb = 1 << bin(qubit_mask).count("1")
        if out is None:
            out = np.empty(nb, dtype=np.float64)
        p, dev, nbytes = _ptr_of(out)
        _check(_lib.sv_marginal_probabilities(self._h, qubit_mask, p, _f64_len(out, nbytes), dev),
               "sv_marginal_probabilities")
        return out

    def amplitudes(self, out=None):
        if out is None:
            out = np.empty(self.dim, dtype=NP_DTYPE[self.dt])
        p, dev, nb = _ptr_of(out)
        _check(_lib.sv_amplitudes(self._h, p, nb, dev), "sv_amplitudes")
        return out

    def set_amplitudes(self, src):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=NP_DTYPE[self.dt])
        p, dev, nb = _ptr_of(src)
        _check(_lib.sv_set_amplitudes(self._h, p, nb, dev), "sv_set_amplitudes")

    def norm(self) -> float:
        v = ctypes.c_double()
        _check(_lib.sv_norm(self._h, ctypes.byref(v)), "sv_norm")
        return v.value


def marginal_probabilities_noalloc(amplitudes_ptr: int, n: int, dtype, qubit_mask: int, out=None, stream=None):
    """Marginal distribution read straight from a state's device pointer,
    without allocating anything (sv_marginal_probabilities_noalloc): for
    callers that cannot have device memory allocated for them.  At most 16
    qubits in the mask; calls must not overlap on the GPU."""
    nb = 1 << bin(qubit_mask).count("1")
    if out is None:
        out = np.empty(nb, dtype=np.float64)
    p, dev, nbytes = _ptr_of(out)
    _check(_lib.sv_marginal_probabilities_noalloc(amplitudes_ptr, n, DTYPES[dtype], qubit_mask, p,
                                                  _f64_len(out, nbytes), dev, stream),
           "sv_marginal_probabilities_noalloc")
    return out


def create(n: int, dtype="c128") -> State:
    return State(n, dtype)


def simulate(n: int, gates, dtype="c128", opts=None):
    """Full-circuit execution: |0..0> -> circuit -> (amplitudes, probabilities)."""
    with State(n, dtype) as s:
        s.apply_circuit(gates, opts)
        return s.amplitudes(), s.probabilities()


def _batch_items(items):
    arr = (BatchItem * len(items))()
    keep, outs = [], []
    for i, (n, dtype, gates, out) in enumerate(items):
        g = as_gates(gates)
        if out is None:
            out = np.empty(1 << n, dtype=np.float64)
        p, dev, nb = _ptr_of(out)
        if nb != 8 << n:
            raise ValueError("probs_out must hold 2^n float64")
        keep.append(g)
        outs.append(out)
        arr[i] = BatchItem(n, DTYPES[dtype], g.ctypes.data if len(g) else None, len(g), p, dev)
    return arr, keep, outs


def batch_run(items, opts=None):
    """Batched form in one call.  items: list of (n, dtype, gates, probs_out
    or None).  Returns (outputs, per-item statuses)."""
    arr, _keep, outs = _batch_items(items)
    st = (ctypes.c_int * max(1, len(items)))()
    _lib.sv_batch_run(arr, len(items), _opts_ptr(opts), st)
    return outs, list(st)[: len(items)]


def batch_arena_bytes(items, opts=None) -> int:
    arr, _keep, _outs = _batch_items(items)
    b = _sz()
    _check(_lib.sv_batch_arena_bytes(arr, len(items), _opts_ptr(opts), ctypes.byref(b)), "sv_batch_arena_bytes")
    return int(b.value)


class Batch:
    """A prepared batch (sv_batch_create): its CUDA graph is replayed by
    execute(); outputs are refreshed in place on every execute()."""

    def __init__(self, items, opts=None, arena=None):
        """arena: optional caller-owned CUDA uint8 tensor of at least
        arena_bytes(items) bytes (kept alive by the Batch)."""
        self._arr, self._keep, self.outputs = _batch_items(items)
        self._arena = arena
        st = (ctypes.c_int * max(1, len(items)))()
        h = _vp()
        if arena is None:
            rc = _lib.sv_batch_create(self._arr, len(items), _opts_ptr(opts), st, ctypes.byref(h))
        else:
            rc = _lib.sv_batch_create_in(self._arr, len(items), _opts_ptr(opts), st, arena.data_ptr(),
                                         arena.numel() * arena.element_size(), ctypes.byref(h))
        self.status = list(st)[: len(items)]
        _check(rc, "sv_batch_create")
        self._h = h

    def execute(self):
        _check(_lib.sv_batch_execute(self._h), "sv_batch_execute")
        return self.outputs

    def stats(self) -> dict:
        b = BatchInfo()
        _check(_lib.sv_batch_stats(self._h, ctypes.byref(b)), "sv_batch_stats")
        return {f: getattr(b, f) for f, _ in BatchInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.sv_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def cut_reconstruct(up_probs, down_probs, width_a, cut_pos, width_b, keep_mask_a=None, keep_mask_b=None,
                    out=None):
    """CutQC reconstruction from device-resident variant distributions
    (torch CUDA tensors of float64): up_probs has 3^K entries, down_probs 4^K.
    Returns the distribution over the kept qubits (kept upstream qubits first)."""
    K = len(cut_pos)
    if keep_mask_a is None:
        keep_mask_a = ((1 << width_a) - 1) & ~sum(1 << q for q in cut_pos)
    if keep_mask_b is None:
        keep_mask_b = (1 << width_b) - 1
    na = bin(keep_mask_a).count("1")
    nb = bin(keep_mask_b).count("1")
    if out is None:
        out = np.empty(1 << (na + nb), dtype=np.float64)
    ups = (_vp * len(up_probs))(*[t.data_ptr() for t in up_probs])
    downs = (_vp * len(down_probs))(*[t.data_ptr() for t in down_probs])
    cp = (ctypes.c_int32 * K)(*cut_pos)
    p, dev, nbytes = _ptr_of(out)
    _check(_lib.sv_cut_reconstruct(ups, downs, K, width_a, cp, width_b, keep_mask_a, keep_mask_b, p,
                                   _f64_len(out, nbytes), dev), "sv_cut_reconstruct")
    return out


def cut_variants(cc, dtype="c128", up_out=None, down_out=None, opts=None):
    """All cut-subcircuit variants of a workloads.CutCircuit with shared work
    (sv_cut_variants).  Outputs: lists of 3^K and 4^K probability vectors
    (numpy on the host, or caller-supplied CUDA tensors)."""
    K = cc.n_cuts
    ga, gb = as_gates(cc.body_a), as_gates(cc.body_b)
    if up_out is None:
        up_out = [np.empty(1 << cc.width_a) for _ in range(3 ** K)]
    if down_out is None:
        down_out = [np.empty(1 << cc.width_b) for _ in range(4 ** K)]
    on_dev = 0 if isinstance(up_out[0], np.ndarray) else 1
    ups = (_vp * len(up_out))(*[_ptr_of(o)[0] for o in up_out])
    downs = (_vp * len(down_out))(*[_ptr_of(o)[0] for o in down_out])
    ca = (ctypes.c_int32 * K)(*cc.cut_qubits)
    cb = (ctypes.c_int32 * K)(*[q - cc.offset_b for q in cc.cut_qubits])
    _check(_lib.sv_cut_variants(DTYPES[dtype], ga.ctypes.data, len(ga), cc.width_a, ca, gb.ctypes.data, len(gb),
                                cc.width_b, cb, K, ups, downs, on_dev, _opts_ptr(opts)), "sv_cut_variants")
    return up_out, down_out


class Plan:
    """Host-side plan of a gate list (sv_plan_build); needs no GPU."""

    def __init__(self, n: int, dtype, gates, opts=None):
        self.gates = as_gates(gates)
        h = _vp()
        _check(_lib.sv_plan_build(n, DTYPES[dtype], self.gates.ctypes.data if len(self.gates) else None,
                                  len(self.gates), _opts_ptr(opts), ctypes.byref(h)), "sv_plan_build")
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None):
            _lib.sv_plan_free(self._h)
            self._h = None

    def summary(self) -> dict:
        s = PlanSummary()
        _check(_lib.sv_plan_summary_get(self._h, ctypes.byref(s)), "sv_plan_summary_get")
        return {f: getattr(s, f) for f, _ in PlanSummary._fields_}

    def block(self, b: int) -> dict:
        kind, k, ng = _i32(), _i32(), _i32()
        qs = (_i32 * 5)()
        _check(_lib.sv_plan_block(self._h, b, ctypes.byref(kind), ctypes.byref(k), qs, ctypes.byref(ng),
                                  None, 0, None, 0), "sv_plan_block")
        ids = (_i32 * max(ng.value, 1))()
        d = 1 << k.value
        diag = kind.value == BLOCK_DIAG
        nm = d if diag else d * d
        mat = (ctypes.c_double * (2 * nm))()
        _check(_lib.sv_plan_block(self._h, b, None, None, None, None, ids, ng.value, mat, 2 * nm), "sv_plan_block")
        m = np.frombuffer(mat, dtype=np.float64).copy().view(np.complex128)
        return {"kind": kind.value, "k": k.value, "qubits": list(qs)[: k.value],
                "gates": list(ids)[: ng.value], "mat": m if diag else m.reshape(d, d)}

    def pass_info(self, i: int) -> dict:
        mask, nb = _u64(), _i32()
        _check(_lib.sv_plan_pass(self._h, i, ctypes.byref(mask), ctypes.byref(nb), None, 0), "sv_plan_pass")
        ids = (_i32 * max(nb.value, 1))()
        _check(_lib.sv_plan_pass(self._h, i, None, None, ids, nb.value), "sv_plan_pass")
        return {"local_mask": mask.value, "blocks": list(ids)[: nb.value]}

    def check(self) -> int:
        return int(_lib.sv_plan_check(self._h, self.gates.ctypes.data if len(self.gates) else None,
                                      len(self.gates)))
