"""CPU oracle for the statevector hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its binding) never imports, links or executes anything here, and this package
imports nothing from the product.

Contents
  sv_oracle.c   plain C, gate-by-gate complex128 statevector simulation
                (``run``, ``probabilities``, ``norm``, ``marginal``,
                ``gate_matrix``), the textbook definition the paper hands to
                Qiskit Aer (Sec. III-B, Listing 3).
  dense.py      numpy brute force: the 2^n x 2^n unitary of a circuit from
                Kronecker products, for n <= 8.  It pins sv_oracle.c.
  cut.py        CutQC reconstruction of the uncut distribution from the
                subcircuit-variant probabilities (Eqs. 3.2-3.7).

The C library is compiled on first use with the host gcc at -O3 (no -march
flags, so it builds and computes alike on x86-64 and Arm; no FMA contraction)
into ``oracle/_build/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsvoracle.so")
_lock = threading.Lock()
# Same memory layout as the C struct or_gate: int32 op, q0, q1, pad, 3 x float64.
_GATE_REC = np.dtype([("op", "<i4"), ("q0", "<i4"), ("q1", "<i4"),
                      ("theta", "<f8"), ("phi", "<f8"), ("lam", "<f8")], align=True)
_lib = None


def build(force: bool = False) -> str:
    """Compile sv_oracle.c into a shared library (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
    if r.returncode != 0:
        r = subprocess.run(base, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.oracle_gate_arity.argtypes = [ctypes.c_int]
            L.oracle_gate_matrix.argtypes = [ctypes.c_void_p, dp]
            L.oracle_gate_matrix.restype = ctypes.c_int
            L.oracle_validate.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]
            L.oracle_validate.restype = ctypes.c_long
            L.oracle_init.argtypes = [ctypes.c_int, dp, ctypes.c_uint64]
            L.oracle_apply.argtypes = [ctypes.c_int, dp, ctypes.c_void_p, ctypes.c_size_t]
            L.oracle_apply.restype = ctypes.c_long
            L.oracle_run.argtypes = [ctypes.c_int, dp, ctypes.c_void_p, ctypes.c_size_t]
            L.oracle_run.restype = ctypes.c_long
            L.oracle_probabilities.argtypes = [ctypes.c_int, dp, dp]
            L.oracle_norm.argtypes = [ctypes.c_int, dp]
            L.oracle_norm.restype = ctypes.c_double
            L.oracle_marginal.argtypes = [ctypes.c_int, dp, ctypes.c_uint64, dp]
            L.oracle_num_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _gates_ptr(g):
    g = np.ascontiguousarray(g)
    assert g.dtype.itemsize == 40
    return g, ctypes.c_void_p(g.ctypes.data if len(g) else 0)


def gate_matrix(op, theta=0.0, phi=0.0, lam=0.0) -> np.ndarray:
    """The oracle's matrix of one gate (2x2 or 4x4 complex128)."""
    rec = np.zeros(1, dtype=_GATE_REC)
    rec[0] = (op, 0, 1, theta, phi, lam)
    out = np.zeros(32)
    k = lib().oracle_gate_matrix(ctypes.c_void_p(rec.ctypes.data), _dp(out))
    if k == 0:
        raise ValueError(f"unknown opcode {op}")
    d = 1 << k
    return (out[: 2 * d * d : 2] + 1j * out[1 : 2 * d * d : 2]).reshape(d, d)


def validate(n: int, g) -> int:
    g, p = _gates_ptr(g)
    return int(lib().oracle_validate(n, p, len(g)))


def run(n: int, g, basis: int = 0) -> np.ndarray:
    """Final complex128 statevector of circuit g applied to |basis>."""
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi_r = psi.view(np.float64)
    lib().oracle_init(n, _dp(psi_r), basis)
    return apply(n, psi, g)


def apply(n: int, psi: np.ndarray, g) -> np.ndarray:
    """Applies circuit g to psi in place (complex128, length 2^n)."""
    assert psi.dtype == np.complex128 and psi.size == (1 << n) and psi.flags.c_contiguous
    g, p = _gates_ptr(g)
    rc = lib().oracle_apply(n, _dp(psi.view(np.float64)), p, len(g))
    if rc != 0:
        raise ValueError(f"invalid gate at index {-1 - rc}")
    return psi


def probabilities(psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = psi.size.bit_length() - 1
    out = np.empty(psi.size)
    lib().oracle_probabilities(n, _dp(psi.view(np.float64)), _dp(out))
    return out


def norm(psi: np.ndarray) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = psi.size.bit_length() - 1
    return float(lib().oracle_norm(n, _dp(psi.view(np.float64))))


def marginal(psi: np.ndarray, mask: int) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    n = psi.size.bit_length() - 1
    out = np.empty(1 << bin(mask).count("1"))
    lib().oracle_marginal(n, _dp(psi.view(np.float64)), mask, _dp(out))
    return out


def num_threads() -> int:
    return int(lib().oracle_num_threads())
