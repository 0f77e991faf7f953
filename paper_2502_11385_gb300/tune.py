"""Measured autotuner: device cost tables for the planner, cached as JSON.

The planner chooses, per circuit, the fusion width (k = 1..5) and the fusion
variant (plain greedy, runs of monomial gates kept as permutation blocks,
gates on disjoint qubits packed together) with a cost model.  This module
measures that model's inputs on the GPU (sv_calibrate: picoseconds per
amplitude of a tile pass, of dense and permutation blocks of every width and
of diagonal blocks, for each arithmetic the library picks automatically),
keeps them in a JSON file keyed by the GPU's name and a hash of the kernel
sources, and installs them (sv_set_costs) so the planner scores plans with
the device's own costs.  The paper's counterparts are found by trial as well:
Aer's blocking_qubits and the Evaluator's worker count (Sec. IV-A, Listing 4).
"""
from __future__ import annotations

import hashlib
import json
import os

from . import sv

PKG = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(PKG, "_build", "autotune.json")
# the (dtype, requested arithmetic) pairs the library uses on its own:
# complex128 double-float (below 20 qubits) and tcgen05 digits, complex64
# float32 FMAs (below 23 qubits) and the tcgen05 triple split
MODES = (("c128", sv.ARITH_DF64), ("c128", sv.ARITH_TC), ("c64", sv.ARITH_NATIVE), ("c64", sv.ARITH_TC))


def kernel_key() -> str:
    """Hash of the library's sources: a table is reused only for the code it
    was measured on."""
    h = hashlib.sha256()
    csrc = os.path.join(PKG, "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def device_key() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def load(path: str = CACHE) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def save(table: dict, path: str = CACHE) -> None:
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def entry_key(dev: str, kern: str, dtype: str, arith: int) -> str:
    return f"{dev}|{kern}|{dtype}|{arith}"


def install(table: dict, dev: str, kern: str, modes=MODES) -> int:
    """Installs every cached table of this device and kernel build; returns
    how many were installed."""
    done = 0
    for dtype, arith in modes:
        e = table.get(entry_key(dev, kern, dtype, arith))
        if e:
            sv.set_costs(dtype, e["arith"], e)
            done += 1
    return done


def ensure(modes=MODES, path: str = CACHE, force: bool = False) -> dict:
    """Loads the cached tables of this GPU and kernel build, measures the
    missing ones (a fraction of a second each), saves them and installs all.
    Returns the entries used."""
    dev, kern = device_key(), kernel_key()
    table = {} if force else load(path)
    changed = False
    for dtype, arith in modes:
        k = entry_key(dev, kern, dtype, arith)
        if k not in table:
            table[k] = sv.calibrate(dtype, arith)
            changed = True
    if changed:
        save(table, path)
    install(table, dev, kern, modes)
    return {k: v for k, v in table.items() if k.startswith(f"{dev}|{kern}|")}


def clear(modes=MODES) -> None:
    """Returns every pair to the analytic model."""
    for dtype, arith in modes:
        for a in {arith, sv.ARITH_NATIVE, sv.ARITH_DF64, sv.ARITH_TC}:
            sv.set_costs(dtype, a, None)
