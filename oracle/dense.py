"""Brute-force dense-unitary simulation for n <= 8 -- TEST INFRASTRUCTURE ONLY.

Independent of sv_oracle.c: every gate's matrix is written out here again and
embedded into the full 2^n x 2^n operator with numpy.kron, qubit q sitting at
Kronecker position n-1-q so that index bit q is qubit q (little-endian, the
convention of the probabilities call in Listings 2 and 3).  A two-qubit gate
G on (q0, q1), with local index b(q0) + 2 b(q1), is expanded as
sum_{r,c} G[r,c] * kron-product of the per-qubit outer products
|r_j><c_j|.  The circuit unitary is the product of these operators, last
gate leftmost.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

I2 = np.eye(2, dtype=complex)


def gate_matrix(op: int, theta=0.0, phi=0.0, lam=0.0) -> np.ndarray:
    c, s = math.cos(theta / 2), math.sin(theta / 2)
    e = cmath.exp
    table = {
        0: np.array([[1, 1], [1, -1]]) / math.sqrt(2),
        1: np.array([[0, 1], [1, 0]]),
        2: np.array([[0, -1j], [1j, 0]]),
        3: np.array([[1, 0], [0, -1]]),
        4: np.array([[1, 0], [0, 1j]]),
        5: np.array([[1, 0], [0, e(1j * math.pi / 4)]]),
        6: np.array([[c, -1j * s], [-1j * s, c]]),
        7: np.array([[c, -s], [s, c]]),
        8: np.array([[e(-0.5j * theta), 0], [0, e(0.5j * theta)]]),
        9: np.array([[c, -e(1j * lam) * s], [e(1j * phi) * s, e(1j * (phi + lam)) * c]]),
    }
    if op in table:
        return np.asarray(table[op], dtype=complex)
    m = np.zeros((4, 4), dtype=complex)
    if op == 10:      # CX, control q0 (local bit 0), target q1 (local bit 1)
        for a in range(4):
            b0, b1 = a & 1, a >> 1
            m[b0 | ((b1 ^ b0) << 1), a] = 1
    elif op == 11:    # CZ
        m = np.diag([1, 1, 1, -1]).astype(complex)
    elif op == 12:    # RZZ
        m = np.diag([e(-0.5j * theta), e(0.5j * theta), e(0.5j * theta), e(-0.5j * theta)])
    elif op == 13:    # SWAP
        for a in range(4):
            b0, b1 = a & 1, a >> 1
            m[b1 | (b0 << 1), a] = 1
    else:
        raise ValueError(op)
    return m


def _outer(r, c):
    m = np.zeros((2, 2), dtype=complex)
    m[r, c] = 1
    return m


def embed(n: int, u: np.ndarray, qubits) -> np.ndarray:
    """Full 2^n operator of u acting on `qubits` (local bit j = qubits[j])."""
    k = len(qubits)
    full = np.zeros((1 << n, 1 << n), dtype=complex)
    for r in range(1 << k):
        for cidx in range(1 << k):
            if u[r, cidx] == 0:
                continue
            factors = []
            for q in range(n - 1, -1, -1):      # Kronecker position 0 = qubit n-1
                if q in qubits:
                    j = qubits.index(q)
                    factors.append(_outer((r >> j) & 1, (cidx >> j) & 1))
                else:
                    factors.append(I2)
            op = factors[0]
            for f in factors[1:]:
                op = np.kron(op, f)
            full += u[r, cidx] * op
    return full


def circuit_unitary(n: int, gates) -> np.ndarray:
    assert n <= 8
    U = np.eye(1 << n, dtype=complex)
    for g in gates:
        op = int(g["op"])
        qs = [int(g["q0"])] if op < 10 else [int(g["q0"]), int(g["q1"])]
        U = embed(n, gate_matrix(op, g["theta"], g["phi"], g["lam"]), qs) @ U
    return U


def run(n: int, gates, basis: int = 0) -> np.ndarray:
    e = np.zeros(1 << n, dtype=complex)
    e[basis] = 1
    return circuit_unitary(n, gates) @ e
