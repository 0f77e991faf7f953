"""Pins of the CPU oracle against facts fixed outside it: textbook gate
identities (matrix exponentials from scipy), a numpy dense-unitary brute force,
closed forms (GHZ, QFT of a basis state, U U^dagger = I, norm 1, the QAOA
bit-flip symmetry) and the numbers the paper prints (Table III)."""
import cmath
import math
import os

import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from oracle import dense
from paper_2502_11385_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
ALL_OPS = list(range(14))


def test_splitmix64_reference_vector():
    # Reference output of SplitMix64 for seed 1234567 (Vigna's splitmix64.c).
    r = W.SplitMix64(1234567)
    assert [r.next_u64() for _ in range(5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423,
        4593380528125082431, 16408922859458223821]


@pytest.mark.parametrize("op", ALL_OPS)
def test_gate_unitary(op):
    rng = np.random.default_rng(op)
    for _ in range(5):
        th, ph, la = rng.uniform(-7, 7, 3)
        m = oracle.gate_matrix(op, th, ph, la)
        assert np.allclose(m @ m.conj().T, np.eye(len(m)), atol=1e-14)
        # the two independently written tables agree
        assert np.allclose(m, dense.gate_matrix(op, th, ph, la), atol=1e-15)


def test_rotations_are_pauli_exponentials():
    zz = np.diag([1, -1, -1, 1]).astype(complex)   # Z(q0) Z(q1) over b0 + 2 b1
    for th in np.linspace(-6, 6, 13):
        assert np.allclose(oracle.gate_matrix(W.RX, th), expm(-0.5j * th * PX), atol=1e-14)
        assert np.allclose(oracle.gate_matrix(W.RY, th), expm(-0.5j * th * PY), atol=1e-14)
        assert np.allclose(oracle.gate_matrix(W.RZ, th), expm(-0.5j * th * PZ), atol=1e-14)
        assert np.allclose(oracle.gate_matrix(W.RZZ, th), expm(-0.5j * th * zz), atol=1e-14)


def test_u3_is_zyz_euler():
    rng = np.random.default_rng(1)
    for _ in range(10):
        th, ph, la = rng.uniform(-7, 7, 3)
        ref = cmath.exp(0.5j * (ph + la)) * expm(-0.5j * ph * PZ) @ expm(-0.5j * th * PY) @ expm(-0.5j * la * PZ)
        assert np.allclose(oracle.gate_matrix(W.U3, th, ph, la), ref, atol=1e-14)


def test_fixed_gates_textbook():
    g = oracle.gate_matrix
    assert np.allclose(g(W.X), PX) and np.allclose(g(W.Y), PY) and np.allclose(g(W.Z), PZ)
    assert np.allclose(g(W.H), (PX + PZ) / math.sqrt(2))
    assert np.allclose(g(W.S) @ g(W.S), PZ)
    assert np.allclose(g(W.T) @ g(W.T), g(W.S))
    assert np.allclose(g(W.S), np.diag([1, 1j]))
    pi = math.pi
    assert np.allclose(g(W.U3, pi / 2, 0, pi), g(W.H), atol=1e-15)
    assert np.allclose(g(W.U3, pi, 0, pi), g(W.X), atol=1e-15)
    assert np.allclose(g(W.U3, 0, 0, pi / 2), g(W.S), atol=1e-15)
    assert np.allclose(g(W.U3, 0, 0, pi / 4), g(W.T), atol=1e-15)


def _basis_action(m, a):
    col = m[:, a]
    nz = np.flatnonzero(np.abs(col) > 0.5)
    assert len(nz) == 1
    return int(nz[0]), col[nz[0]]


def test_two_qubit_gates_on_basis_states():
    # local index = b(q0) + 2*b(q1); CX: q0 control, q1 target
    for a in range(4):
        b0, b1 = a & 1, a >> 1
        assert _basis_action(oracle.gate_matrix(W.CX), a) == (b0 | ((b1 ^ b0) << 1), 1)
        assert _basis_action(oracle.gate_matrix(W.SWAP), a) == (b1 | (b0 << 1), 1)
        assert _basis_action(oracle.gate_matrix(W.CZ), a) == (a, -1 if a == 3 else 1)
    # CZ = (I x H) CX (I x H) with H on the target q1
    hq1 = np.kron(oracle.gate_matrix(W.H), np.eye(2))   # kron order: q1 (high bit) first
    assert np.allclose(hq1 @ oracle.gate_matrix(W.CX) @ hq1, oracle.gate_matrix(W.CZ), atol=1e-15)


def _random_circuit(n, count, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(count):
        op = int(rng.integers(0, 14))
        q0 = int(rng.integers(0, n))
        q1 = -1
        if op >= W.CX:
            q1 = int(rng.choice([q for q in range(n) if q != q0]))
        rows.append((op, q0, q1, *rng.uniform(-7, 7, 3)))
    return W.gates(rows)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_oracle_vs_dense_bruteforce(n):
    count = 30 if n > 1 else 12
    g = _random_circuit(n, count, 100 + n) if n > 1 else W.gates(
        [(op, 0, -1, 0.3 * op, 0.7, -1.1) for op in range(10)])
    for basis in (0, (1 << n) - 1):
        a = oracle.run(n, g, basis)
        b = dense.run(n, g, basis)
        assert np.abs(a - b).max() < 1e-13


def test_dense_bruteforce_embedding_bit_order():
    # X on qubit q of |0..0> gives index 2^q (qubit q = index bit q).
    for n in (3, 5):
        for q in range(n):
            psi = dense.run(n, W.gates([(W.X, q, -1)]))
            assert abs(psi[1 << q] - 1) < 1e-15


@pytest.mark.parametrize("n", [1, 2, 5, 12, 20])
def test_ghz_closed_form(n):
    psi = oracle.run(n, W.ghz_prefix(n))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.abs(psi - ref).max() < 1e-15


@pytest.mark.parametrize("n,j", [(3, 5), (6, 0), (6, 37), (10, 613)])
def test_qft_of_basis_state(n, j):
    psi = oracle.run(n, W.qft_basis(n, j))
    k = np.arange(1 << n)
    ref = np.exp(2j * np.pi * j * k / (1 << n)) / math.sqrt(1 << n)
    assert np.abs(psi - ref).max() < 1e-13


def test_u_udagger_returns_to_ghz():
    n = 10
    body = W.brickwork(n, 6, 11)
    g = W.concat(W.ghz_prefix(n), body, W.inverse(body))
    psi = oracle.run(n, g)
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    assert np.abs(psi - ref).max() < 1e-13


def test_inverse_of_every_gate():
    g = _random_circuit(4, 40, 5)
    psi = oracle.run(4, W.concat(g, W.inverse(g)))
    assert abs(psi[0] - 1) < 1e-13 and np.abs(psi[1:]).max() < 1e-13


def test_probabilities_norm_marginal():
    n = 9
    psi = oracle.run(n, W.brickwork(n, 5, 3))
    p = oracle.probabilities(psi)
    assert np.allclose(p, np.abs(psi) ** 2, atol=1e-17)
    assert abs(oracle.norm(psi) - 1) < 1e-14
    assert abs(oracle.norm(psi) - math.fsum(p)) < 1e-15
    mask = 0b100100110
    m = oracle.marginal(psi, mask)
    qs = [q for q in range(n) if (mask >> q) & 1]
    t = p.reshape([2] * n)          # axis a <-> qubit n-1-a
    other = tuple(n - 1 - q for q in range(n) if q not in qs)
    ref = t.sum(axis=other)          # remaining axes: qubits in descending order
    ref = ref.transpose(list(range(len(qs)))[::-1]).reshape(-1, order="F")
    assert np.allclose(m, ref, atol=1e-16)
    assert np.allclose(oracle.marginal(psi, (1 << n) - 1), p)


def test_qaoa_bitflip_symmetry_and_cost_layer_modulus():
    n = 10
    g, edges, gam, bet = W.qaoa(n, 2, 3)
    assert len(edges) == 15 and all(sum(v in e for e in edges) == 3 for v in range(n))
    psi = oracle.run(n, g)
    x = np.arange(1 << n)
    assert np.abs(psi - psi[x ^ ((1 << n) - 1)]).max() < 1e-14
    # H on all, then one cost layer: every |a_x|^2 = 2^-n
    pre = g[: n + len(edges)]
    p = np.abs(oracle.run(n, pre)) ** 2
    assert np.abs(p - 2.0 ** -n).max() < 1e-16


def test_validate():
    assert oracle.validate(3, W.gates([(W.CX, 0, 2)])) == -1
    assert oracle.validate(3, W.gates([(W.H, 0, -1), (W.CX, 1, 1)])) == 1
    assert oracle.validate(3, W.gates([(W.H, 3, -1)])) == 0
    assert oracle.validate(3, W.gates([(99, 0, -1)])) == 0
    with pytest.raises(ValueError):
        oracle.run(3, W.gates([(W.CZ, 0, 5)]))


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _truncate_like(value, printed):
    s = printed
    if "e" in s:
        mant, exp = s.split("e")
        dec = len(mant.split(".")[1])
        scale = 10.0 ** int(exp)
        return math.floor(value / scale * 10 ** dec + 1e-9) / 10 ** dec * scale
    dec = len(s.split(".")[1])
    return math.floor(value * 10 ** dec + 1e-9) / 10 ** dec


def test_table3_bytes_per_amplitude_is_16():
    for width, printed in _golden("table3_statevector_gb.txt"):
        n = int(width)
        gb = (2 ** n) * 16 / 1e9
        assert math.isclose(_truncate_like(gb, printed), float(printed), rel_tol=1e-12), (n, gb, printed)


def test_cut_metadata_identity():
    for fam, width, w1, e1, w2, e2, k in _golden("cut_metadata.txt"):
        width, w1, e1, w2, e2, k = map(int, (width, w1, e1, w2, e2, k))
        assert e1 + e2 == width, fam
        if k >= 0:
            assert w1 + w2 == width + k, (fam, width)


def test_generators_match_stated_shapes():
    assert len(W.workload_brickwork12()) == 175
    assert len(W.workload_ghz_brickwork()) == 920
    g, edges, _, _ = W.workload_qaoa(32)
    assert len(g) == 192 and len(edges) == 48
    _, e33, _, _ = W.qaoa(33, 2, 3)
    deg = [sum(v in e for e in e33) for v in range(33)]
    assert len(e33) == 49 and deg.count(3) == 32 and deg[32] == 2
    c = W.workload_cut40()
    assert (c.width_a, c.width_b, len(c.body_a), len(c.body_b)) == (21, 22, 345, 363)
    assert c.width_a + c.width_b == 40 + c.n_cuts
    assert len(c.upstream_variants()) == 27 and len(c.downstream_variants()) == 64
