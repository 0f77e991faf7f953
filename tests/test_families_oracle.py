"""The benchmark families' generators against what their defining papers fix:
the Toffoli decomposition's truth table, the Cuccaro adder's sums, the
Bernstein-Vazirani secret read-out, and the AQFT reducing to the exact QFT."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_11385_gb300 import workloads as W


def test_toffoli_truth_table():
    for a in (0, 1):
        for b in (0, 1):
            for t in (0, 1):
                basis = a | (b << 1) | (t << 2)
                psi = oracle.run(3, W.gates(W.toffoli(0, 1, 2)), basis)
                want = a | (b << 1) | ((t ^ (a & b)) << 2)
                assert abs(abs(psi[want]) - 1) < 1e-14 and abs(psi[want] - 1) < 1e-14


@pytest.mark.parametrize("m", [1, 2, 4])
def test_cuccaro_adder_adds(m):
    n = 2 * m + 2
    for a in range(1 << m):
        for b in (0, (1 << m) - 1, a ^ 1 if m > 1 else 1):
            psi = oracle.run(n, W.cuccaro_adder(m, a, b))
            idx = W.adder_output_index(m, a, b)
            assert abs(psi[idx] - 1) < 1e-12, (m, a, b)


def test_bernstein_vazirani_reads_secret():
    n, secret = 9, 0b10110101
    p = oracle.probabilities(oracle.run(n, W.bernstein_vazirani(n, secret)))
    data = oracle.marginal(oracle.run(n, W.bernstein_vazirani(n, secret)), (1 << (n - 1)) - 1)
    assert abs(data[secret] - 1) < 1e-12 and abs(p.sum() - 1) < 1e-12


def test_aqft_full_degree_is_qft():
    n, j = 7, 77
    a = oracle.run(n, W.aqft(n, n - 1, j))
    b = oracle.run(n, W.qft_basis(n, j))
    assert np.abs(a - b).max() < 1e-13
    # a lower degree drops rotations: the state changes but stays normalised
    c = oracle.run(n, W.aqft(n, 2, j))
    assert np.abs(c - b).max() > 1e-3 and abs(np.linalg.norm(c) - 1) < 1e-13


def test_hwea_and_supremacy_shapes():
    g = W.hwea(6, 3, 1)
    assert len(g) == 3 * (2 * 6 + 5)
    s = W.supremacy(3, 4, 8, 2)
    assert int(s["q0"].max()) == 11 and all(int(r["op"]) in (W.H, W.CZ, W.RX, W.RY, W.T) for r in s)
    psi = oracle.run(12, s)
    assert abs(np.linalg.norm(psi) - 1) < 1e-12
