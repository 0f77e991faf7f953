"""Pin of the cut reconstruction (Sec. III-A, Eqs. 3.2-3.7): simulating every
upstream and downstream variant with the oracle and reconstructing must give
the uncut circuit's probabilities (the identity is exact; only rounding
differs)."""
import numpy as np
import pytest

import oracle
from oracle import cut
from paper_2502_11385_gb300 import workloads as W


@pytest.mark.parametrize("n,depth,cut_lo,k,switch", [(6, 4, 2, 1, 2), (9, 5, 3, 2, 2), (10, 6, 4, 3, 3)])
def test_cut_identity(n, depth, cut_lo, k, switch):
    cc = W.cuttable_brickwork(n, depth, 100 + n, cut_lo=cut_lo, n_cuts=k, switch_layer=switch)
    assert cc.width_a + cc.width_b == n + k
    p_up = [oracle.probabilities(oracle.run(cc.width_a, g)) for g in cc.upstream_variants()]
    p_down = [oracle.probabilities(oracle.run(cc.width_b, g)) for g in cc.downstream_variants()]
    rec = cut.reconstruct(p_up, p_down, cc.width_a, list(cc.cut_qubits))
    full = oracle.probabilities(oracle.run(n, cc.full))
    assert np.abs(rec - full).max() < 1e-13
    assert abs(rec.sum() - 1) < 1e-12


def test_cut_reconstruction_catches_wrong_init_state():
    """Using |-> instead of |+i> for the fourth initialisation (the list in
    Sec. III-A) breaks the identity, so the pin distinguishes the readings."""
    n, depth = 6, 4
    cc = W.cuttable_brickwork(n, depth, 7, cut_lo=2, n_cuts=1, switch_layer=2)
    p_up = [oracle.probabilities(oracle.run(cc.width_a, g)) for g in cc.upstream_variants()]
    downs = cc.downstream_variants()
    minus = W.concat(W.gates([(W.X, 0, -1), (W.H, 0, -1)]), cc.body_b)   # |->
    p_down = [oracle.probabilities(oracle.run(cc.width_b, g)) for g in downs[:3] + [minus]]
    rec = cut.reconstruct(p_up, p_down, cc.width_a, list(cc.cut_qubits))
    full = oracle.probabilities(oracle.run(n, cc.full))
    assert np.abs(rec - full).max() > 1e-3
