"""CutQC reconstruction of an uncut distribution from subcircuit-variant
probabilities -- TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Follows Sec. III-A.  One wire cut splits an operator A into four terms
(Eq. 3.2, A = (A1 + A2 + A3 + A4) / 2, Eqs. 3.3-3.6): the upstream subcircuit
is measured on the cut qubit in the I/Z basis (one circuit), the X basis or
the Y basis, and the downstream subcircuit starts the cut qubit in |0>, |1>,
|+> or |+i>.  For term i the upstream factor attributes each measured outcome
y of the cut qubit (Eq. 3.7 and the worked terms p_{1,1..4}):

    i = 1:  I + Z  ->  weight 2 for y = 0, 0 for y = 1   (I/Z variant)
    i = 2:  I - Z  ->  weight 0 for y = 0, 2 for y = 1   (I/Z variant)
    i = 3:  X      ->  weight +1 for y = 0, -1 for y = 1 (X variant)
    i = 4:  Y      ->  weight +1 for y = 0, -1 for y = 1 (Y variant)

and the downstream factor combines initialisations (worked terms p_{2,1..4}):

    i = 1: p(|0>)          i = 2: p(|1>)
    i = 3: 2 p(|+>)  - p(|0>) - p(|1>)
    i = 4: 2 p(|+i>) - p(|0>) - p(|1>)

With K cuts the factors multiply per cut and the uncut distribution is
p(x_A, x_B) = (1/2)^K sum_{i in {1..4}^K} p_1[i](x_A) p_2[i](x_B)
(the printed sum's index typo read as p_{1,i} (x) p_{2,i}).
Variant indices: upstream sum_j m_j 3^j with m_j in {0: I/Z, 1: X, 2: Y};
downstream sum_j s_j 4^j with s_j in {0: |0>, 1: |1>, 2: |+>, 3: |+i>};
digit j belongs to cut j.
"""
from __future__ import annotations

import itertools

import numpy as np

UP_BASIS = {1: 0, 2: 0, 3: 1, 4: 2}                       # term -> measurement variant digit
UP_WEIGHT = {1: (2.0, 0.0), 2: (0.0, 2.0), 3: (1.0, -1.0), 4: (1.0, -1.0)}
DOWN_WEIGHT = {1: (1.0, 0.0, 0.0, 0.0), 2: (0.0, 1.0, 0.0, 0.0),
               3: (-1.0, -1.0, 2.0, 0.0), 4: (-1.0, -1.0, 0.0, 2.0)}


def upstream_terms(p_up, width_a, cut_pos):
    """p_1[i] for every i in {1..4}^K: array (4^K, 2^(width_a - K)) indexed by
    i encoded as sum_j (i_j - 1) 4^j; the remaining (effective) qubits keep
    their order.  p_up[v] is the distribution of upstream variant v over the
    width_a qubits; cut_pos[j] is cut j's qubit inside the upstream circuit."""
    K = len(cut_pos)
    eff = [q for q in range(width_a) if q not in cut_pos]
    out = np.zeros((4 ** K, 1 << len(eff)))
    for terms in itertools.product((1, 2, 3, 4), repeat=K):
        code = sum((t - 1) * 4 ** j for j, t in enumerate(terms))
        variant = sum(UP_BASIS[t] * 3 ** j for j, t in enumerate(terms))
        p = np.asarray(p_up[variant], dtype=np.float64).reshape([2] * width_a)  # axis a <-> qubit width_a-1-a
        acc = np.zeros([2] * len(eff))
        for ys in itertools.product((0, 1), repeat=K):
            w = 1.0
            for j, t in enumerate(terms):
                w *= UP_WEIGHT[t][ys[j]]
            if w == 0.0:
                continue
            index = [slice(None)] * width_a
            for j, q in enumerate(cut_pos):
                index[width_a - 1 - q] = ys[j]
            acc = acc + w * p[tuple(index)]
        out[code] = acc.reshape(-1)
    return out


def downstream_terms(p_down, K):
    """p_2[i] for every i: array (4^K, 2^width_b)."""
    out = np.zeros((4 ** K, len(p_down[0])))
    for terms in itertools.product((1, 2, 3, 4), repeat=K):
        code = sum((t - 1) * 4 ** j for j, t in enumerate(terms))
        acc = np.zeros(len(p_down[0]))
        for inits in itertools.product(range(4), repeat=K):
            w = 1.0
            for j, t in enumerate(terms):
                w *= DOWN_WEIGHT[t][inits[j]]
            if w == 0.0:
                continue
            acc = acc + w * np.asarray(p_down[sum(s * 4 ** j for j, s in enumerate(inits))])
        out[code] = acc
    return out


def reconstruct(p_up, p_down, width_a, cut_pos):
    """Uncut distribution: index = x_A_eff + 2^(width_a - K) * x_B."""
    K = len(cut_pos)
    up = upstream_terms(p_up, width_a, cut_pos)
    down = downstream_terms(p_down, K)
    full = np.zeros((up.shape[1], down.shape[1]))
    for code in range(4 ** K):
        full += np.outer(up[code], down[code])
    return (0.5 ** K) * full.T.reshape(-1)      # x_B slow, x_A_eff fast
