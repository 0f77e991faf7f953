"""Seeded synthetic circuit generators (the only module shared by the CUDA path's
tests and the CPU oracle's tests).

This module holds no statevector arithmetic: it only draws random numbers and lays
out gate lists.  A gate list is a numpy structured array with ``GATE_DTYPE``, whose
memory layout equals the C struct ``sv_gate`` (int32 op, q0, q1; three float64
parameters), so it can be handed to the C-ABI without copying.

Circuit shapes follow the workloads of the paper: full-circuit execution of a
2^n statevector (Sec. III-B) and the cut-subcircuit instances that the CutQC
Evaluator simulates (Sec. III-A, Sec. IV-A "Evaluator"), each with three upstream
measurement bases and four downstream initialisations per cut wire (Fig. 1,
Eqs. 3.2-3.6).  The paper's own circuits come from public suites that are not
reproduced here; these seeded families stand in for their shapes.

Randomness: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014); a uniform double is (x >> 11) * 2^-53.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Gate opcodes of the C-ABI (sv_op).
H, X, Y, Z, S, T, RX, RY, RZ, U3, CX, CZ, RZZ, SWAP = range(14)
OP_NAMES = ["H", "X", "Y", "Z", "S", "T", "RX", "RY", "RZ", "U3", "CX", "CZ", "RZZ", "SWAP"]
TWO_QUBIT = frozenset({CX, CZ, RZZ, SWAP})

GATE_DTYPE = np.dtype(
    [("op", "<i4"), ("q0", "<i4"), ("q1", "<i4"),
     ("theta", "<f8"), ("phi", "<f8"), ("lam", "<f8")], align=True)
assert GATE_DTYPE.itemsize == 40

MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator: state += golden gamma, then two xor-shift-multiply
    mixing rounds (Steele, Lea, Flood 2014)."""

    def __init__(self, seed: int):
        self.x = seed & MASK64

    def next_u64(self) -> int:
        self.x = (self.x + 0x9E3779B97F4A7C15) & MASK64
        z = self.x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def below(self, k: int) -> int:
        """Integer in [0, k) as floor(u * k)."""
        return min(int(self.uniform() * k), k - 1)


def gates(rows) -> np.ndarray:
    """Build a gate array from (op, q0, q1, theta, phi, lam) tuples."""
    arr = np.zeros(len(rows), dtype=GATE_DTYPE)
    for i, r in enumerate(rows):
        op, q0, q1 = r[0], r[1], r[2]
        th, ph, la = (tuple(r[3:]) + (0.0, 0.0, 0.0))[:3]
        arr[i] = (op, q0, q1, th, ph, la)
    return arr


def concat(*parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=GATE_DTYPE) for p in parts])


def ghz_prefix(n: int) -> np.ndarray:
    """H on qubit 0 followed by the CX chain CX(0,1), CX(1,2), ..., CX(n-2,n-1)."""
    rows = [(H, 0, -1)]
    rows += [(CX, q, q + 1) for q in range(n - 1)]
    return gates(rows)


def brickwork_angles(n: int, depth: int, seed: int) -> np.ndarray:
    """(depth, n, 3) array of U3 angles, drawn layer-major, qubit-major, in the
    order (theta, phi, lambda), each 2*pi*u."""
    rng = SplitMix64(seed)
    a = np.empty((depth, n, 3))
    for l in range(depth):
        for q in range(n):
            for k in range(3):
                a[l, q, k] = 2.0 * math.pi * rng.uniform()
    return a


def brickwork(n: int, depth: int, seed: int, mask=None) -> np.ndarray:
    """Random 1-D brickwork: layer l is U3 on every qubit, then CZ on (q, q+1)
    for q = l (mod 2), q+1 < n, open chain.  ``mask(l, q)`` may drop a gate
    (U3 when called with q1=None) for the cuttable variant."""
    ang = brickwork_angles(n, depth, seed)
    rows = []
    for l in range(depth):
        for q in range(n):
            rows.append((U3, q, -1, *ang[l, q]))
        for q in range(l % 2, n - 1, 2):
            if mask is not None and mask(l, q):
                continue
            rows.append((CZ, q, q + 1))
    return gates(rows)


def inverse(g: np.ndarray) -> np.ndarray:
    """Gate list of the inverse circuit: gates reversed, each replaced by its
    inverse (U3(t,p,l)^-1 = U3(-t,-l,-p); rotations negate the angle; S, T map
    to U3(0,0,-pi/2), U3(0,0,-pi/4); H, X, Y, Z, CX, CZ, SWAP are self-inverse)."""
    rows = []
    for r in g[::-1]:
        op, q0, q1 = int(r["op"]), int(r["q0"]), int(r["q1"])
        th, ph, la = float(r["theta"]), float(r["phi"]), float(r["lam"])
        if op == U3:
            rows.append((U3, q0, q1, -th, -la, -ph))
        elif op in (RX, RY, RZ, RZZ):
            rows.append((op, q0, q1, -th))
        elif op == S:
            rows.append((U3, q0, -1, 0.0, 0.0, -math.pi / 2))
        elif op == T:
            rows.append((U3, q0, -1, 0.0, 0.0, -math.pi / 4))
        else:
            rows.append((op, q0, q1))
    return gates(rows)


def qft_basis(n: int, j: int) -> np.ndarray:
    """Circuit preparing QFT|j> from |0...0>: X gates set the basis state j, then
    the textbook QFT (H and controlled phases, most significant qubit first)
    followed by the bit-reversal SWAPs.  The controlled phase CP(phi) on
    (c, t) is P(phi/2) on c, CX, P(-phi/2) on t, CX, P(phi/2) on t, with
    P(x) = U3(0, 0, x)."""
    rows = [(X, q, -1) for q in range(n) if (j >> q) & 1]

    def cp(phi, c, t):
        return [(U3, c, -1, 0.0, 0.0, phi / 2), (CX, c, t),
                (U3, t, -1, 0.0, 0.0, -phi / 2), (CX, c, t),
                (U3, t, -1, 0.0, 0.0, phi / 2)]

    for tq in range(n - 1, -1, -1):
        rows.append((H, tq, -1))
        for cq in range(tq - 1, -1, -1):
            rows += cp(math.pi / (1 << (tq - cq)), cq, tq)
    for q in range(n // 2):
        rows.append((SWAP, q, n - 1 - q))
    return gates(rows)


def random_regular_graph(n: int, seed: int, degree: int = 3):
    """Random graph by the pairing (configuration) model with restarts on any
    self-loop or repeated edge.  When n*degree is odd (no such regular graph
    exists) vertex n-1 gets degree-1 stubs.  Stubs are shuffled by Fisher-Yates
    with j = floor(u*(i+1)) and paired consecutively; edges are returned sorted
    as (a, b) with a < b."""
    rng = SplitMix64(seed)
    degs = [degree] * n
    if (n * degree) % 2:
        degs[n - 1] = degree - 1
    stubs0 = [v for v in range(n) for _ in range(degs[v])]
    for _attempt in range(100000):
        stubs = list(stubs0)
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.below(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for k in range(0, len(stubs), 2):
            a, b = stubs[k], stubs[k + 1]
            if a == b:
                ok = False
                break
            e = (min(a, b), max(a, b))
            if e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("pairing model failed to produce a simple graph")


def qaoa(n: int, p: int, seed: int):
    """QAOA circuit on a seeded random 3-regular graph: H on every qubit, then
    for each layer l: RZZ(gamma_l) on every edge (sorted edge order) and
    RX(beta_l) on every qubit.  gamma_l, beta_l ~ U[0, pi), drawn as
    gamma_1, beta_1, gamma_2, beta_2, ... from the stream that follows the
    graph draw.  Returns (gates, edges, gammas, betas)."""
    rng = SplitMix64(seed)
    edges = random_regular_graph(n, rng.next_u64())
    gam, bet = [], []
    for _ in range(p):
        gam.append(math.pi * rng.uniform())
        bet.append(math.pi * rng.uniform())
    rows = [(H, q, -1) for q in range(n)]
    for l in range(p):
        rows += [(RZZ, a, b, gam[l]) for (a, b) in edges]
        rows += [(RX, q, -1, bet[l]) for q in range(n)]
    return gates(rows), edges, gam, bet


# ---------------------------------------------------------------------------
# Cut-subcircuit variants (Sec. III-A, Fig. 1, Eqs. 3.2-3.7).
# Upstream cut outputs are measured in I/Z (nothing appended), X (H) or
# Y (S^dagger then H).  Downstream cut inputs start in |0> (nothing), |1> (X),
# |+> (H) or |+i> (H then S).  Digit j of a variant index is for cut wire j.
# ---------------------------------------------------------------------------
MEAS_BASES = ("I", "X", "Y")
INIT_STATES = ("0", "1", "+", "+i")


def meas_suffix(qubit: int, basis: str):
    if basis == "I":
        return []
    if basis == "X":
        return [(H, qubit, -1)]
    if basis == "Y":
        return [(U3, qubit, -1, 0.0, 0.0, -math.pi / 2), (H, qubit, -1)]
    raise ValueError(basis)


def init_prefix(qubit: int, state: str):
    if state == "0":
        return []
    if state == "1":
        return [(X, qubit, -1)]
    if state == "+":
        return [(H, qubit, -1)]
    if state == "+i":
        return [(H, qubit, -1), (S, qubit, -1)]
    raise ValueError(state)


def digits(index: int, base: int, count: int):
    return [(index // base ** j) % base for j in range(count)]


@dataclass
class CutCircuit:
    """A circuit split at wire cuts into an upstream part A and a downstream
    part B.  Qubits of A are global qubits 0..width_a-1; qubits of B are global
    qubits offset_b..offset_b+width_b-1 (B's local qubit = global - offset_b).
    ``cut_qubits`` are global qubits that end A and begin B."""
    n: int
    body_a: np.ndarray      # gates of A on A-local qubits
    body_b: np.ndarray      # gates of B on B-local qubits
    width_a: int
    width_b: int
    offset_b: int
    cut_qubits: tuple
    full: np.ndarray        # the uncut circuit on global qubits

    @property
    def n_cuts(self):
        return len(self.cut_qubits)

    def upstream_variant(self, index: int) -> np.ndarray:
        ds = digits(index, 3, self.n_cuts)
        rows = []
        for j, q in enumerate(self.cut_qubits):
            rows += meas_suffix(q, MEAS_BASES[ds[j]])
        return concat(self.body_a, gates(rows)) if rows else self.body_a.copy()

    def downstream_variant(self, index: int) -> np.ndarray:
        ds = digits(index, 4, self.n_cuts)
        rows = []
        for j, q in enumerate(self.cut_qubits):
            rows += init_prefix(q - self.offset_b, INIT_STATES[ds[j]])
        return concat(gates(rows), self.body_b) if rows else self.body_b.copy()

    def upstream_variants(self):
        return [self.upstream_variant(i) for i in range(3 ** self.n_cuts)]

    def downstream_variants(self):
        return [self.downstream_variant(i) for i in range(4 ** self.n_cuts)]


def cuttable_brickwork(n: int, depth: int, seed: int, cut_lo: int, n_cuts: int,
                       switch_layer: int) -> CutCircuit:
    """Brickwork that can be cut at ``n_cuts`` wires cut_lo..cut_lo+n_cuts-1.

    Layers [0, switch_layer): A holds qubits 0..cut_hi (cut_hi = cut_lo+n_cuts-1),
    B holds qubits cut_hi+1..n-1, and CZ(cut_hi, cut_hi+1) is dropped.
    Layers [switch_layer, depth): A holds qubits 0..cut_lo-1, B holds
    cut_lo..n-1, and CZ(cut_lo-1, cut_lo) is dropped.  The cut wires pass from
    A to B between layer switch_layer-1 and switch_layer.  At n=40, depth 12,
    cut_lo=18, 3 cuts, switch 6 this gives widths 21 and 22."""
    cut_hi = cut_lo + n_cuts - 1

    def dropped(l, q):
        if l < switch_layer:
            return q == cut_hi
        return q == cut_lo - 1

    ang = brickwork_angles(n, depth, seed)
    full, a_rows, b_rows = [], [], []
    off_b = cut_lo
    for l in range(depth):
        a_max = cut_hi if l < switch_layer else cut_lo - 1
        for q in range(n):
            g = (U3, q, -1, *ang[l, q])
            full.append(g)
            if q <= a_max:
                a_rows.append(g)
            else:
                b_rows.append((U3, q - off_b, -1, *ang[l, q]))
        for q in range(l % 2, n - 1, 2):
            if dropped(l, q):
                continue
            full.append((CZ, q, q + 1))
            if q + 1 <= a_max:
                a_rows.append((CZ, q, q + 1))
            else:
                b_rows.append((CZ, q - off_b, q + 1 - off_b))
    return CutCircuit(n=n, body_a=gates(a_rows), body_b=gates(b_rows),
                      width_a=cut_hi + 1, width_b=n - cut_lo, offset_b=off_b,
                      cut_qubits=tuple(range(cut_lo, cut_hi + 1)), full=gates(full))


# ---------------------------------------------------------------------------
# Named workloads.
# ---------------------------------------------------------------------------
def workload_brickwork12():
    """12 qubits, brickwork depth 10, seed 1 (175 gates), complex128, unfused."""
    return brickwork(12, 10, seed=1)


def workload_ghz_brickwork(n=30, depth=20, seed=2):
    """GHZ prefix then brickwork depth 20, seed 2 (920 gates at n=30)."""
    return concat(ghz_prefix(n), brickwork(n, depth, seed))


def workload_qaoa(n=32, p=2, seed=3):
    return qaoa(n, p, seed)


def workload_cut40(seed=4):
    """40-qubit brickwork, depth 12, cut at wires 18, 19, 20 into 21 + 22 qubits."""
    return cuttable_brickwork(40, 12, seed, cut_lo=18, n_cuts=3, switch_layer=6)


@dataclass
class Request:
    rid: int
    arrival: float          # seconds after stream start
    n: int
    dtype: str              # "c64" or "c128"
    family: str             # "brickwork" or "qaoa"
    depth: int
    gates: np.ndarray


def serving_stream(count: int, rate: float, seed: int = 5, wmin=10, wmax=30,
                   dmin=5, dmax=40):
    """Poisson request stream: exponential gaps with mean 1/rate; width
    floor(exp(U[ln wmin, ln(wmax+1)))); depth uniform on dmin..dmax; 50 %
    brickwork of that depth, 50 % QAOA with p = max(1, depth // 5); dtype 50/50.
    Request i draws its circuit from seed * 2^32 + i."""
    rng = SplitMix64(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - rng.uniform()) / rate
        w = int(math.exp(math.log(wmin) + rng.uniform() * (math.log(wmax + 1) - math.log(wmin))))
        w = max(wmin, min(wmax, w))
        d = dmin + rng.below(dmax - dmin + 1)
        fam = "brickwork" if rng.uniform() < 0.5 else "qaoa"
        dt = "c64" if rng.uniform() < 0.5 else "c128"
        sub = (seed << 32) + i
        if fam == "brickwork":
            g = brickwork(w, d, sub)
        else:
            g = qaoa(w, max(1, d // 5), sub)[0]
        out.append(Request(i, t, w, dt, fam, d, g))
    return out


# ---------------------------------------------------------------------------
# The paper's benchmark families (Sec. V-B), as generators written from their
# defining papers onto this gate set.  T^dagger = U3(0, 0, -pi/4); sqrt(X),
# sqrt(Y) are RX(pi/2), RY(pi/2) (equal up to a global phase).
# ---------------------------------------------------------------------------
def _tdg(q):
    return (U3, q, -1, 0.0, 0.0, -math.pi / 4)


def toffoli(a: int, b: int, t: int):
    """CCX(a, b -> t) from H, T, T^dagger and six CX (the standard exact
    Clifford+T decomposition)."""
    return [(H, t, -1), (CX, b, t), _tdg(t), (CX, a, t), (T, t, -1), (CX, b, t), _tdg(t), (CX, a, t),
            (T, b, -1), (T, t, -1), (H, t, -1), (CX, a, b), (T, a, -1), _tdg(b), (CX, a, b)]


def cuccaro_adder(m: int, a_val: int = None, b_val: int = None):
    """Ripple-carry adder of Cuccaro, Draper, Kutin and Moulton (2004) on two
    m-bit registers with one ancilla and a carry-out: 2m + 2 qubits.
    Layout: qubit 0 = carry-in ancilla c, qubits 1 + 2i = a_i, 2 + 2i = b_i,
    qubit 2m + 1 = carry-out z.  Computes b <- a + b (mod 2^m), z <- carry.
    MAJ(c, b, a) = CX(a, b) CX(a, c) CCX(c, b -> a);
    UMA(c, b, a) = CCX(c, b -> a) CX(a, c) CX(c, b).
    Optional a_val / b_val prepend X gates that load basis inputs."""
    n = 2 * m + 2
    A = lambda i: 1 + 2 * i
    B = lambda i: 2 + 2 * i
    rows = []
    if a_val is not None:
        rows += [(X, A(i), -1) for i in range(m) if (a_val >> i) & 1]
    if b_val is not None:
        rows += [(X, B(i), -1) for i in range(m) if (b_val >> i) & 1]

    def maj(c, b, a):
        return [(CX, a, b), (CX, a, c)] + toffoli(c, b, a)

    def uma(c, b, a):
        return toffoli(c, b, a) + [(CX, a, c), (CX, c, b)]

    carries = [0] + [A(i) for i in range(m - 1)]
    for i in range(m):
        rows += maj(carries[i], B(i), A(i))
    rows.append((CX, A(m - 1), n - 1))
    for i in range(m - 1, -1, -1):
        rows += uma(carries[i], B(i), A(i))
    return gates(rows)


def adder_output_index(m: int, a_val: int, b_val: int) -> int:
    """Basis index the adder maps |a, b> to: a unchanged, b = a + b mod 2^m,
    carry-out set, ancilla back to 0."""
    s = a_val + b_val
    idx = 0
    for i in range(m):
        idx |= ((a_val >> i) & 1) << (1 + 2 * i)
        idx |= ((s >> i) & 1) << (2 + 2 * i)
    idx |= ((s >> m) & 1) << (2 * m + 1)
    return idx


def bernstein_vazirani(n: int, secret: int):
    """Bernstein-Vazirani (1993): n - 1 data qubits (0..n-2) and an ancilla
    (n-1) prepared in |->; the oracle CX(i, ancilla) for every set bit of the
    secret; H on the data qubits reads the secret out with probability 1."""
    anc = n - 1
    rows = [(X, anc, -1), (H, anc, -1)] + [(H, q, -1) for q in range(n - 1)]
    rows += [(CX, q, anc) for q in range(n - 1) if (secret >> q) & 1]
    rows += [(H, q, -1) for q in range(n - 1)]
    return gates(rows)


def aqft(n: int, degree: int, j: int = 0):
    """Approximate QFT (Barenco, Ekert, Suominen, Torma 1996) of the basis state
    |j>: the QFT with only the controlled phases between qubits at distance
    <= degree kept (degree >= n - 1 gives the exact QFT), then bit reversal."""
    rows = [(X, q, -1) for q in range(n) if (j >> q) & 1]

    def cp(phi, c, t):
        return [(U3, c, -1, 0.0, 0.0, phi / 2), (CX, c, t),
                (U3, t, -1, 0.0, 0.0, -phi / 2), (CX, c, t),
                (U3, t, -1, 0.0, 0.0, phi / 2)]

    for tq in range(n - 1, -1, -1):
        rows.append((H, tq, -1))
        for cq in range(tq - 1, -1, -1):
            if tq - cq <= degree:
                rows += cp(math.pi / (1 << (tq - cq)), cq, tq)
    for q in range(n // 2):
        rows.append((SWAP, q, n - 1 - q))
    return gates(rows)


def hwea(n: int, layers: int, seed: int):
    """Hardware-efficient ansatz (Moll et al. 2018 style): per layer RY and RZ
    on every qubit with seeded angles, then a CX ladder CX(q, q+1)."""
    rng = SplitMix64(seed)
    rows = []
    for _ in range(layers):
        for q in range(n):
            rows.append((RY, q, -1, 2 * math.pi * rng.uniform()))
            rows.append((RZ, q, -1, 2 * math.pi * rng.uniform()))
        rows += [(CX, q, q + 1) for q in range(n - 1)]
    return gates(rows)


def supremacy(rows_: int, cols: int, cycles: int, seed: int):
    """2-D random circuit in the style of Boixo et al. (2018) on a rows x cols
    grid (qubit r*cols + c): H on every qubit, then per cycle CZ on one of
    eight edge patterns (cycling horizontal / vertical, even / odd offsets)
    and, on qubits outside this cycle's CZs, a seeded single-qubit gate from
    {sqrt(X), sqrt(Y), T}, never repeating the qubit's previous one."""
    rng = SplitMix64(seed)
    n = rows_ * cols
    q = lambda r, c: r * cols + c
    out = [(H, i, -1) for i in range(n)]
    last = [-1] * n
    for cyc in range(cycles):
        pat = cyc % 8
        horiz = pat in (0, 1, 4, 5)
        par, off = pat % 2, (pat // 2) % 2
        edges = []
        for r in range(rows_):
            for c in range(cols):
                if horiz and c + 1 < cols and (c % 2) == par and (r % 2) == off:
                    edges.append((q(r, c), q(r, c + 1)))
                if not horiz and r + 1 < rows_ and (r % 2) == par and (c % 2) == off:
                    edges.append((q(r, c), q(r + 1, c)))
        busy = set()
        for a, b in edges:
            out.append((CZ, a, b))
            busy |= {a, b}
        for i in range(n):
            if i in busy:
                continue
            choices = [k for k in range(3) if k != last[i]]
            k = choices[rng.below(len(choices))]
            last[i] = k
            out.append([(RX, i, -1, math.pi / 2), (RY, i, -1, math.pi / 2), (T, i, -1)][k])
    return gates(out)
