"""Sharded statevector across ranks: the multi-GPU full-circuit form of the
paper (Sec. III-B, Fig. 3b).

A 2^n state is split over P = 2^g ranks by its top g qubit positions: rank r
holds the 2^(n-g) amplitudes whose physical index has r in its top g bits.
A logical-to-physical map records where every qubit currently sits.  Gates
whose qubits all sit at local positions run on the rank's chunk as one
circuit (the local applier: the CUDA library on a GPU rank).  A gate that
needs a global position is served in one of two ways:

- diagonal gates (Z, S, T, RZ, CZ, RZZ) need no data: the global qubit's
  value is the rank's bit, so they become local gates (CZ with a global
  control becomes Z on the local qubit; RZZ becomes RZ(+-theta)) or a phase
  of the whole chunk;
- any other gate swaps the global qubit with a local one first: the
  pairwise half-chunk exchange of Fig. 3b.  Rank r and its partner
  r ^ 2^b trade the halves where the local qubit differs from their bit b,
  pipelined in 2^c sub-chunks through one buffer (send a sub-chunk, receive
  the partner's into the buffer, copy it into place), so the exchange needs
  1/2^(c+1) of a chunk of extra memory.  The local qubit chosen is the one
  whose next use lies furthest ahead.  A rank's pending phase is applied
  before every exchange (the halves that move carry it).

At the end the map is restored to the identity (exchanges for the global
positions, SWAP gates for the local ones), so chunk r is amplitudes
[r 2^(n-g), (r+1) 2^(n-g)) of the state and probabilities concatenate in
rank order; the norm is one all-reduce.  Transfers use torch.distributed
point-to-point calls (NCCL between GPUs, gloo on the host), never a
collective in the data path except that all-reduce.
"""
from __future__ import annotations

import math

import numpy as np

from . import workloads as W

DIAGONAL = {W.Z, W.S, W.T, W.RZ, W.CZ, W.RZZ}


def _phase_gates(q: int, lam: float):
    """Gates that multiply the whole state by e^{i lam}: P(lam) X P(lam) X on
    qubit q (P(lam) = U3(0, 0, lam) = diag(1, e^{i lam})), in list order."""
    p = (W.U3, q, -1, 0.0, 0.0, lam)
    return [(W.X, q, -1), p, (W.X, q, -1), p]


class ShardedState:
    """One rank's part of an n-qubit state sharded over the process group.

    chunk: this rank's amplitudes, a 1-D complex tensor of 2^(n - g)
        elements (on the rank's GPU with NCCL, on the host with gloo),
        initialised by the caller (reset() gives |0...0>).
    local_apply(chunk, n_local, gates): applies a gate list (workloads gate
        records, positions in 0..n_local-1) to the chunk in place.
    sub_chunk_log2: c, the exchange is pipelined in 2^c sub-chunks.
    """

    def __init__(self, n: int, chunk, group=None, local_apply=None, sub_chunk_log2: int = 2):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        g = int(round(math.log2(self.world)))
        if 1 << g != self.world:
            raise ValueError("the number of ranks must be a power of two")
        if n - g < 2:
            raise ValueError("each rank needs at least 2 local qubits")
        self.n, self.g, self.nl = n, g, n - g
        if chunk.numel() != 1 << self.nl:
            raise ValueError("chunk must hold 2^(n - g) amplitudes")
        self.chunk = chunk
        self.local_apply = local_apply if local_apply is not None else _library_apply
        self.c = max(0, int(sub_chunk_log2))
        self.pos = list(range(n))        # logical qubit -> physical position
        self.at = list(range(n))         # physical position -> logical qubit
        self.phase = 0.0                 # pending e^{i phase} of this rank's chunk
        self.exchanges = 0
        self.bytes_sent = 0

    # -- state --------------------------------------------------------------
    def reset(self):
        self.chunk.zero_()
        if self.rank == 0:
            self.chunk[0] = 1
        self.pos = list(range(self.n))
        self.at = list(range(self.n))
        self.phase = 0.0

    def _bit(self, position: int) -> int:
        """Value of a global physical position on this rank."""
        return (self.rank >> (position - self.nl)) & 1

    # -- the exchange (Fig. 3b) ---------------------------------------------
    def _swap_positions(self, pg: int, pl: int):
        """Exchanges global position pg with local position pl: amplitude
        (pg = x, pl = y) moves to (pg = y, pl = x).  Only entries with x != y
        move, between this rank and partner rank ^ 2^(pg - nl)."""
        import torch
        b = pg - self.nl
        partner = self.rank ^ (1 << b)
        x = (self.rank >> b) & 1
        # entries of this rank with pl = 1 - x leave; they are replaced by the
        # partner's entries with pl = x, which land at pl = 1 - x here
        v = self.chunk.view(1 << (self.nl - pl - 1), 2, 1 << pl)
        half = v[:, 1 - x, :]
        rows = half.shape[0]
        parts = min(1 << self.c, rows) if rows > 1 else 1
        step = rows // parts
        buf = None
        for j in range(parts):
            sl = slice(j * step, (j + 1) * step if j + 1 < parts else rows)
            out = half[sl].contiguous()
            if buf is None or buf.shape != out.shape:
                buf = torch.empty_like(out)
            # complex data travels as its real pairs; the lower rank sends first
            # and the higher receives first, so blocking calls cannot deadlock
            o, r = torch.view_as_real(out), torch.view_as_real(buf)
            if self.rank < partner:
                self.dist.send(o, partner, group=self.group)
                self.dist.recv(r, partner, group=self.group)
            else:
                self.dist.recv(r, partner, group=self.group)
                self.dist.send(o, partner, group=self.group)
            half[sl].copy_(buf)
            self.bytes_sent += out.numel() * out.element_size()
        qg, ql = self.at[pg], self.at[pl]
        self.at[pg], self.at[pl] = ql, qg
        self.pos[qg], self.pos[ql] = pl, pg
        self.exchanges += 1

    def _make_local(self, qubits, upcoming):
        """Brings every qubit of `qubits` to a local position, swapping each
        global one with the local qubit (not in `qubits`) whose next use in
        `upcoming` lies furthest ahead."""
        for q in qubits:
            if self.pos[q] < self.nl:
                continue
            next_use = {}
            for i, (op, q0, q1) in enumerate(upcoming):
                for u in (q0, q1):
                    if u >= 0 and u not in next_use:
                        next_use[u] = i
            best, best_t = None, -1
            for p in range(self.nl):
                lq = self.at[p]
                if lq in qubits:
                    continue
                t = next_use.get(lq, 1 << 30)
                if t > best_t:
                    best, best_t = p, t
            self._swap_positions(self.pos[q], best)

    # -- gates ----------------------------------------------------------------
    def _diag_local(self, op, q0, q1, th):
        """A diagonal gate touching a global position as local gates and a
        phase of the chunk; returns the local gate rows."""
        p0 = self.pos[q0]
        p1 = self.pos[q1] if q1 >= 0 else -1
        g0, g1 = p0 >= self.nl, p1 >= self.nl
        s0 = self._bit(p0) if g0 else None
        s1 = self._bit(p1) if (p1 >= 0 and g1) else None
        if op in (W.Z, W.S, W.T, W.RZ):  # one global qubit with value s0
            lam = {W.Z: math.pi, W.S: math.pi / 2, W.T: math.pi / 4}.get(op)
            if op == W.RZ:
                self.phase += th / 2 if s0 else -th / 2
            elif s0:
                self.phase += lam
            return []
        if op == W.CZ:
            if g0 and g1:
                if s0 and s1:
                    self.phase += math.pi
                return []
            s, pl = (s0, p1) if g0 else (s1, p0)
            return [(W.Z, pl, -1)] if s else []
        # RZZ(th) = exp(-i th/2 Z(x) Z): with a global qubit of sign (-1)^s it is
        # RZ(+-th) on the other; with two it is the phase exp(-i th/2 (-1)^(s0+s1))
        if g0 and g1:
            self.phase += -th / 2 if (s0 ^ s1) == 0 else th / 2
            return []
        s, pl = (s0, p1) if g0 else (s1, p0)
        return [(W.RZ, pl, -1, th if s == 0 else -th)]

    def apply(self, gates):
        """Applies a gate list (logical qubits), in order."""
        rows = [(int(r["op"]), int(r["q0"]), int(r["q1"]), float(r["theta"]), float(r["phi"]),
                 float(r["lam"])) for r in np.asarray(gates)]
        upcoming = [(op, q0, q1) for op, q0, q1, *_ in rows]
        segment = []

        def flush():
            # the chunk's pending phase goes out with the segment: an exchange
            # moves half the chunk to a rank whose phase differs
            segment.extend(self._take_phase())
            if segment:
                self.local_apply(self.chunk, self.nl, W.gates(segment))
                segment.clear()

        for i, (op, q0, q1, th, ph, la) in enumerate(rows):
            qs = (q0,) if q1 < 0 else (q0, q1)
            if all(self.pos[q] < self.nl for q in qs):
                p1 = self.pos[q1] if q1 >= 0 else -1
                segment.append((op, self.pos[q0], p1, th, ph, la))
                continue
            if op in DIAGONAL:
                segment += self._diag_local(op, q0, q1, th)
                continue
            flush()
            self._make_local(qs, upcoming[i + 1:])
            p1 = self.pos[q1] if q1 >= 0 else -1
            segment.append((op, self.pos[q0], p1, th, ph, la))
        flush()

    def _take_phase(self):
        """Gates applying this rank's pending phase (none if it is 1)."""
        lam = math.remainder(self.phase, 2 * math.pi)
        self.phase = 0.0
        return _phase_gates(0, lam) if lam != 0.0 else []

    def finish(self):
        """Restores the identity map (exchanges for global positions, local
        SWAPs for the rest) and applies this rank's pending phase, so chunk r
        holds amplitudes [r 2^(n-g), (r+1) 2^(n-g))."""
        pending = self._take_phase()
        if pending:  # before any exchange
            self.local_apply(self.chunk, self.nl, W.gates(pending))
        for pg in range(self.nl, self.n):  # logical qubit pg belongs at position pg
            if self.pos[pg] >= self.nl and self.pos[pg] != pg:
                self._swap_positions(self.pos[pg], 0)  # another global position: through local 0
            if self.pos[pg] != pg:
                self._swap_positions(pg, self.pos[pg])
        swaps = []
        for p in range(self.nl):
            q = self.at[p]
            if q != p:  # SWAP positions p and pos[p] (where qubit p sits)
                other = self.pos[p]
                swaps.append((W.SWAP, p, other))
                self.at[p], self.at[other] = p, q
                self.pos[p], self.pos[q] = p, other
        if swaps:
            self.local_apply(self.chunk, self.nl, W.gates(swaps))

    def norm(self) -> float:
        """sum |a|^2 over all ranks (one all-reduce)."""
        import torch
        local = torch.tensor([float((self.chunk.abs() ** 2).sum())], dtype=torch.float64)
        self.dist.all_reduce(local, group=self.group)
        return float(local.item())


def _library_apply(chunk, n_local, gates):
    """The default local applier: the CUDA library on the chunk in place."""
    from . import sv
    dt = "c128" if chunk.dtype.itemsize == 16 else "c64"
    with sv.State.from_tensor(chunk, n_local, dt) as s:
        s.apply_circuit(gates)
