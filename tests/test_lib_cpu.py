"""Host-side checks of libsv that need no GPU: the library loads and exports
every entry point its headers declare; state sizes follow Table III; the
planner's fusion and tile passes keep every gate exactly once, in a legal
order, and compute the circuit's unitary (checked against the oracle)."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import dense
from paper_2502_11385_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sv():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv as _sv
    return _sv


def _declared():
    names = []
    for h in ("sv.h", "sv_plan.h"):
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(sv_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_exports_every_declared_symbol(sv):
    import ctypes
    lib = ctypes.CDLL(sv.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 24
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(sv.EXPORTED)
    assert "sm_103a" in sv.version()
    assert sv.status_str(sv.SV_ERR_QUBIT).startswith("qubit")


def test_state_bytes_table3(sv):
    for line in open(os.path.join(ROOT, "tests", "golden", "table3_statevector_gb.txt")):
        line = line.split("#")[0].split()
        if line:
            n = int(line[0])
            assert sv.state_bytes(n, "c128") == 16 << n
            assert sv.state_bytes(n, "c64") == 8 << n
    assert sv.state_bytes(0, "c128") == 0 and sv.state_bytes(35, "c64") == 0
    assert sv.state_bytes(34, "c128") == 16 << 34


def _random_circuit(n, count, seed, ops=range(14)):
    rng = np.random.default_rng(seed)
    ops = list(ops)
    rows = []
    for _ in range(count):
        op = int(rng.choice(ops))
        q0 = int(rng.integers(0, n))
        q1 = -1
        if op >= W.CX:
            q1 = int(rng.choice([q for q in range(n) if q != q0]))
        rows.append((op, q0, q1, *rng.uniform(-7, 7, 3)))
    return W.gates(rows)


def _plan_unitary_state(sv, plan, n):
    """Applies the plan's blocks, pass by pass, to |0..0> with dense algebra."""
    psi = np.zeros(1 << n, dtype=complex)
    psi[0] = 1
    nb = plan.summary()["n_passes"]
    for i in range(nb):
        for b in plan.pass_info(i)["blocks"]:
            blk = plan.block(b)
            m = np.diag(blk["mat"]) if blk["kind"] == sv.BLOCK_DIAG else blk["mat"]
            psi = dense.embed(n, m, blk["qubits"]) @ psi
    return psi


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("seed", [0, 1])
def test_plan_reproduces_circuit(sv, k, seed):
    n = 7
    g = _random_circuit(n, 60, seed)
    p = sv.Plan(n, "c128", g, sv.run_opts(max_fuse_k=k))
    assert p.check() == 0
    s = p.summary()
    assert s["fuse_k"] == k
    for b in range(s["n_blocks"]):
        assert 1 <= p.block(b)["k"] <= k or (k == 1 and p.block(b)["k"] == 2)
    ref = oracle.run(n, g)
    assert np.abs(_plan_unitary_state(sv, p, n) - ref).max() < 1e-12


def test_plan_multi_pass_locality(sv):
    n = 14
    g = W.concat(W.ghz_prefix(n), W.brickwork(n, 6, 9))
    p = sv.Plan(n, "c64", g, sv.run_opts(max_fuse_k=3, tile_qubits=9))
    s = p.summary()
    assert p.check() == 0 and s["n_passes"] > 1 and s["tile_qubits"] == 10  # >= coalesce + 5
    for i in range(s["n_passes"]):
        pi = p.pass_info(i)
        assert bin(pi["local_mask"]).count("1") == 10
        assert pi["local_mask"] & 0b11111 == 0b11111      # coalescing qubits always local
        for b in pi["blocks"]:
            blk = p.block(b)
            if blk["kind"] != sv.BLOCK_DIAG:
                assert all((pi["local_mask"] >> q) & 1 for q in blk["qubits"])


def test_fused_block_matrix_is_product_of_oracle_gates(sv):
    n = 5
    g = _random_circuit(n, 25, 3)
    p = sv.Plan(n, "c128", g, sv.run_opts(max_fuse_k=5))
    for b in range(p.summary()["n_blocks"]):
        blk = p.block(b)
        qs = blk["qubits"]
        d = 1 << len(qs)
        ref = np.eye(d, dtype=complex)
        for t in blk["gates"]:
            r = g[t]
            op = int(r["op"])
            u = oracle.gate_matrix(op, r["theta"], r["phi"], r["lam"])
            gq = [int(r["q0"])] + ([int(r["q1"])] if op >= W.CX else [])
            # embed into the block's local space (bit j = qs[j]) via the dense helper
            ref = dense.embed(len(qs), u, [qs.index(q) for q in gq]) @ ref
        m = np.diag(blk["mat"]) if blk["kind"] == sv.BLOCK_DIAG else blk["mat"]
        assert np.abs(m - ref).max() < 1e-13


def test_diagonal_runs_classified(sv):
    n = 6
    g = W.gates([(W.CZ, 0, 1), (W.CZ, 2, 3), (W.Z, 4, -1), (W.RZZ, 1, 2, 0.3), (W.T, 5, -1)])
    p = sv.Plan(n, "c128", g, sv.run_opts(max_fuse_k=5))
    kinds = [p.block(b)["kind"] for b in range(p.summary()["n_blocks"])]
    assert all(k == 1 for k in kinds)


@pytest.mark.parametrize("bad,code", [
    ((W.H, 6, -1), -2), ((W.CX, 1, 1), -2), ((99, 0, -1), -1), ((W.RX, 0, -1, float("nan")), -1)])
def test_plan_rejects_bad_gates(sv, bad, code):
    with pytest.raises(sv.SvError) as e:
        sv.Plan(6, "c128", W.gates([(W.H, 0, -1), bad]))
    assert e.value.code == code


def test_autotuned_plan_is_valid_for_workloads(sv):
    for n, dt, g in [(12, "c128", W.workload_brickwork12()),
                     (30, "c128", W.workload_ghz_brickwork()),
                     (30, "c64", W.workload_ghz_brickwork()),
                     (32, "c64", W.workload_qaoa(32)[0])]:
        p = sv.Plan(n, dt, g)
        assert p.check() == 0, (n, dt)
        s = p.summary()
        assert s["n_passes"] >= 1 and 1 <= s["fuse_k"] <= 5


def test_permutation_blocks_classified(sv):
    """Runs of X / Y / CX / SWAP with diagonal gates fuse into permutation
    blocks: one nonzero per row, of modulus 1 (the GHZ chain, a SWAP network,
    Paulis and S / T phases); the plan still reproduces the circuit."""
    n = 8
    rows = [(W.CX, q, q + 1) for q in range(n - 1)]
    rows += [(W.SWAP, 0, 5), (W.X, 3, -1), (W.Y, 6, -1), (W.S, 2, -1), (W.T, 7, -1), (W.CX, 7, 1), (W.CZ, 4, 6)]
    g = W.gates(rows)
    p = sv.Plan(n, "c128", g, sv.run_opts(max_fuse_k=4))
    assert p.check() == 0
    kinds = set()
    for b in range(p.summary()["n_blocks"]):
        blk = p.block(b)
        kinds.add(blk["kind"])
        if blk["kind"] == sv.BLOCK_PERM:
            m = blk["mat"]
            nz = np.abs(m) > 0
            assert (nz.sum(axis=0) == 1).all() and (nz.sum(axis=1) == 1).all()
            assert np.allclose(np.abs(m[nz]), 1.0, atol=1e-15)
    assert kinds <= {sv.BLOCK_PERM, sv.BLOCK_DIAG} and sv.BLOCK_PERM in kinds
    assert np.abs(_plan_unitary_state(sv, p, n) - oracle.run(n, g)).max() < 1e-14


def test_kronecker_blocks_are_tensor_products(sv):
    """A layer of one-qubit gates on disjoint qubits packs into Kronecker
    blocks whose matrix is the tensor product of the per-qubit products (bit
    j of the block index is its j-th qubit, so the last qubit's factor comes
    first in numpy's kron)."""
    n = 8
    rows = [(W.U3, q, -1, 0.3 + q, 0.1 * q, -0.7) for q in range(n)]
    rows += [(W.RY, q, -1, 0.2 * q) for q in range(n)]
    g = W.gates(rows)
    p = sv.Plan(n, "c64", g, sv.run_opts(max_fuse_k=4))
    assert p.check() == 0
    found = 0
    for b in range(p.summary()["n_blocks"]):
        blk = p.block(b)
        if blk["kind"] != sv.BLOCK_KRON:
            continue
        found += 1
        ref = np.ones((1, 1), dtype=complex)
        for q in blk["qubits"]:
            f = np.eye(2, dtype=complex)
            for t in blk["gates"]:
                r = g[t]
                if int(r["q0"]) == q:
                    f = oracle.gate_matrix(int(r["op"]), r["theta"], r["phi"], r["lam"]) @ f
            ref = np.kron(f, ref)
        assert np.abs(blk["mat"] - ref).max() < 1e-14
    assert found >= 1
    assert np.abs(_plan_unitary_state(sv, p, n) - oracle.run(n, g)).max() < 1e-14


def _table(**over):
    t = {"pass_ps": 5.0, "dense_ps": [0, 1.0, 2.0, 3.0, 4.0, 5.0], "diag_ps": 0.5, "sign_ps": 0.2,
         "perm_ps": [0, 0.1, 0.1, 0.1, 0.1, 0.1]}
    t.update(over)
    return t


def test_installed_costs_steer_the_planner(sv):
    """A measured table replaces the analytic model for its (dtype, arith)
    pair: with wide blocks priced out the planner fuses at most 2 qubits, with
    passes priced out it takes the widest blocks; removing the table restores
    the analytic choice.  Every plan keeps its invariants."""
    n = 16
    g = W.concat(W.ghz_prefix(n), W.brickwork(n, 6, 4))
    o = sv.run_opts(arith=sv.ARITH_NATIVE)
    base = sv.Plan(n, "c64", g, o).summary()
    try:
        sv.set_costs("c64", sv.ARITH_NATIVE, _table(dense_ps=[0, 1.0, 2.0, 500.0, 900.0, 1900.0]))
        p = sv.Plan(n, "c64", g, o)
        assert p.summary()["fuse_k"] <= 2 and p.check() == 0
        sv.set_costs("c64", sv.ARITH_NATIVE, _table(pass_ps=1e4, dense_ps=[0, 1.0, 1.0, 1.0, 1.0, 1.0]))
        p = sv.Plan(n, "c64", g, o)
        assert p.summary()["fuse_k"] == 5 and p.check() == 0
        # a table for another pair leaves this one alone
        sv.set_costs("c64", sv.ARITH_NATIVE, None)
        sv.set_costs("c128", sv.ARITH_DF64, _table(pass_ps=1e4))
        assert sv.Plan(n, "c64", g, o).summary() == base
    finally:
        sv.set_costs("c64", sv.ARITH_NATIVE, None)
        sv.set_costs("c128", sv.ARITH_DF64, None)
    with pytest.raises(sv.SvError):
        sv.set_costs("c64", sv.ARITH_AUTO, _table())


def test_autotune_cache_round_trip(sv, tmp_path):
    """The JSON cache keeps one table per (GPU, kernel build, dtype, arith);
    install() picks the entries of this GPU and build only."""
    from paper_2502_11385_gb300 import tune
    path = str(tmp_path / "autotune.json")
    kern = tune.kernel_key()
    t = _table()
    t["arith"] = sv.ARITH_NATIVE
    table = {tune.entry_key("GPU-A", kern, "c64", sv.ARITH_NATIVE): t,
             tune.entry_key("GPU-B", kern, "c128", sv.ARITH_TC): dict(t, arith=sv.ARITH_TC)}
    tune.save(table, path)
    back = tune.load(path)
    assert back == table
    try:
        assert tune.install(back, "GPU-A", kern) == 1
        assert tune.install(back, "GPU-A", "other-build") == 0
    finally:
        tune.clear()
