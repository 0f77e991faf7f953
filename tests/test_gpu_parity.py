"""GPU parity: the sm_103a path (through the C-ABI) against the CPU oracle,
element by element on the same seeded inputs.

Tolerances: max |delta amplitude| <= 1e-12 for complex128 and <= 1e-5 for
complex64; |sum p - 1| <= 1e-10 (complex128) and <= 1e-4 (complex64)."""
import math

import numpy as np
import pytest

import oracle
from paper_2502_11385_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c64": 1e-5}
NORM_TOL = {"c128": 1e-10, "c64": 1e-4}


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv as _sv
    return _sv


def _random_circuit(n, count, seed, ops=range(14)):
    rng = np.random.default_rng(seed)
    ops = list(ops)
    rows = []
    for _ in range(count):
        op = int(rng.choice(ops))
        q0 = int(rng.integers(0, n))
        q1 = -1
        if op >= W.CX:
            if n < 2:
                continue
            q1 = int(rng.choice([q for q in range(n) if q != q0]))
        rows.append((op, q0, q1, *rng.uniform(-7, 7, 3)))
    return W.gates(rows)


def _run(sv, n, dtype, g, **opts):
    with sv.State(n, dtype) as s:
        s.apply_circuit(g, sv.run_opts(**opts) if opts else None)
        return s.amplitudes().astype(np.complex128), s.probabilities(), s.norm(), s.stats()


def _check(sv, n, dtype, g, ref=None, **opts):
    if ref is None:
        ref = oracle.run(n, g)
    amp, p, nrm, st = _run(sv, n, dtype, g, **opts)
    err = np.abs(amp - ref).max()
    assert err <= TOL[dtype], (n, dtype, opts, err)
    pref = oracle.probabilities(ref)
    assert np.abs(p - pref).max() <= 4 * TOL[dtype]
    assert abs(nrm - 1.0) <= NORM_TOL[dtype]
    return st


def test_brickwork12_unfused_c128(sv):
    """12 qubits, brickwork depth 10, seed 1, complex128, no fusion."""
    g = W.workload_brickwork12()
    ref = oracle.run(12, g)
    st = _check(sv, 12, "c128", g, ref, max_fuse_k=1)
    assert st["n_blocks"] == 175 and st["n_passes"] == 1
    _check(sv, 12, "c64", g, ref, max_fuse_k=1)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12])
def test_every_gate_on_every_operand(sv, n, dtype):
    """Each gate type on every target (and every ordered control/target pair)
    after a random preparation, unfused and fused."""
    prep = _random_circuit(n, 3 * n, 7 + n, ops=[W.U3, W.CX] if n > 1 else [W.U3])
    for op in range(14):
        rows = []
        for q0 in range(n):
            if op >= W.CX:
                rows += [(op, q0, q1, 0.37 + q0 - 0.11 * q1) for q1 in range(n) if q1 != q0]
            else:
                rows.append((op, q0, -1, 0.3 + 0.7 * q0, -1.1 + q0, 2.3 - q0))
        if not rows:
            continue
        g = W.concat(prep, W.gates(rows))
        ref = oracle.run(n, g)
        _check(sv, n, dtype, g, ref, max_fuse_k=1)
        _check(sv, n, dtype, g, ref, max_fuse_k=4)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,tile", [(10, 0), (16, 9), (18, 10), (20, 0)])
def test_random_circuits_multi_pass(sv, n, tile, k, dtype):
    g = _random_circuit(n, 120, 1000 * n + k)
    st = _check(sv, n, dtype, g, max_fuse_k=k, tile_qubits=tile)
    if tile and n > tile + 2:
        assert st["n_passes"] > 1


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_high_qubits_and_ragged_tiles(sv, dtype):
    # n just above the tile size, gates concentrated on the top qubits
    n = 15
    rows = []
    for rep in range(4):
        for q in range(n - 1, n - 6, -1):
            rows.append((W.U3, q, -1, 0.2 * q + rep, 0.1 * rep, -0.3 * q))
        rows += [(W.CX, n - 1, 0), (W.RZZ, 0, n - 1, 0.7), (W.SWAP, 1, n - 2), (W.CZ, n - 3, 2)]
    g = W.gates(rows)
    for tile in (0, 10, 11):
        _check(sv, n, dtype, g, max_fuse_k=5, tile_qubits=tile)


def test_ghz_closed_form_large(sv):
    for n, dtype in ((26, "c128"), (27, "c64")):
        with sv.State(n, dtype) as s:
            s.apply_circuit(W.ghz_prefix(n))
            p = s.probabilities()
            assert abs(p[0] - 0.5) < NORM_TOL[dtype] and abs(p[-1] - 0.5) < NORM_TOL[dtype]
            assert np.abs(p[1:-1]).max() < 1e-12
            a = s.amplitudes()
            assert abs(a[0] - 1 / math.sqrt(2)) <= TOL[dtype]


def test_qft_of_basis_state(sv):
    n, j = 16, 40503
    g = W.qft_basis(n, j)
    k = np.arange(1 << n)
    ref = np.exp(2j * np.pi * j * k / (1 << n)) / math.sqrt(1 << n)
    for dtype in ("c128", "c64"):
        amp, _, _, _ = _run(sv, n, dtype, g)
        assert np.abs(amp - ref).max() <= TOL[dtype]


def test_marginals_and_norm_exactness(sv):
    """Marginals are sums of |a_i|^2 accumulated exactly (128-bit fixed point),
    so their error comes from the amplitudes alone: over a bin of B amplitudes,
    |sum (|a_i + d_i|^2 - |a_i|^2)| <= e (2 sqrt(B) + B e) with e = max |d_i|
    (Cauchy-Schwarz, sum |a_i|^2 <= 1), plus the oracle's plain float64 sum
    over the bin (at most B 2^-53) and the final roundings.  The bound uses the
    measured amplitude error e."""
    n = 14
    g = W.concat(W.ghz_prefix(n), W.brickwork(n, 5, 3))
    ref = oracle.run(n, g)
    for dtype in ("c128", "c64"):
        with sv.State(n, dtype) as s:
            s.apply_circuit(g)
            e = float(np.abs(s.amplitudes().astype(np.complex128) - ref).max())
            assert e <= TOL[dtype]
            for mask in (0b1, 0b10000000000001, 0b11111000000000, (1 << n) - 1, 0b1010101):
                m = s.marginal_probabilities(mask)
                B = 1 << (n - bin(mask).count("1"))
                bound = e * (2 * math.sqrt(B) + B * e) + B * 2.0**-53 + 4e-16
                assert np.abs(m - oracle.marginal(ref, mask)).max() <= bound, (dtype, mask)
            a, b = s.norm(), s.norm()
            assert a == b                       # order-independent accumulation
            amp = s.amplitudes().astype(np.complex128)
            assert abs(a - math.fsum(np.abs(amp) ** 2)) < 1e-15


def test_reset_basis_and_set_amplitudes(sv):
    n = 9
    with sv.State(n, "c128") as s:
        s.reset(300)
        a = s.amplitudes()
        assert a[300] == 1 and np.count_nonzero(a) == 1
        g = W.brickwork(n, 4, 5)
        s.apply_circuit(g)
        assert np.abs(s.amplitudes() - oracle.run(n, g, basis=300)).max() <= 1e-12
        rng = np.random.default_rng(0)
        v = rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n)
        v /= np.linalg.norm(v)
        s.set_amplitudes(v)
        s.apply_circuit(g)
        assert np.abs(s.amplitudes() - oracle.apply(n, v.copy(), g)).max() <= 1e-12


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_probabilities_pinned_pageable_and_device_outputs_agree(sv, dtype):
    """The three output routes (kernel stores into mapped page-locked host
    memory, staged copy into pageable memory, device buffer) give the same
    bits; n = 25 spans two 128 MiB staging chunks."""
    import torch
    n = 25
    g = W.concat(W.ghz_prefix(n), W.brickwork(n, 2, seed=4))
    with sv.State(n, dtype) as s:
        s.apply_circuit(g)
        dev = torch.full((1 << n,), -1.0, dtype=torch.float64, device="cuda")
        s.probabilities(dev)
        pinned = torch.full((1 << n,), -1.0, dtype=torch.float64, pin_memory=True)
        s.probabilities(pinned.numpy())
        pageable = s.probabilities()
        d = dev.cpu().numpy()
        assert np.array_equal(pinned.numpy(), d)
        assert np.array_equal(pageable, d)
        assert abs(math.fsum(d) - 1.0) <= NORM_TOL[dtype]
        assert d.min() >= 0.0


def test_errors_leave_state_untouched(sv):
    n = 6
    with sv.State(n, "c64") as s:
        s.apply_circuit(W.gates([(W.H, 0, -1)]))
        before = s.amplitudes().copy()
        for bad, code in [((W.CX, 2, 2), sv.SV_ERR_QUBIT), ((W.H, 6, -1), sv.SV_ERR_QUBIT),
                          ((77, 0, -1), sv.SV_ERR_ARG)]:
            with pytest.raises(sv.SvError) as e:
                s.apply_circuit(W.gates([(W.X, 1, -1), bad]))
            assert e.value.code == code
        assert np.array_equal(s.amplitudes(), before)
        s.apply_circuit(W.gates([]))
        assert np.array_equal(s.amplitudes(), before)
        with pytest.raises(sv.SvError) as e:
            s.probabilities(np.empty(10))
        assert e.value.code == sv.SV_ERR_SIZE
    with pytest.raises(sv.SvError):
        sv.State(0, "c64")
    with pytest.raises(sv.SvError):
        sv.State(35, "c128")


def test_wrap_torch_tensor(sv):
    import torch
    n = 11
    t = torch.zeros(1 << n, dtype=torch.complex128, device="cuda")
    t[0] = 1
    torch.cuda.synchronize()
    s = sv.State.from_tensor(t, n, "c128", stream=torch.cuda.current_stream().cuda_stream)
    g = W.brickwork(n, 5, 8)
    s.apply_circuit(g)
    torch.cuda.synchronize()
    ref = oracle.run(n, g)
    assert np.abs(t.cpu().numpy() - ref).max() <= 1e-12
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    s.probabilities(p)
    assert np.abs(p.cpu().numpy() - oracle.probabilities(ref)).max() <= 1e-12
    s.close()


def test_config2_30q_uudagger_is_ghz(sv):
    """30 qubits, complex64 (the complex128 run is in test_gpu_fullsize and
    test_gpu_oracle_large): GHZ prefix + depth-20 brickwork (seed 2), then the
    inverse brickwork; the result must be the GHZ closed form."""
    n = 30
    body = W.brickwork(n, 20, 2)
    g = W.concat(W.ghz_prefix(n), body, W.inverse(body))
    import torch
    with sv.State(n, "c64") as s:
        s.apply_circuit(g)
        p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
        s.probabilities(p)
        assert abs(p[0].item() - 0.5) < 1e-4 and abs(p[-1].item() - 0.5) < 1e-4
        p[0] = 0
        p[-1] = 0
        assert p.max().item() < 1e-9
        assert abs(s.norm() - 1) < 1e-4


# ---------------------------------------------------------------------------
# complex128 with double-float arithmetic on the FP32 units (SV_ARITH_DF64)
# ---------------------------------------------------------------------------
def test_df64_brickwork12(sv):
    g = W.workload_brickwork12()
    ref = oracle.run(12, g)
    _check(sv, 12, "c128", g, ref, max_fuse_k=1, arith=sv.ARITH_DF64)
    st = _check(sv, 12, "c128", g, ref, arith=sv.ARITH_DF64)
    assert st["arith"] == sv.ARITH_DF64


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,tile", [(10, 0), (16, 9), (20, 0)])
def test_df64_random_circuits(sv, n, tile, k):
    g = _random_circuit(n, 120, 7000 * n + k)
    _check(sv, n, "c128", g, max_fuse_k=k, tile_qubits=tile, arith=sv.ARITH_DF64)


@pytest.mark.parametrize("n", [3, 8, 12])
def test_df64_every_gate_on_every_operand(sv, n):
    prep = _random_circuit(n, 3 * n, 17 + n, ops=[W.U3, W.CX])
    rows = []
    for op in range(14):
        for q0 in range(n):
            if op >= W.CX:
                rows += [(op, q0, q1, 0.37 + q0 - 0.11 * q1) for q1 in range(n) if q1 != q0]
            else:
                rows.append((op, q0, -1, 0.3 + 0.7 * q0, -1.1 + q0, 2.3 - q0))
    g = W.concat(prep, W.gates(rows))
    ref = oracle.run(n, g)
    for k in (1, 3, 5):
        _check(sv, n, "c128", g, ref, max_fuse_k=k, arith=sv.ARITH_DF64)


def test_df64_conversion_roundtrip(sv):
    """float64 -> (hi, lo) float pair -> float64 keeps 47 significant bits
    (components >= 2^-100 in magnitude) across powers of two, signs and
    magnitudes from 1 down to 1e-30; components below 2^-126 flush to zero."""
    n = 12
    rng = np.random.default_rng(5)
    mag = 10.0 ** rng.uniform(-30, 0, size=(1 << n, 2))
    sgn = rng.choice([-1.0, 1.0], size=(1 << n, 2))
    v = mag * sgn
    v[:64, 0] = 2.0 ** -np.arange(64)                       # powers of two
    v[64:128, 1] = -(2.0 ** -np.arange(64)) * (1 + 2.0 ** -30)
    v[128:136] = 1e-40                                      # below float's range
    a = v[:, 0] + 1j * v[:, 1]
    with sv.State(n, "c128") as s:
        s.set_amplitudes(a)
        s.apply_circuit(W.gates([(W.X, 0, -1), (W.X, 0, -1)]), sv.run_opts(max_fuse_k=1, arith=sv.ARITH_DF64))
        out = s.amplitudes()
    for got, want in ((out.real, v[:, 0]), (out.imag, v[:, 1])):
        big = np.abs(want) >= 2.0 ** -100
        rel = np.abs(got[big] - want[big]) / np.abs(want[big])
        assert rel.max() <= 2.0 ** -46, rel.max()
        assert np.all(got[np.abs(want) < 2.0 ** -126] == 0)


# ---------------------------------------------------------------------------
# batched form
# ---------------------------------------------------------------------------
def test_batch_matches_solo_bitwise_and_oracle(sv):
    rng = np.random.default_rng(9)
    items, solo = [], []
    specs = [(9, "c64"), (12, "c128"), (14, "c64"), (10, "c128"), (16, "c128"), (5, "c64"), (13, "c128")]
    for i, (n, dt) in enumerate(specs):
        g = _random_circuit(n, 60 + 5 * i, 400 + i)
        items.append((n, dt, g, None))
    for arith in (sv.ARITH_NATIVE, sv.ARITH_DF64, sv.ARITH_TC, sv.ARITH_TC_SYNC):
        opts = sv.run_opts(arith=arith)
        with sv.Batch(items, opts) as b:
            assert b.status == [0] * len(items)
            outs = b.execute()
            outs2 = [o.copy() for o in b.execute()]  # replay of the captured graph
            st = b.stats()
            assert st["n_items"] == len(items) and st["n_launches"] >= 3
        for (n, dt, g, _), o, o2 in zip(items, outs, outs2):
            with sv.State(n, dt) as s:
                s.apply_circuit(g, opts)
                p = s.probabilities()
            assert np.array_equal(o, p)            # same plan, same kernels: bitwise
            assert np.array_equal(o, o2)
            pref = oracle.probabilities(oracle.run(n, g))
            assert np.abs(o - pref).max() <= 4 * TOL[dt]


def test_batch_device_outputs_and_invalid_items(sv):
    import torch
    g_ok = W.brickwork(11, 4, 3)
    dev = torch.empty(1 << 11, dtype=torch.float64, device="cuda")
    items = [(11, "c128", g_ok, dev), (11, "c64", W.gates([(W.H, 11, -1)]), None), (8, "c64", W.ghz_prefix(8), None)]
    outs, status = sv.batch_run(items)
    assert status[0] == 0 and status[1] == sv.SV_ERR_QUBIT and status[2] == 0
    ref = oracle.probabilities(oracle.run(11, g_ok))
    assert np.abs(dev.cpu().numpy() - ref).max() <= 4e-12
    assert abs(outs[2][0] - 0.5) < 1e-6 and abs(outs[2][-1] - 0.5) < 1e-6


def test_cut_variants_batched(sv):
    """Cut-subcircuit variants of a small cuttable brickwork (12 qubits, 2 cut
    wires): all 9 upstream and 16 downstream variants in one batch."""
    cc = W.cuttable_brickwork(12, 6, 11, cut_lo=5, n_cuts=2, switch_layer=3)
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    items = [(cc.width_a, "c128", g, None) for g in ups] + [(cc.width_b, "c64", g, None) for g in downs]
    outs, status = sv.batch_run(items, sv.run_opts(arith=sv.ARITH_DF64))
    assert all(s == 0 for s in status)
    for (n, dt, g, _), o in zip(items, outs):
        assert np.abs(o - oracle.probabilities(oracle.run(n, g))).max() <= 4 * TOL[dt]


# ---------------------------------------------------------------------------
# cut reconstruction (Sec. III-A, Eqs. 3.2-3.7)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,depth,cut_lo,k,switch", [(6, 4, 2, 1, 2), (10, 6, 4, 3, 3), (12, 6, 5, 2, 3)])
def test_cut_reconstruction_on_gpu(sv, n, depth, cut_lo, k, switch):
    import torch
    from oracle import cut
    cc = W.cuttable_brickwork(n, depth, 300 + n, cut_lo=cut_lo, n_cuts=k, switch_layer=switch)
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    up_t = [torch.empty(1 << cc.width_a, dtype=torch.float64, device="cuda") for _ in ups]
    dn_t = [torch.empty(1 << cc.width_b, dtype=torch.float64, device="cuda") for _ in downs]
    items = [(cc.width_a, "c128", g, t) for g, t in zip(ups, up_t)] + \
            [(cc.width_b, "c128", g, t) for g, t in zip(downs, dn_t)]
    _, status = sv.batch_run(items)
    assert all(s == 0 for s in status)
    rec = sv.cut_reconstruct(up_t, dn_t, cc.width_a, list(cc.cut_qubits), cc.width_b)
    full = oracle.probabilities(oracle.run(n, cc.full))
    assert np.abs(rec - full).max() <= 1e-12
    p_up = [t.cpu().numpy() for t in up_t]
    p_dn = [t.cpu().numpy() for t in dn_t]
    assert np.abs(rec - cut.reconstruct(p_up, p_dn, cc.width_a, list(cc.cut_qubits))).max() <= 1e-13
    # partial reconstruction over chosen qubits: upstream qubit 0 and the last downstream qubit
    ka, kb = 0b1, 1 << (cc.width_b - 1)
    part = sv.cut_reconstruct(up_t, dn_t, cc.width_a, list(cc.cut_qubits), cc.width_b, ka, kb)
    gmask = 1 | (1 << (n - 1))   # the same two qubits in the uncut circuit
    assert np.abs(part - oracle.marginal(oracle.run(n, cc.full), gmask)).max() <= 1e-12


@pytest.mark.parametrize("n,depth,cut_lo,k,switch", [(14, 6, 5, 4, 3), (16, 8, 6, 4, 4)])
def test_cut_reconstruction_four_cuts_and_partial_masks(sv, n, depth, cut_lo, k, switch):
    """K = 4 (256 term codes, several chunks of the contraction), the full
    distribution and marginals over several kept qubits on both sides against
    the uncut oracle."""
    import torch
    cc = W.cuttable_brickwork(n, depth, 300 + n, cut_lo=cut_lo, n_cuts=k, switch_layer=switch)
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    up_t = [torch.empty(1 << cc.width_a, dtype=torch.float64, device="cuda") for _ in ups]
    dn_t = [torch.empty(1 << cc.width_b, dtype=torch.float64, device="cuda") for _ in downs]
    items = [(cc.width_a, "c128", g, t) for g, t in zip(ups, up_t)] + \
            [(cc.width_b, "c128", g, t) for g, t in zip(downs, dn_t)]
    _, status = sv.batch_run(items)
    assert all(s == 0 for s in status)
    psi = oracle.run(n, cc.full)
    rec = sv.cut_reconstruct(up_t, dn_t, cc.width_a, list(cc.cut_qubits), cc.width_b)
    assert np.abs(rec - oracle.probabilities(psi)).max() <= 1e-12
    eff_a = [q for q in range(cc.width_a) if q not in cc.cut_qubits]  # upstream qubit eff_a[i] = global i
    for ka, kb in ((0b1011, 0b1), (0b1, 0b110010), ((1 << len(eff_a)) - 1, 0b1)):
        mask_a = sum(1 << eff_a[i] for i in range(len(eff_a)) if (ka >> i) & 1)
        part = sv.cut_reconstruct(up_t, dn_t, cc.width_a, list(cc.cut_qubits), cc.width_b, mask_a, kb)
        gmask = ka | (kb << len(eff_a))
        assert np.abs(part - oracle.marginal(psi, gmask)).max() <= 1e-12, (ka, kb)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_cut_variants_shared_work_matches_plain(sv, dtype):
    """Variant shortcuts (shared upstream body, downstream by linearity) give
    the same distributions as simulating every variant on its own."""
    cc = W.cuttable_brickwork(13, 6, 41, cut_lo=5, n_cuts=3, switch_layer=3)
    up, down = sv.cut_variants(cc, dtype)
    ups, downs = cc.upstream_variants(), cc.downstream_variants()
    for g, p in zip(ups, up):
        assert np.abs(p - oracle.probabilities(oracle.run(cc.width_a, g))).max() <= 4 * TOL[dtype]
    for g, p in zip(downs, down):
        assert np.abs(p - oracle.probabilities(oracle.run(cc.width_b, g))).max() <= 4 * TOL[dtype]
    # and reconstruction from the shared-work variants gives the uncut circuit
    if dtype == "c128":
        from oracle import cut
        rec = cut.reconstruct(up, down, cc.width_a, list(cc.cut_qubits))
        assert np.abs(rec - oracle.probabilities(oracle.run(13, cc.full))).max() <= 1e-12


# ---------------------------------------------------------------------------
# complex128 on the tensor cores: SV_ARITH_TC (tcgen05, accumulators in
# tensor memory, balanced digits) and SV_ARITH_TC_SYNC (warp-level mma.sync)
# ---------------------------------------------------------------------------
TC_MODES = ("tc", "tc_sync")


def _tc_arith(sv, mode):
    return sv.ARITH_TC if mode == "tc" else sv.ARITH_TC_SYNC


@pytest.mark.parametrize("mode", TC_MODES)
def test_tc_brickwork12(sv, mode):
    """Unfused, the 175 blocks share one pass, past the kernel's 48-op cache
    (the op computes its own address table); fused, the pass's tables are
    built once per CTA."""
    g = W.workload_brickwork12()
    ref = oracle.run(12, g)
    opts = sv.run_opts(max_fuse_k=1, arith=_tc_arith(sv, mode))
    assert max(len(sv.Plan(12, "c128", g, opts).pass_info(i)["blocks"])
               for i in range(sv.Plan(12, "c128", g, opts).summary()["n_passes"])) > 48
    for k in (1, 3, 4, 5):
        st = _check(sv, 12, "c128", g, ref, max_fuse_k=k, arith=_tc_arith(sv, mode))
        assert st["arith"] == _tc_arith(sv, mode)


@pytest.mark.parametrize("mode", TC_MODES)
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,tile", [(9, 0), (16, 9), (20, 0)])
def test_tc_random_circuits(sv, n, tile, k, mode):
    g = _random_circuit(n, 120, 9000 * n + k)
    _check(sv, n, "c128", g, max_fuse_k=k, tile_qubits=tile, arith=_tc_arith(sv, mode))


@pytest.mark.parametrize("tile", [9, 10, 11, 12, 13])
def test_tc_tile_sizes(sv, tile):
    """tcgen05 mode across tile sizes: partial M-tiles (9, 10), two CTAs per SM
    (11), one (12, 13)."""
    n = 17
    g = _random_circuit(n, 150, 31 + tile)
    ref = oracle.run(n, g)
    for k in (3, 4):
        st = _check(sv, n, "c128", g, ref, max_fuse_k=k, tile_qubits=tile, arith=sv.ARITH_TC)
        assert st["tile_qubits"] == tile and st["arith"] == sv.ARITH_TC


@pytest.mark.parametrize("mode", TC_MODES)
@pytest.mark.parametrize("n", [8, 12])
def test_tc_every_gate_on_every_operand(sv, n, mode):
    prep = _random_circuit(n, 3 * n, 27 + n, ops=[W.U3, W.CX])
    rows = []
    for op in range(14):
        for q0 in range(n):
            if op >= W.CX:
                rows += [(op, q0, q1, 0.37 + q0 - 0.11 * q1) for q1 in range(n) if q1 != q0]
            else:
                rows.append((op, q0, -1, 0.3 + 0.7 * q0, -1.1 + q0, 2.3 - q0))
    g = W.concat(prep, W.gates(rows))
    ref = oracle.run(n, g)
    for k in (1, 3, 4, 5):
        _check(sv, n, "c128", g, ref, max_fuse_k=k, arith=_tc_arith(sv, mode))


def test_tc_basis_states_and_extreme_amplitudes(sv):
    """Components of magnitude exactly 1 (basis states, permutations, signs)
    sit at the edge of the fixed-point range: X/CX/SWAP/Z networks keep every
    amplitude at 0 or +-1, and the result must be exact."""
    n = 13
    rng = np.random.default_rng(12)
    rows = []
    for _ in range(200):
        op = int(rng.choice([W.X, W.Y, W.Z, W.CX, W.CZ, W.SWAP]))
        q0 = int(rng.integers(n))
        q1 = int(rng.choice([q for q in range(n) if q != q0])) if op >= W.CX else -1
        rows.append((op, q0, q1))
    g = W.gates(rows)
    ref = oracle.run(n, g)
    for k in (1, 3, 4):
        amp, _, _, st = _run(sv, n, "c128", g, max_fuse_k=k, arith=sv.ARITH_TC)
        assert st["arith"] == sv.ARITH_TC
        assert np.array_equal(amp, ref), np.abs(amp - ref).max()


def test_tc_small_states_fall_back(sv):
    g = _random_circuit(5, 40, 5)
    st = _check(sv, 5, "c128", g, arith=sv.ARITH_TC)
    assert st["arith"] == sv.ARITH_DF64


def test_auto_arith_falls_back_for_unnormalised_amplitudes(sv):
    """A caller-supplied state with components above 1 in magnitude is outside
    the tensor-core mode's fixed-point range: the call uses double-float."""
    n = 20
    rng = np.random.default_rng(4)
    v = 3.0 * (rng.normal(size=1 << n) + 1j * rng.normal(size=1 << n))
    g = _random_circuit(n, 30, 77)
    with sv.State(n, "c128") as s:
        s.set_amplitudes(v)
        s.apply_circuit(g)
        assert s.stats()["arith"] == sv.ARITH_DF64
        ref = oracle.apply(n, v.astype(np.complex128).copy(), g)
        assert np.abs(s.amplitudes() - ref).max() <= 1e-11
        s.set_amplitudes(v / np.linalg.norm(v))
        s.apply_circuit(g)
        assert s.stats()["arith"] == sv.ARITH_TC
        assert np.abs(s.amplitudes() - oracle.apply(n, (v / np.linalg.norm(v)).copy(), g)).max() <= 1e-12


def test_tc_gate_uses_the_norm_not_the_component_bound(sv):
    """Components at most 1 do not keep later states in range: with every
    amplitude (1 + i)/sqrt 2 (norm 2^n) a Hadamard layer makes components of
    sqrt 2 at the first gate.  The tensor-core mode is gated on the exact norm
    (at most 1, kept by unitary blocks), so this state runs in double-float and
    matches the oracle; a state normalised in float64 keeps the tensor cores."""
    n = 20
    v = np.full(1 << n, (1 + 1j) / math.sqrt(2), dtype=np.complex128)
    g = W.gates([(W.H, q, -1) for q in range(n)] + [(W.U3, q, -1, 0.3 * q, 0.2, -0.4) for q in range(n)])
    with sv.State(n, "c128") as s:
        s.set_amplitudes(v)
        s.apply_circuit(g, sv.run_opts(arith=sv.ARITH_TC))
        assert s.stats()["arith"] == sv.ARITH_DF64
        ref = oracle.apply(n, v.copy(), g)
        # |a| grows to 2^(n/2) here; the tolerance is relative to it
        assert np.abs(s.amplitudes() - ref).max() <= 1e-12 * np.abs(ref).max()
        w = v / np.linalg.norm(v)
        s.set_amplitudes(w)
        s.apply_circuit(g, sv.run_opts(arith=sv.ARITH_TC))
        assert s.stats()["arith"] == sv.ARITH_TC
        assert np.abs(s.amplitudes() - oracle.apply(n, w.copy(), g)).max() <= 1e-12


def test_auto_arith_threshold(sv):
    """SV_ARITH_AUTO: complex128 below 20 qubits in double-float, tcgen05
    digits from 20 on; complex64 below 23 qubits in float32 FMAs, tcgen05
    triple split from 23 on."""
    for n, want in ((19, sv.ARITH_DF64), (20, sv.ARITH_TC)):
        g = _random_circuit(n, 40, 700 + n)
        st = _check(sv, n, "c128", g)
        assert st["arith"] == want, (n, st["arith"])
    for n, want in ((22, sv.ARITH_NATIVE), (23, sv.ARITH_TC)):  # complex64: float32 FMAs / triple split
        g = _random_circuit(n, 40, 800 + n)
        st = _check(sv, n, "c64", g)
        assert st["arith"] == want, (n, st["arith"])


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_tc_bounded_wait_reports_timeout_and_recovers(sv, dtype):
    """Failure detection without a GPU fault: a test hook makes the first
    tensor-memory block issue no MMAs, so the kernel's bounded wait (one
    second) runs out.  The call reports SV_ERR_TIMEOUT, the handle refuses
    further use until it is reset, and the context stays usable."""
    import time
    n = 14
    g = _random_circuit(n, 60, 1234)
    ref = oracle.run(n, g)
    with sv.State(n, dtype) as s:
        t0 = time.perf_counter()
        with pytest.raises(sv.SvError) as e1:
            s.apply_circuit(g, sv.run_opts(arith=sv.ARITH_TC, debug_checks=2))
        assert e1.value.code == sv.SV_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 30
        with pytest.raises(sv.SvError) as e2:
            s.probabilities()
        assert e2.value.code == sv.SV_ERR_STATE
        s.reset(0)
        s.apply_circuit(g, sv.run_opts(arith=sv.ARITH_TC))
        assert s.stats()["arith"] == sv.ARITH_TC
        assert np.abs(s.amplitudes() - ref).max() <= TOL[dtype]
    # a fresh handle on the same context works as well
    _check(sv, n, dtype, g, ref, arith=sv.ARITH_TC)


# ---------------------------------------------------------------------------
# complex64 on the tensor cores (SV_ARITH_TC: bfloat16 triple split)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("n,tile", [(10, 0), (16, 10), (20, 0)])
def test_tc32_random_circuits(sv, n, tile, k):
    g = _random_circuit(n, 120, 5000 * n + k)
    st = _check(sv, n, "c64", g, max_fuse_k=k, tile_qubits=tile, arith=sv.ARITH_TC)
    assert st["arith"] == sv.ARITH_TC


@pytest.mark.parametrize("tile", [10, 11, 12, 13, 14])
def test_tc32_tile_sizes(sv, tile):
    n = 17
    g = _random_circuit(n, 150, 77 + tile)
    ref = oracle.run(n, g)
    for k in (3, 4, 5):
        st = _check(sv, n, "c64", g, ref, max_fuse_k=k, tile_qubits=tile, arith=sv.ARITH_TC)
        assert st["tile_qubits"] == tile and st["arith"] == sv.ARITH_TC


@pytest.mark.parametrize("n", [8, 12])
def test_tc32_every_gate_on_every_operand(sv, n):
    prep = _random_circuit(n, 3 * n, 37 + n, ops=[W.U3, W.CX])
    rows = []
    for op in range(14):
        for q0 in range(n):
            if op >= W.CX:
                rows += [(op, q0, q1, 0.41 + q0 - 0.13 * q1) for q1 in range(n) if q1 != q0]
            else:
                rows.append((op, q0, -1, 0.2 + 0.6 * q0, -1.3 + q0, 2.1 - q0))
    g = W.concat(prep, W.gates(rows))
    ref = oracle.run(n, g)
    for k in (1, 3, 4, 5):
        _check(sv, n, "c64", g, ref, max_fuse_k=k, arith=sv.ARITH_TC)


def test_tc32_accuracy_matches_float32(sv):
    """The triple split carries float32 accuracy: on a 20-qubit circuit its
    error against the complex128 oracle is of the same order as the FP32
    FMA path's (relative L2 error, and max |delta a| well inside 1e-5)."""
    n = 20
    g = W.workload_ghz_brickwork(n, 12, 9)
    ref = oracle.run(n, g)
    errs = {}
    for arith in (sv.ARITH_NATIVE, sv.ARITH_TC):
        amp, _, _, st = _run(sv, n, "c64", g, arith=arith)
        assert st["arith"] == arith
        errs[arith] = (np.linalg.norm(amp - ref) / np.linalg.norm(ref), np.abs(amp - ref).max())
    assert errs[sv.ARITH_TC][1] <= 1e-6, errs
    assert errs[sv.ARITH_TC][0] <= 8 * max(errs[sv.ARITH_NATIVE][0], 1e-7), errs


# ---------------------------------------------------------------------------
# Block classes: permutation blocks (amplitude moves with quarter phases, or
# a move then a diagonal pass for T / RZ / RZZ phases) and Kronecker blocks
# (one butterfly per qubit outside the tensor-core modes)
# ---------------------------------------------------------------------------
ALL_MODES = [("c128", 0), ("c128", 1), ("c128", 2), ("c128", 3), ("c128", 4), ("c64", 1), ("c64", 3)]


def _perm_network(n, count, seed):
    """CX / SWAP / X / Y / Z / S / T / CZ / RZZ networks with a few H and U3
    gates between them."""
    rng = np.random.default_rng(seed)
    ops = [W.CX, W.CX, W.SWAP, W.X, W.Y, W.Z, W.S, W.T, W.CZ, W.RZZ]
    rows = []
    for i in range(count):
        op = ops[int(rng.integers(0, len(ops)))] if i % 9 else [W.H, W.U3][int(rng.integers(0, 2))]
        q0 = int(rng.integers(0, n))
        q1 = int(rng.choice([q for q in range(n) if q != q0])) if op >= W.CX else -1
        rows.append((op, q0, q1, *rng.uniform(-4, 4, 3)))
    return W.gates(rows)


@pytest.mark.parametrize("dtype,arith", ALL_MODES)
@pytest.mark.parametrize("n,tile", [(10, 0), (16, 10), (20, 0)])
def test_permutation_blocks_every_mode(sv, n, tile, dtype, arith):
    g = _perm_network(n, 160, 300 + n)
    p = sv.Plan(n, dtype, g, sv.run_opts(arith=arith, tile_qubits=tile))
    kinds = {p.block(b)["kind"] for b in range(p.summary()["n_blocks"])}
    assert sv.BLOCK_PERM in kinds
    _check(sv, n, dtype, g, arith=arith, tile_qubits=tile)


@pytest.mark.parametrize("dtype,arith", ALL_MODES)
def test_kronecker_layers_every_mode(sv, dtype, arith):
    """Layers of one-qubit rotations on every qubit between CZ layers."""
    n = 14
    rows = []
    for layer in range(6):
        rows += [(W.U3, q, -1, 0.3 * q + layer, 0.2 * layer, -0.1 * q) for q in range(n)]
        rows += [(W.RX, q, -1, 0.5 + 0.1 * q) for q in range(n)]
        rows += [(W.CZ, q, q + 1) for q in range(layer % 2, n - 1, 2)]
    g = W.gates(rows)
    _check(sv, n, dtype, g, arith=arith)
    _check(sv, n, dtype, g, arith=arith, tile_qubits=10)


def test_sharded_local_applier_is_the_library(sv):
    """The sharded state's default local applier runs a rank's gate segment
    through the CUDA library on its chunk in place (a GPU rank of a sharded
    run; the exchanges between ranks are tested on CPU ranks)."""
    import torch
    from paper_2502_11385_gb300 import shard
    n = 14
    g = _random_circuit(n, 90, 4242)
    for dtype, ct in (("c128", torch.complex128), ("c64", torch.complex64)):
        chunk = torch.zeros(1 << n, dtype=ct, device="cuda")
        chunk[0] = 1
        shard._library_apply(chunk, n, g)
        torch.cuda.synchronize()
        assert np.abs(chunk.cpu().numpy().astype(np.complex128) - oracle.run(n, g)).max() <= TOL[dtype]
