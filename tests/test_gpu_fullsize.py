"""Full-size runs of the configurations that do not fit the oracle, checked by
properties that hold at any size:

- QAOA (precision form, 32 q complex128 and 32 / 33 q complex64): the global
  bit flip X^n commutes with H^n|0>, RZZ and RX, so a(x) = a(x XOR 1...1)
  exactly; after H on all qubits and one cost layer every |a_x|^2 = 2^-n;
  the norm is 1.  The complex64 error is measured against the complex128 run.
- 30 q complex128 brickwork (the benchmark workload): U U^dagger returns the
  GHZ state (closed form).
Each run holds at most about 160 GiB on the device."""
import math

import numpy as np
import pytest

from paper_2502_11385_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv
    free, _ = torch.cuda.mem_get_info()
    return torch, sv, free


def _state(torch, sv, n, dtype):
    ct = torch.complex128 if dtype == "c128" else torch.complex64
    buf = torch.empty(1 << n, dtype=ct, device="cuda")
    st = sv.State.from_tensor(buf, n, dtype)
    st.reset(0)
    return buf, st


@pytest.mark.parametrize("n,dtype", [(32, "c128"), (33, "c64")])
def test_qaoa_symmetry_and_norm(env, n, dtype):
    torch, sv, free = env
    need = (1 << n) * (16 if dtype == "c128" else 8) * 1.6
    if free < need:
        pytest.skip("not enough device memory")
    g, edges, _, _ = W.qaoa(n, 2, 3)
    buf, st = _state(torch, sv, n, dtype)
    st.apply_circuit(g)
    torch.cuda.synchronize()
    asym = (buf - buf.flip(0)).abs().max().item()
    assert asym <= (1e-12 if dtype == "c128" else 1e-6)
    assert abs(st.norm() - 1) <= (1e-10 if dtype == "c128" else 1e-4)
    st.close()
    del buf
    torch.cuda.empty_cache()


def test_qaoa_first_cost_layer_is_flat(env):
    torch, sv, free = env
    n = 32
    g, edges, _, _ = W.qaoa(n, 2, 3)
    pre = g[: n + len(edges)]
    buf, st = _state(torch, sv, n, "c64")
    st.apply_circuit(pre)
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    st.probabilities(p)
    assert (p - 2.0 ** -n).abs().max().item() <= 2.0 ** -n * 1e-5
    st.close()
    del buf, p
    torch.cuda.empty_cache()


def test_qaoa32_c64_against_c128(env):
    """Precision form: complex64 (FP32 arithmetic, FP64 probabilities) against
    the complex128 path at 32 qubits: max |delta a| and the probability L1."""
    torch, sv, free = env
    n = 32
    if free < 170 * 2 ** 30:
        pytest.skip("not enough device memory")
    g = W.qaoa(n, 2, 3)[0]
    b128, s128 = _state(torch, sv, n, "c128")
    s128.apply_circuit(g)
    b64, s64 = _state(torch, sv, n, "c64")
    s64.apply_circuit(g)
    torch.cuda.synchronize()
    err = 0.0
    chunk = 1 << 28
    for i in range(0, 1 << n, chunk):
        err = max(err, (b128[i:i + chunk] - b64[i:i + chunk].to(torch.complex128)).abs().max().item())
    assert err <= 1e-5
    p128 = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    p64 = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    s128.probabilities(p128)
    s64.probabilities(p64)
    l1 = (p128 - p64).abs().sum().item()
    assert l1 <= 1e-3
    print(f"qaoa32 complex64 vs complex128: max|da| = {err:.3e}, L1(p) = {l1:.3e}")
    for s in (s128, s64):
        s.close()
    del b128, b64, p128, p64
    torch.cuda.empty_cache()


def test_bench_workload_uudagger_c128(env):
    torch, sv, free = env
    n = 30
    body = W.brickwork(n, 20, 2)
    g = W.concat(W.ghz_prefix(n), body, W.inverse(body))
    buf, st = _state(torch, sv, n, "c128")
    st.apply_circuit(g)
    torch.cuda.synchronize()
    r = 1 / math.sqrt(2)
    assert abs(buf[0].item() - r) <= 1e-12 and abs(buf[-1].item() - r) <= 1e-12
    buf[0] = 0
    buf[-1] = 0
    assert buf.abs().max().item() <= 1e-12
    st.close()
    del buf
    torch.cuda.empty_cache()


def test_adder_30q_exact_sum(env):
    """Cuccaro adder, 14-bit registers (30 qubits, complex128): the basis input
    |a, b> must end in the single basis state |a, a+b, carry>."""
    torch, sv, free = env
    m = 14
    a, b = 12345, 9876
    n = 2 * m + 2
    buf, st = _state(torch, sv, n, "c128")
    st.apply_circuit(W.cuccaro_adder(m, a, b))
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    st.probabilities(p)
    idx = W.adder_output_index(m, a, b)
    assert abs(p[idx].item() - 1) <= 1e-10
    assert abs(st.norm() - 1) <= 1e-10
    st.close()
    del buf, p
    torch.cuda.empty_cache()


def test_bernstein_vazirani_30q(env):
    torch, sv, free = env
    n = 30
    secret = 0b10110011100011110000111110101
    buf, st = _state(torch, sv, n, "c64")
    st.apply_circuit(W.bernstein_vazirani(n, secret))
    p = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    st.probabilities(p)
    got = p[secret].item() + p[secret | (1 << (n - 1))].item()   # ancilla is |->
    assert abs(got - 1) <= 1e-4
    st.close()
    del buf, p
    torch.cuda.empty_cache()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_qft_30q_sampled_amplitudes(env, dtype):
    """QFT of a basis state at 30 qubits: 65536 sampled amplitudes against the
    closed form e^{2 pi i j k / 2^n} / 2^(n/2)."""
    torch, sv, free = env
    n, j = 30, 0x2345677
    buf, st = _state(torch, sv, n, dtype)
    st.apply_circuit(W.qft_basis(n, j))
    torch.cuda.synchronize()
    rng = np.random.default_rng(3)
    k = np.sort(rng.choice(1 << n, size=65536, replace=False))
    got = buf[torch.from_numpy(k).cuda()].cpu().numpy().astype(np.complex128)
    ref = np.exp(2j * np.pi * ((j * k) % (1 << n)) / (1 << n)) / 2 ** (n / 2)
    assert np.abs(got - ref).max() <= (1e-12 if dtype == "c128" else 1e-5)
    st.close()
    del buf
    torch.cuda.empty_cache()
