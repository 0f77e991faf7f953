"""The no-allocation marginal entry point (sv_marginal_probabilities_noalloc),
for callers that cannot have device memory allocated for them.  Its output
must match the regular entry point's, call after call: every call reuses the
same static scratch, so the second call checks that nothing is left over from
the first.  Collected last on purpose (file name), and self-contained so it
also passes alone in a fresh process."""
import numpy as np
import pytest

from paper_2502_11385_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def sv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import sv as _sv
    return _sv


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_marginal_matches_regular_entry_point(sv, dtype):
    import torch
    n = 14
    g = W.concat(W.ghz_prefix(n), W.brickwork(n, 6, 31))
    with sv.State(n, dtype) as s:
        s.apply_circuit(g)
        ptr = s.device_ptr
        for mask in (0b10110000001101, (1 << n) - 1 - (1 << 3) - (1 << 9), 0b1, 0b11):
            ref = s.marginal_probabilities(mask)
            tol = 4 * TOL[dtype] * (1 << (n // 2))
            for _call in range(2):                      # two calls in a row
                host = sv.marginal_probabilities_noalloc(ptr, n, dtype, mask)
                assert np.abs(host - ref).max() <= tol
                dev = torch.empty(len(ref), dtype=torch.float64, device="cuda")
                sv.marginal_probabilities_noalloc(ptr, n, dtype, mask, out=dev)
                assert np.abs(dev.cpu().numpy() - ref).max() <= tol


def test_noalloc_marginal_rejects_masks_beyond_static_scratch(sv):
    n = 18
    with sv.State(n, "c64") as s:
        s.apply_circuit(W.ghz_prefix(n))
        with pytest.raises(sv.SvError) as e:
            sv.marginal_probabilities_noalloc(s.device_ptr, n, "c64", (1 << 17) - 1)
        assert e.value.code == sv.SV_ERR_SIZE
        with pytest.raises(sv.SvError) as e:
            sv.marginal_probabilities_noalloc(s.device_ptr, n, "c64", 1 << 18)
        assert e.value.code == sv.SV_ERR_QUBIT
        out = sv.marginal_probabilities_noalloc(s.device_ptr, n, "c64", (1 << 16) - 1)  # the maximum
        assert abs(out[0] - 0.5) < 1e-6 and abs(out[-1] - 0.5) < 1e-6


def test_noalloc_marginal_leaves_free_device_memory_unchanged(sv):
    """The entry point's defining property: after the first calls (which look
    the static scratch up and load the kernels), repeated calls change the
    device's free memory by nothing, for host and device outputs alike."""
    import torch
    n = 16
    with sv.State(n, "c128") as s:
        s.apply_circuit(W.concat(W.ghz_prefix(n), W.brickwork(n, 4, 9)))
        ptr = s.device_ptr
        mask = 0b1011000000110111
        dev = torch.empty(1 << bin(mask).count("1"), dtype=torch.float64, device="cuda")
        first = sv.marginal_probabilities_noalloc(ptr, n, "c128", mask)
        sv.marginal_probabilities_noalloc(ptr, n, "c128", mask, out=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(5):
            host = sv.marginal_probabilities_noalloc(ptr, n, "c128", mask)
            sv.marginal_probabilities_noalloc(ptr, n, "c128", mask, out=dev)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert np.array_equal(host, first)
