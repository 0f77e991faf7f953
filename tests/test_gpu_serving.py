"""Serving form on the GPU: requests admitted by bytes, small ones batched
continuously while large ones run on their own streams; every result must be
bitwise the same as the request run alone, and match the oracle."""
import numpy as np
import pytest

import oracle
from paper_2502_11385_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = {"c128": 1e-12, "c64": 1e-5}


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2502_11385_gb300 import serve, sv
    return serve, sv


def test_served_results_equal_solo_and_oracle(mods):
    serve, sv = mods
    reqs = W.serving_stream(40, rate=400.0, seed=21, wmin=6, wmax=15, dmin=3, dmax=10)
    opts = sv.run_opts()
    srv = serve.Server(large_qubits=13, large_workers=2, opts=opts)
    res, st = srv.run(reqs)
    assert st["ok"] == len(reqs)
    paths = {r.path for r in res}
    assert paths == {"batch", "large"}
    assert st["batches"] >= 1
    for q, r in zip(reqs, res):
        with sv.State(q.n, q.dtype) as s:
            s.apply_circuit(q.gates, opts)
            solo = s.probabilities()
        assert np.array_equal(r.probs, solo), (q.rid, r.path)
        ref = oracle.probabilities(oracle.run(q.n, q.gates))
        assert np.abs(r.probs - ref).max() <= 4 * TOL[q.dtype]
        assert r.finish >= r.arrival


def test_admission_respects_budget(mods):
    serve, sv = mods
    reqs = W.serving_stream(24, rate=1e4, seed=22, wmin=12, wmax=16, dmin=2, dmax=4)
    budget = max(serve.need_bytes(q.n, q.dtype) for q in reqs) * 2
    srv = serve.Server(budget_bytes=budget, large_qubits=14, opts=sv.run_opts(), keep_outputs=False)
    res, st = srv.run(reqs)
    assert st["ok"] == len(reqs)
    assert srv.peak_resident <= budget


def test_serial_baseline_runs(mods):
    serve, sv = mods
    reqs = W.serving_stream(10, rate=1e3, seed=23, wmin=6, wmax=12, dmin=2, dmax=6)
    res, st = serve.run_serial(reqs, sv.run_opts())
    assert st["requests"] == 10 and all(r.path == "serial" for r in res)
