"""The sharded statevector (paper Sec. III-B, Fig. 3b) on CPU ranks: gloo
process groups of 2 and 4 ranks move real halves of their chunks through the
pairwise exchange; the oracle, injected as each rank's local applier, runs
the local gate segments.  The gathered state must equal the unsharded
oracle's, and diagonal gates on global qubits must cost no exchange."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2502_11385_gb300 import workloads as W

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _oracle_apply(chunk, n_local, gates):
    oracle.apply(n_local, chunk.numpy(), gates)


def _random_circuit(n, count, seed):
    rng = np.random.default_rng(seed)
    rows = []
    for _ in range(count):
        op = int(rng.integers(0, 14))
        # half the gates on the top qubits, which start at global positions
        q0 = int(rng.integers(n - 3, n)) if rng.random() < 0.5 else int(rng.integers(0, n))
        q1 = int(rng.choice([q for q in range(n) if q != q0])) if op >= W.CX else -1
        rows.append((op, q0, q1, *rng.uniform(-4, 4, 3)))
    return W.gates(rows)


def _worker(rank, world, port, n, seed, c, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2502_11385_gb300.shard import ShardedState
        g = _random_circuit(n, 80, seed)
        nl = n - (world.bit_length() - 1)
        chunk = torch.zeros(1 << nl, dtype=torch.complex128)
        st = ShardedState(n, chunk, local_apply=_oracle_apply, sub_chunk_log2=c)
        st.reset()
        st.apply(g)
        st.finish()
        nrm = st.norm()
        parts = [torch.zeros_like(torch.view_as_real(chunk)) for _ in range(world)] if rank == 0 else None
        dist.gather(torch.view_as_real(chunk), parts, dst=0)  # complex data as real pairs
        if rank == 0:
            out["state"] = torch.view_as_complex(torch.cat(parts)).numpy().copy()
            out["exchanges"] = st.exchanges
        out[f"norm{rank}"] = nrm
        # diagonal gates only, many on global qubits: no exchange at all
        st.reset()
        before = st.exchanges
        diag = W.gates([(W.CZ, n - 1, 0), (W.RZZ, n - 1, n - 2, 0.7), (W.T, n - 1, -1), (W.RZ, n - 2, -1, 0.3),
                        (W.S, 1, -1), (W.Z, n - 2, -1), (W.CZ, n - 1, n - 2)])
        st.apply(W.concat(W.gates([(W.H, q, -1) for q in range(n - 2)]), diag))
        st.finish()
        out[f"diag_exchanges{rank}"] = st.exchanges - before
        parts = [torch.zeros_like(torch.view_as_real(chunk)) for _ in range(world)] if rank == 0 else None
        dist.gather(torch.view_as_real(chunk), parts, dst=0)
        if rank == 0:
            out["diag_state"] = torch.view_as_complex(torch.cat(parts)).numpy().copy()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n,c", [(2, 8, 0), (2, 11, 2), (4, 10, 1), (4, 12, 3)])
def test_sharded_state_matches_oracle(world, n, c):
    seed = 100 * world + n
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, port, n, seed, c, out), nprocs=world, join=True,
                       start_method="spawn")
    ref = oracle.run(n, _random_circuit(n, 80, seed))
    assert np.abs(out["state"] - ref).max() < 1e-12
    assert out["exchanges"] > 0
    for r in range(world):
        assert abs(out[f"norm{r}"] - 1.0) < 1e-12
        assert out[f"diag_exchanges{r}"] == 0
    diag = W.gates([(W.CZ, n - 1, 0), (W.RZZ, n - 1, n - 2, 0.7), (W.T, n - 1, -1), (W.RZ, n - 2, -1, 0.3),
                    (W.S, 1, -1), (W.Z, n - 2, -1), (W.CZ, n - 1, n - 2)])
    ref_d = oracle.run(n, W.concat(W.gates([(W.H, q, -1) for q in range(n - 2)]), diag))
    assert np.abs(out["diag_state"] - ref_d).max() < 1e-12
