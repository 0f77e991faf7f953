"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica with its
own step time; the job time is the slowest rank's and the job throughput is
world x per-rank bytes / that time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    dist.barrier()
    ms = [120.0, 180.0][rank]
    job_ms = bench.reduce_max(ms, dist, "cpu")
    value = bench.job_throughput(34.36e9, world, job_ms)
    out[rank] = (job_ms, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
    assert out[0] == out[1]
    job_ms, value = out[0]
    assert job_ms == 180.0
    assert abs(value - 2 * 34.36e9 / 0.18 / 1e9) < 1e-6


def test_single_rank_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert abs(bench.job_throughput(1e9, 1, 1000.0) - 1.0) < 1e-12
