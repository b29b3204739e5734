"""N > 1 ranks: the bench runs independent replicas (no collective on the data
path); only the timing reduction is collective. Checked with world_size 2 on
the gloo backend (CPU)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.5][rank]
    mx = bench.reduce_max_ms(ms, dist, "cpu")
    val = bench.replica_throughput(1000, 10, world, mx)
    q.put((rank, mx, val))
    dist.destroy_process_group()


def test_replica_timing_reduction_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, val in res:
        assert mx == 55.5                       # the slowest rank bounds the job
        assert abs(val - 1000 * 10 * 2 / 0.0555) < 1e-6


def test_single_rank_reduction_is_identity():
    import bench
    assert bench.reduce_max_ms(12.5, None, "cpu") == 12.5
    assert bench.replica_throughput(100, 2, 1, 1000.0) == 200.0
