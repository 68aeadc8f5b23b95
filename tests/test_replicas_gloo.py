"""The multi-GPU path is independent replicas (one design per rank, no data-path
collective); the only cross-rank step is the timing reduction.  Exercised here
with two gloo ranks on the CPU."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        t = bench.max_over_ranks(0.010 * (rank + 1), world, device="cpu")
        v = bench.job_throughput(1000, t, world)
        q.put((rank, t, v))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    import socket

    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in out:
        assert t == pytest.approx(0.020)  # the slowest rank's time, on every rank
        assert v == pytest.approx(2 * 1000 / 0.020)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.5, 1) == 0.5
    assert bench.job_throughput(10, 2.0, 1) == 5.0
