"""The replicas-only multi-GPU bookkeeping of bench.py, on two CPU ranks
(gloo): barriers, the maximum of the per-rank times, and the whole-job
throughput (every rank's units over the slowest rank's time).  The
operator itself needs no exchange between ranks, so nothing else is
distributed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r = bench.Ranks(dist, "cpu")
    r.barrier()
    t_max = r.allmax(10.0 + rank)          # rank 1 is the slower one
    value = bench.job_throughput(world, 1000, 3264, t_max)
    r.barrier()
    q.put((rank, t_max, value))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        for p in procs:
            p.join(timeout=120)
    finally:
        for p in procs:          # a hung rank must not outlive the test
            if p.is_alive():
                p.terminate()
                p.join(timeout=10)
    for p in procs:
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for _, t_max, value in out:
        assert t_max == 11.0
        assert value == pytest.approx(2 * 1000 * 3264 / 11e-3 / 1e9)


def test_single_rank_is_identity():
    import bench
    r = bench.Ranks(None)
    r.barrier()
    assert r.allmax(3.5) == 3.5
    assert bench.job_throughput(1, 10, 100.0, 1.0) == pytest.approx(1e-3)
