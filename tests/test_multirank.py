"""Host logic of the N > 1 benchmark path (replicas), on CPU ranks over gloo.

Every rank orthogonalizes its own problem; the job's time is the slowest
rank's and its throughput counts the bytes of all ranks.  Two processes with
different local times must agree on the maximum and on the whole-job value.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        local_ms = 100.0 + 50.0 * rank
        dist.barrier()
        worst = bench.max_over_ranks(local_ms)
        value = bench.replica_throughput(34359738368, 5, world, worst)
        out[rank] = (worst, value)
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    expect_ms = 150.0
    expect_val = 34359738368 * 2 * 5 / (expect_ms * 1e-3) / 1e9
    for r in range(2):
        worst, value = out[r]
        assert worst == pytest.approx(expect_ms)
        assert value == pytest.approx(expect_val)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(8e9, 2, 1, 1000.0) == pytest.approx(16.0)
