"""Replica runs (bench.py --gpus N): each rank solves its own copy of the workload,
the job's step time is the slowest rank's (max over ranks), the throughput counts
every rank's work.  Two gloo ranks on the CPU exercise the reduction; no GPU."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [3.0, 7.5][rank]
    out[rank] = bench.max_over_ranks(local, world)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == 7.5 and out[1] == 7.5


def test_job_throughput_counts_every_replica():
    import bench
    assert bench.max_over_ranks(4.0, 1) == 4.0
    one = bench.job_throughput(1, 9600 ** 2 * 19, 2.5)
    assert abs(bench.job_throughput(4, 9600 ** 2 * 19, 2.5) - 4 * one) < 1e-9 * one
