"""Multi-GPU path of the benchmark on CPU ranks (gloo): the work does not
shard, so N ranks are N independent replicas; the only collective is the
max over ranks of the step time, and the job throughput counts every
replica's batch."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + rank, world)
    out[rank] = ms
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_step():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    assert dict(out) == {0: 11.0, 1: 11.0}


def test_job_throughput_counts_every_replica():
    import bench
    one = bench.job_throughput(1, 64, 1.048576, 250.0)
    assert abs(one - 64 * 1.048576 / 0.25) < 1e-9
    assert abs(bench.job_throughput(4, 64, 1.048576, 250.0) - 4 * one) < 1e-9
    assert bench.reduce_max(3.5, 1) == 3.5
