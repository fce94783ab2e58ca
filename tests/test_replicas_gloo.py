"""The multi-GPU path of the benchmark is replicas only: every rank times its own copy of
the workload, the job's time is the slowest rank's, and the throughput is all ranks'
units over that time.  Checked here with two gloo ranks on the CPU (127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(dist, 1.0 + rank, "cpu")      # rank r took 1 + r seconds
        out[rank] = (t, bench.replica_throughput(world, 100.0, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 100.0)     # max(1, 2) s; 2 ranks x 100 units / 2 s


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(None, 1.5, "cpu") == 1.5
    assert bench.replica_throughput(1, 30.0, 1.5) == 20.0
