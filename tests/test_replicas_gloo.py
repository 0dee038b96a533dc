"""The multi-GPU form of this path is replicas: every rank advances its own
copy of the workload with no collective on the data path; the benchmark takes
the slowest rank's time.  This checks that host logic with two gloo ranks on
the CPU (no GPU involved)."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local = [1.0 + rank, 10.0 - 3 * rank]
    got = bench.reduce_max_over_ranks(local)
    value = bench.whole_job_mlups(world, 2048 * 2048, 100, got[0])
    dist.barrier()
    q.put((rank, got, value))
    dist.destroy_process_group()


def test_two_rank_max_and_whole_job_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, value in res:
        assert got == [2.0, 10.0]
        assert value == pytest.approx(2 * 2048 * 2048 * 100 / 2.0 / 1e6)


def test_single_process_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max_over_ranks([3.0, 4.0]) == [3.0, 4.0]
    assert bench.whole_job_mlups(1, 1000, 10, 1e-3) == pytest.approx(10.0)
