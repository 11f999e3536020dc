"""The multi-rank timing path of bench.py (replicas: every rank renders its
own copy of the workload, no collective on the data path; ranks agree only on
the slowest time) with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 180.0][rank]
    slow = bench.reduce_max_over_ranks(ms, dist, "cpu")
    q.put((rank, slow, bench.job_throughput(64 * 10, world, slow)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_slowest_time_and_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[1] for r in res] == [180.0, 180.0]
    assert all(abs(r[2] - 64 * 10 * 2 / 0.18) < 1e-6 for r in res)


def test_single_rank_needs_no_group():
    import bench
    assert bench.reduce_max_over_ranks(5.0, None, "cpu") == 5.0
    assert bench.job_throughput(64, 1, 1000.0) == 64.0
