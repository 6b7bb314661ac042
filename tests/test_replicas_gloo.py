"""The N > 1 path of bench.py on CPU: two gloo ranks, each timing its own
replica; the reported time is the slowest rank's and the rate counts both
ranks' work (replicas only: the GEMM has no exchange step)."""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [120.0, 150.0][rank]
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 2.0 * 2048**3, 5, t)
    dist.barrier()
    q.put((rank, t, rate))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in out:
        assert t == 150.0
        assert rate == pytest.approx(2 * 2.0 * 2048**3 * 5 / 0.150 / 1e9)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.whole_job_rate(1, 2.0, 10, 1000.0) == pytest.approx(2e-8)
