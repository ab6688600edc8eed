"""The N > 1 bench path on CPU: two gloo ranks (127.0.0.1), each timing its own replica; the
job time is the slowest rank's and the value counts every rank's units; the reference arm
prints on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist)
    out.put((rank, ms, bench.job_value(1000, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time():
    world, times = 2, [10.0, 30.0]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 30.0
        assert value == pytest.approx(2 * 1000 / 0.030)



def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_value(8192 * 3, 1, 500.0) == pytest.approx(8192 * 3 / 0.5)


def test_reference_arm_prints_on_rank_zero_only():
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 0, 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(A, "c1", rank=1)
    assert buf.getvalue() == ""
