"""The N > 1 path of the benchmark on CPU: two gloo ranks (world size 2) run the
host-side logic bench.py uses under torchrun -- one independent system per rank
(no data-path collective), the barrier, the max-over-ranks time and the
whole-job throughput -- and the reference arm's rank filter."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, queue):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_seconds = 1.5 + rank          # rank 1 is the slow one
        t = bench.max_over_ranks(local_seconds, dist, "cpu")
        rate = bench.job_rate(world, 1000.0, t)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            class A:
                steps, warmup, gpus = 1, 3, world
            if rank != 0:
                bench.run_reference(A, rank, world)   # ranks other than 0 do no work
        queue.put((rank, bench.rank_seed(rank), t, rate, buf.getvalue()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, v0, out0), (r1, s1, t1, v1, out1) = res
    assert s0 != s1                         # each rank advances its own system
    assert t0 == t1 == 2.5                  # the job's time is the slowest rank's
    assert v0 == v1 == pytest.approx(2 * 1000.0 / 2.5)
    assert out1 == ""


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0) == 3.0
    assert bench.job_rate(1, 10.0, 2.0) == 5.0
