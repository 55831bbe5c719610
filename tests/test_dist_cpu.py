"""The multi-rank side of the benchmark on CPU: two gloo ranks (127.0.0.1).

bench.py under torchrun runs one replica of the workload per rank, takes the
slowest rank's timed region and reports world * steps solves in that time; the
reference arm runs on rank 0 alone.  These tests drive the same functions with
the gloo backend, so the aggregation is checked without a GPU.
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 180.0][rank]
        ms, value = bench.aggregate_over_ranks(local_ms, 10, world, dist, "cpu")
        # the reference arm prints on rank 0 only
        args = type("A", (), {"steps": 1, "warmup": 0})()
        buf = io.StringIO()
        if rank != 0:
            with redirect_stdout(buf):
                bench.run_reference(args, rank, world)
        q.put((rank, ms, value, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_work():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    got = sorted(q.get(timeout=5) for _ in range(world))
    for rank, ms, value, printed in got:
        assert ms == 180.0  # max over ranks
        assert abs(value - world * 10 / 0.180) < 1e-9  # whole-job solves per second
        if rank != 0:
            assert printed == ""  # non-zero ranks of the reference arm do no work


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate_over_ranks(250.0, 5, 1) == (250.0, 5 / 0.25)
