"""The N > 1 host logic of bench.py on CPU ranks (gloo, world size 2): process-group set-up from
the launcher's environment, the max over ranks of the timed region, the whole-job throughput
of the replicas, and the reference arm doing no work on ranks other than 0."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, local, ws, dist = bench.dist_setup()
    try:
        ms = [120.0, 150.0][r]  # rank 1 is the slow one
        ms_max = bench.max_over_ranks(ms, dist)
        bench.barrier(dist)
        value = bench.job_throughput(ws, 1000, 10, ms_max)
        out = io.StringIO()
        with contextlib.redirect_stdout(out):
            if r != 0:
                bench.run_reference(None, r, ws, dist)  # returns before touching its arguments
        q.put((r, local, ws, ms_max, value, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, local, ws, ms_max, value, printed) in enumerate(res):
        assert (rank, local, ws) == (r, r, 2)
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 1000 * 10 / 0.150)
        assert printed == ""


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("WORLD_SIZE",) if k in os.environ}
    try:
        assert bench.dist_setup() == (0, 0, 1, None)
        assert bench.max_over_ranks(3.5, None) == 3.5
        assert bench.job_throughput(1, 10, 4, 2000.0) == pytest.approx(20.0)
    finally:
        os.environ.update(env)
