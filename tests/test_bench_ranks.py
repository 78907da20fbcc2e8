"""The multi-process side of bench.py on CPU (gloo, world size 2): every rank
gets the slowest rank's time and the whole-job rate from it, as the
benchmark reports for N replicas."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms, out):
    import torch.distributed as td
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    td.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    res = bench.job_rate(ms[rank], 100, world, device="cpu")
    td.destroy_process_group()
    out.put((rank, res))


def test_job_rate_takes_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ms = [250.0, 400.0]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, ms, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        t, v = res[r]
        assert t == 400.0
        assert v == pytest.approx(100 * 2 / 0.4)


def test_job_rate_single_process():
    import bench
    assert bench.job_rate(500.0, 10, 1) == (500.0, 20.0)
