"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): the timed
region's length is the slowest rank's, and the whole-job rate counts the
units of every rank over that time.  The GPU path runs one independent
replica per rank (no data-path collective), so this reduction is the only
exchange between ranks."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ms = [120.0, 150.0][rank]               # rank 1 is the slow one
        slowest = b.max_over_ranks(ms, dist)
        rate = b.whole_job_rate(world, 5, slowest / 1e3)
        out[rank] = (slowest, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for r in range(world):
        slowest, rate = res[r]
        assert slowest == 150.0
        assert rate == pytest.approx(2 * 5 / 0.150)


def test_single_process_keeps_its_own_time():
    b = _bench()
    assert b.max_over_ranks(42.0, None) == 42.0
    assert b.whole_job_rate(1, 4, 2.0) == 2.0
