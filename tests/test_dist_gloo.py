"""The multi-process path of bench.py (one replica per rank) on CPU with the
gloo backend, world size 2: barrier, max over ranks of the timed duration,
whole-job value, and the reference arm staying silent off rank 0."""
import contextlib
import io
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.dist_barrier(world)
        ms_local = 10.0 + 5.0 * rank        # rank 1 is the slowest
        ms = bench.max_over_ranks_of(ms_local, world, "cpu")
        bench.dist_barrier(world)
        out[rank] = (ms, bench.replicas_value(1000, 20, ms, world))
    finally:
        dist.destroy_process_group()


def test_replicas_aggregate_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == 15.0                                 # the max over ranks, seen by every rank
        assert value == pytest.approx(2 * 1000 * 20 / 15e-3)   # all ranks' updates over the slowest time


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks_of(3.5, 1, "cpu") == 3.5
    bench.dist_barrier(1)
    assert bench.replicas_value(10, 4, 2.0, 1) == pytest.approx(20000.0)


def test_reference_arm_prints_nothing_off_rank_zero():
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(None, rank=1, world=2)
    assert buf.getvalue() == ""
