"""Host logic of bench.py's multi-GPU path (independent replicas, no collective
on the data path), run as two gloo ranks on the CPU: the job's timed region
is the maximum over ranks, the whole-job rate counts every rank's
invocations, and the reference arm runs on rank 0 only."""
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        t_loc = [0.25, 0.75][rank]  # the second rank is the slower one
        t_all = bench.job_time(t_loc, world, "cpu")
        out[rank] = (t_all, bench.per_invocation(t_all, 10, world))
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_the_rate_counts_all_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    t_all, s_per_iter = res[0]
    assert t_all == 0.75
    assert s_per_iter == pytest.approx(0.75 / 20)


def test_single_rank_needs_no_process_group():
    assert bench.job_time(1.5, 1, "cpu") == 1.5
    assert bench.per_invocation(1.5, 3, 1) == pytest.approx(0.5)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(None) is None  # returns before reading its arguments
    assert buf.getvalue() == ""
