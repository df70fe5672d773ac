"""Host-side logic of the benchmark's multi-rank path, on CPU: two gloo ranks (spawned processes)
reduce their step times to the slowest rank's, and the whole-job rate counts every rank's units over
that time; the reference arm does nothing on ranks other than 0."""
import os
import socket
import sys
import types

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


def _rank(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (ms, bench.job_rate(world, 1000.0, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world, times = 2, [3.0, 7.5]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), times, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 7.5
        assert rate == pytest.approx(world * 1000.0 / 7.5e-3 / 1e6)


def test_one_rank_is_its_own_time():
    assert bench.max_over_ranks(4.25, 1, "cpu") == 4.25
    assert bench.job_rate(1, 393216 * 10, 3.0) == pytest.approx(393216 * 10 / 3e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    args = types.SimpleNamespace(steps=1, warmup=1, gpus=2)
    assert bench.run_reference(args, rank=1) is None
    assert capsys.readouterr().out == ""
