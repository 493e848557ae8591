"""The multi-process logic of bench.py on CPU (gloo, two ranks): each rank
times its own replica, the job's step time is the slowest rank's, the value
counts every rank's bytes, and the reference arm runs on rank 0 only."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 3.0 * rank, dist, "cpu")
        dist.barrier()
        out[rank] = (ms, bench.job_value(ms, world))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0][0] == out[1][0] == 13.0
    expected = world * bench.b_alg(bench.M, bench.N, bench.PASSES) / 13.0e-3 / 1e9
    assert out[0][1] == pytest.approx(expected) and out[1][1] == pytest.approx(expected)


def test_single_rank_passes_its_time_through():
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_value(7.5, 1) == pytest.approx(bench.b_alg(bench.M, bench.N, bench.PASSES) / 7.5e-3 / 1e9)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup, variant = 1, 0, "qr"

    assert bench.reference_arm(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
