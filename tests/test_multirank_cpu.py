"""The replica path of bench.py with more than one rank (torchrun, one replica per GPU), on CPU:
two gloo ranks agree on the slowest rank's time and report the whole-job rate; the reference arm
does no work on ranks other than 0."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, updates, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.job_rate(times[rank], updates, dist)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_two_gloo_ranks():
    times, updates = [12.5, 20.0], 4_000_000
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, free_port(), times, updates, out), nprocs=2, join=True)
        res = dict(out)
    for r in (0, 1):
        ms, value = res[r]
        assert ms == 20.0
        assert value == pytest.approx(2 * updates / 20e-3 / 1e6)


def test_job_rate_single_process():
    ms, value = bench.job_rate(8.0, 1_000_000)
    assert ms == 8.0 and value == pytest.approx(1e6 / 8e-3 / 1e6)


def test_reference_arm_does_nothing_off_rank_zero(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup = 1, 0

    assert bench.run_reference(Args()) is None
    assert capsys.readouterr().out == ""


def test_bench_rejects_a_16bit_cavity():
    """The power-law cavity workload is FP32 only: the command line says so before any GPU work."""
    import subprocess
    import sys

    r = subprocess.run([sys.executable, os.path.join(os.path.dirname(bench.__file__), "bench.py"), "--workload",
                        "cavity", "--precision", "fp16s"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "FP32" in r.stderr
