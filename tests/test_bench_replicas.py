"""The multi-GPU path of bench.py is replicas (each rank solves its own copy,
no data exchange): the timed region's length is the maximum over ranks and
the whole-job value is all ranks' units over it.  Checked here with two gloo
ranks on the CPU; the reference arm runs on rank 0 only."""

import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        local_ms = 100.0 + 50.0 * rank
        m = b.max_over_ranks(local_ms, True, "cpu")
        v = b.job_value(1.0e9, world, m)
        out[rank] = (m, v)
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_time_and_the_sum_of_units():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        m, v = out[r]
        assert m == 150.0
        assert abs(v - 2.0e9 / 0.15) < 1e-3 * v


def test_single_process_needs_no_collective():
    b = _bench()
    assert b.max_over_ranks(12.5, False, "cpu") == 12.5
    assert b.job_value(3.0, 1, 1000.0) == 3.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    b = _bench()

    class Args:
        N, cpu_rows, warmup, steps, gpus = 50, 1, 0, 1, 2

    b.run_reference(Args(), rank=1)
    assert capsys.readouterr().out == ""
