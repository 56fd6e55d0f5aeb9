"""Host logic of the multi-GPU bench (replicas only), on CPU with two gloo ranks.

Each rank solves its own seeded instance; the job's rate is every rank's instances over the
slowest rank's timed region (a max all-reduce); the reference arm runs on rank 0 alone.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, local_ms, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        out[rank] = bench.replica_rate(local_ms[rank], steps, world, torch.device("cpu"))
    finally:
        dist.destroy_process_group()


def test_replica_rate_takes_the_slowest_rank():
    world, steps = 2, 3
    local_ms = [100.0, 150.0]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), local_ms, steps, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, total_ms = res[rank]
        assert total_ms == 150.0
        assert value == pytest.approx(world * steps / 0.150)


def test_single_rank_rate_needs_no_process_group():
    import bench
    value, total_ms = bench.replica_rate(250.0, 5, 1)
    assert total_ms == 250.0 and value == pytest.approx(20.0)


def test_ranks_draw_their_own_instances():
    import bench
    p0, p1 = bench.make_problem(bench.WORKLOAD, 0), bench.make_problem(bench.WORKLOAD, 1)
    assert p0.A.shape == p1.A.shape and p0.y.shape == p1.y.shape
    assert not np.array_equal(p0.y, p1.y)
    again = bench.make_problem(bench.WORKLOAD, 1)
    assert np.array_equal(again.y, p1.y) and np.array_equal(again.A, p1.A)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    ran = []
    monkeypatch.setattr(bench, "oracle_sample", lambda *a, **k: ran.append(1) or {"value": 1.0})
    bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=2))
    assert ran == [] and capsys.readouterr().out == ""
