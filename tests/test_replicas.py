"""The multi-GPU path of the bench is replicas: each rank runs whole mocks on
its own seed and only the timing is combined (max over ranks).  Two gloo
ranks on the CPU check that logic; each rank's work is an oracle replica of a
tiny survey, which needs no exchange with the other rank."""
import math
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402
import mockgen  # noqa: E402
from oracle import power as op  # noqa: E402


def _tiny_power(seed):
    sv = mockgen.survey_small(N=32, assign=2)
    gal = mockgen.uniform_points(300, 420.0, 580.0, seed=seed)
    ran = mockgen.uniform_points(3000, 420.0, 580.0, seed=seed + 1000)
    geom = dict(L=1000.0, N=32, assign=2, origin=(0.0, 0.0, 0.0), observer=(500.0, 500.0, -2000.0))
    kf = 2 * math.pi / sv.L
    return op.power(gal, ran, geom, (0.5 * kf, kf, 8))["P0"]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.replica_seed(7, rank)
        p0 = _tiny_power(seed)
        step_s = 0.010 * (rank + 1)  # a slower second rank
        slowest = bench.max_over_ranks(step_s, world)
        q.put((rank, seed, p0, slowest, bench.job_rate(world, slowest)))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted([q.get(timeout=300) for _ in range(world)], key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, p0, m0, v0), (r1, s1, p1, m1, v1) = res
    assert (s0, s1) == (7, 8)  # the seed range is partitioned by rank
    assert m0 == m1 == pytest.approx(0.020)  # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(world / 0.020)  # whole-job mocks/s
    # each replica equals the same mock computed alone: no data-path exchange
    assert np.allclose(p0, _tiny_power(7), equal_nan=True)
    assert np.allclose(p1, _tiny_power(8), equal_nan=True)
    assert not np.allclose(p0, p1, equal_nan=True)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun only rank 0 times the oracle and prints the line."""
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    import argparse
    ns = argparse.Namespace(steps=1, warmup=0, seed=0)
    bench.run_reference(ns)
    assert capsys.readouterr().out == ""
