"""Multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2).

Ranks solve independent problems (seed = rank) with no exchange of data; the only
collective is the max-over-ranks reduction of the timed region, and the reported rate
is every rank's units over the slowest rank's time.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    s = bench.make_inputs(seed=rank, edge=16)
    chk = torch.tensor([float(np.abs(s.phi).sum()), float(np.abs(s.psi).sum())], dtype=torch.float64)
    got = [torch.zeros_like(chk) for _ in range(world)]
    dist.all_gather(got, chk)
    ms = 10.0 + 5.0 * rank                       # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, dist, torch.device("cpu"))
    rate = bench.aggregate_rate(world, bench.SOLVES_PER_STEP, 4, ms_max)
    q.put((rank, [g.tolist() for g in got], ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import bench
    for rank, got, ms_max, rate in res:
        assert ms_max == 15.0                                    # the slowest rank's time
        assert rate == pytest.approx(2 * bench.SOLVES_PER_STEP * 4 / 0.015)
        # each rank's problem is the single-process one with seed = rank, and they differ
        for r in range(world):
            s = bench.make_inputs(seed=r, edge=16)
            assert got[r] == pytest.approx([float(np.abs(s.phi).sum()), float(np.abs(s.psi).sum())], rel=1e-12)
        assert got[0] != got[1]


def test_single_rank_helpers():
    import bench
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.aggregate_rate(1, 648, 10, 1000.0) == pytest.approx(6480.0)
