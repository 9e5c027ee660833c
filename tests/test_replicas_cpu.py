"""The N > 1 path of bench.py is independent replicas: each rank steps its own problem and
only the timing crosses ranks (the slowest rank over all steps of all ranks).  Two gloo
ranks on CPU check that reduction and the per-rank seeds."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    t_local = [2.0, 3.0][rank]                       # rank 1 is the slower one
    v = bench.job_seconds_per_step(t_local, steps=10, world=world, dist=dist, device="cpu")
    out[rank] = v
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    torch = pytest.importorskip("torch")
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_gloo_available():
        pytest.skip("no gloo")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    # 2 ranks x 10 steps in max(2, 3) = 3 s: 0.15 s per step for the whole job, on every rank
    assert out[0] == pytest.approx(0.15) and out[1] == pytest.approx(0.15)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_seconds_per_step(2.0, steps=4, world=1) == pytest.approx(0.5)


def test_replicas_get_distinct_seeds():
    """Rank r builds its mesh with seed 11 + r: same workload, differently jittered grids."""
    import numpy as np
    import bench
    a = bench.make_problem("grf128_p3", seed=11 + 0)
    b = bench.make_problem("grf128_p3", seed=11 + 1)
    assert a[0] == b[0] and np.array_equal(a[2], b[2])   # same config and connectivity
    assert not np.array_equal(a[1], b[1])                 # different vertex jitter
