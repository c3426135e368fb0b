"""The N > 1 path of bench.py on CPU with world_size-2 gloo process groups:
replica seeds per rank, the max over ranks of the timed region and the
whole-job value (the GPU part of each rank is independent; there is no
collective on the data path)."""

import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist

    import bench
    from synth import make_maps

    dist.init_process_group("gloo", rank=rank, world_size=world)
    seed = bench.replica_seed(bench.WORKLOAD["seed"], rank)
    maps = make_maps(8, 8, 8, corr_len=2.0, seed=seed)
    local_ms = 10.0 + 5.0 * rank                   # ranks finish at different times
    dist.barrier()
    t = bench.max_over_ranks(local_ms, dist, "cpu")
    value = bench.job_value(world, 8 ** 3, 4, t)
    out.put((rank, seed, float(maps.p_cell.sum()), t, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_and_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0, t0, v0), (r1, s1, m1, t1, v1) = res
    assert (r0, r1) == (0, 1) and s1 == s0 + 1 and m0 != m1     # own replicate per rank
    assert t0 == t1 == 15.0                                       # the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 8 ** 3 * 4 / 0.015)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(12.5, None, "cpu") == 12.5
    assert bench.job_value(1, 100, 2, 1000.0) == 200.0
