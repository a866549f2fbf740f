"""The multi-GPU benchmark path on CPU: two gloo ranks run the same host logic
the bench runs under torchrun (replicas only: disjoint seeds, one MAX
reduction of the timed total, whole-job throughput)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import oracle as O
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        # each rank's replicas: the Philox draw keyed by its own seed
        x0 = O.init_uniform(4, 16, bench.rank_seed(r))
        local_ms = 10.0 + 5.0 * r  # rank 1 is the slower one
        total_ms, value = bench.job_time_and_value(local_ms, 1000, w)
        q.put((r, w, total_ms, value, x0))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_disjoint_replicas():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort(key=lambda t: t[0])
    for r, w, total_ms, value, _ in out:
        assert w == world
        assert total_ms == 15.0  # the slowest rank's time on every rank
        assert value == pytest.approx(1000 * world / 15e-3)  # all ranks' units
    # replicas only: the two ranks draw different initial states
    assert not np.array_equal(out[0][4], out[1][4])


def test_single_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_and_value(20.0, 500, 1) == (20.0, 500 / 20e-3)
    assert bench.rank_seed(0) == 0 and bench.rank_seed(3) != bench.rank_seed(2)
