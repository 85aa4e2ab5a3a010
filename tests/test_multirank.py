"""The multi-GPU form is replicas: every rank runs its own graph and the job's
rate is the units all ranks processed over the slowest rank's time.  The
host-side part of that (per-rank seeds, the max over ranks, the job rate) is
exercised here with two gloo ranks on the CPU."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_env()
        slowest = bench.max_over_ranks(times[rank], w, "cpu")
        dist.barrier()
        q.put((r, bench.rank_seed(r), slowest, bench.job_rate(1000, w, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_distinct_graphs():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [12.5, 20.0]
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seed0, t0, rate0), (r1, seed1, t1, rate1) = out
    assert (r0, r1) == (0, 1) and seed0 != seed1
    assert t0 == t1 == 20.0  # every rank reports the slowest rank's time
    assert rate0 == rate1 == pytest.approx(2 * 1000 / 0.020)


def test_one_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.job_rate(1000, 1, 10.0) == pytest.approx(1e5)
