"""Failure detection across ranks, on the CPU with gloo: one of two ranks
fails in the middle of the row-decomposed pipeline (its Kernel 2 step
raises, as a failed C call would through the binding); the other rank does
not hang in its next collective but gets an error within the process
group's timeout, and both processes end.  Nothing runs on a GPU."""
import datetime
import multiprocessing as mp
import os
import socket
import sys
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCALE, SEED = 10, 5
TIMEOUT_S = 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import kernel0
    from paper_1603_01876_gb300 import parallel
    from row_ops_numpy import NumpyRowOps

    class FailingOps(NumpyRowOps):
        def build_rows(self, us, vs, d_in_all, rule):
            raise RuntimeError("pp_build_filter_normalize_rows failed: injected")

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=TIMEOUT_S))
    t0 = time.monotonic()
    try:
        N = 1 << SCALE
        u, v = kernel0.edges_host(SCALE, SEED)
        M = len(u)
        a, b = rank * M // world, (rank + 1) * M // world
        bounds = parallel.row_bounds(N, world)
        r0 = kernel0.r0_host(N, SEED)[bounds[rank]:bounds[rank + 1]]
        ops = FailingOps(SCALE) if rank == 1 else NumpyRowOps(SCALE)
        parallel.pipeline(ops, parallel.Comm(), torch.from_numpy(u[a:b].view(np.int32)),
                          torch.from_numpy(v[a:b].view(np.int32)), SCALE, torch.from_numpy(r0.copy()), 20, 0.85)
        q.put((rank, "finished", time.monotonic() - t0))
    except Exception as e:  # the failure, or its effect on the other rank
        q.put((rank, type(e).__name__ + ": " + str(e)[:200], time.monotonic() - t0))
    # no destroy_process_group: the peer may be gone


def test_a_failing_rank_does_not_hang_the_other():
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (msg, t)) for r, msg, t in (q.get(timeout=TIMEOUT_S + 120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert "injected" in out[1][0]
    assert out[0][0] != "finished", out[0]  # rank 0 learned of the failure through its collective
    assert out[0][1] <= TIMEOUT_S + 60, out[0]
