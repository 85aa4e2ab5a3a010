"""The row-decomposed form of Kernels 1-3 (paper_1603_01876_gb300.parallel)
with two or three gloo ranks on the CPU (three: ragged row ranges), against the oracle's single-rank pipeline:
the ranks' sorted edges one after the other equal Kernel 1's output, every
rank's rows of the filtered A and the global in-degree equal Kernel 2's, and
the ranks one after the other equal Kernel 3's within 1e-12 (binary64).  The
local steps run in a host stand-in (tests/row_ops_numpy.py); the exchange,
the sums over the ranks and the update order are the product's."""
import multiprocessing as mp
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCALE, SEED, ITERS = 10, 5, 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, rule, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch
    import torch.distributed as dist

    import kernel0
    from paper_1603_01876_gb300 import parallel
    from row_ops_numpy import NumpyRowOps

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        N = 1 << SCALE
        u, v = kernel0.edges_host(SCALE, SEED)
        M = len(u)
        a, b = rank * M // world, (rank + 1) * M // world
        bounds = parallel.row_bounds(N, world)
        r0 = kernel0.r0_host(N, SEED)[bounds[rank]:bounds[rank + 1]]
        us, vs, g, d_in, r = parallel.pipeline(
            NumpyRowOps(SCALE), parallel.Comm(), torch.from_numpy(u[a:b].view(np.int32)),
            torch.from_numpy(v[a:b].view(np.int32)), SCALE, torch.from_numpy(r0.copy()), ITERS, 0.85, rule)
        q.put((rank, us.numpy().view(np.uint32), vs.numpy().view(np.uint32), d_in.numpy(), g, r.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,rule", [(2, "lowest"), (2, "all_ties"), (3, "lowest")])
def test_ranks_equal_the_single_rank_pipeline(oracle_mod, k0, world, rule):
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, rule, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    N = 1 << SCALE
    u, v = k0.edges_host(SCALE, SEED)
    ous, ovs = oracle_mod.k1_sort(u, v)
    R = oracle_mod.k2_filter(ous, ovs, N, rule)
    want_r = oracle_mod.k3_pagerank(R, k0.r0_host(N, SEED), ITERS, 0.85)
    # Kernel 1: the ranks' lists one after the other
    assert np.array_equal(np.concatenate([o[1] for o in out]), ous)
    assert np.array_equal(np.concatenate([o[2] for o in out]), ovs)
    # Kernel 2: the global in-degree on every rank, every rank's rows
    rowptr = R["rowptr"].astype(np.int64)
    for rank, _, _, d_in, g, _ in out:
        assert np.array_equal(d_in.astype(np.uint32), R["d_in"])
        lo, hi = rank * N // world, (rank + 1) * N // world
        e0, e1 = rowptr[lo], rowptr[hi]
        o = np.lexsort((g["v"], g["u"]))
        assert np.array_equal(g["u"][o], np.repeat(np.arange(lo, hi), np.diff(rowptr[lo:hi + 1])))
        assert np.array_equal(g["v"][o], R["col"][e0:e1].astype(np.int64))
        assert np.array_equal(g["cnt"][o], R["cnt"][e0:e1].astype(np.int64))
        assert np.array_equal(g["d_out"][lo:hi], R["d_out"][lo:hi].astype(np.int64))
    # Kernel 3
    r = np.concatenate([o[5] for o in out])
    assert np.abs(r - want_r).sum() / np.abs(want_r).sum() <= 1e-12


def test_row_bounds_cover_every_vertex_once():
    sys.path.insert(0, ROOT)
    from paper_1603_01876_gb300 import parallel

    for N, P in ((1024, 2), (1024, 3), (16, 5), (8, 8)):
        b = parallel.row_bounds(N, P)
        assert b[0] == 0 and b[-1] == N and all(x <= y for x, y in zip(b, b[1:])) and len(b) == P + 1
