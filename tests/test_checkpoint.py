"""Stage checkpoints (paper_1603_01876_gb300.checkpoint): on the CPU, the
file round trip of edges, Kernel 2's arrays and ranks, keyed by (scale,
seed), with shape and scale checks; on the GPU, Kernel 3 on a reloaded
graph gives the same bits and a run resumed from saved ranks equals the
uninterrupted run within rounding."""
import numpy as np
import pytest


@pytest.fixture
def ck():
    from paper_1603_01876_gb300 import checkpoint

    return checkpoint


def test_round_trip_on_the_host(ck, tmp_path):
    import torch

    import paper_1603_01876_gb300 as pp

    scale, seed, M = 6, 3, 1000
    g = pp.Graph(M, scale, "cpu")
    rng = np.random.default_rng(0)
    for f in ck.GRAPH_FIELDS:
        t = getattr(g, f)
        t.copy_(torch.from_numpy(rng.integers(0, 1 << 20, t.numel()).astype(t.numpy().dtype)))
    ck.save_graph(tmp_path, scale, seed, g)
    h = ck.load_graph(tmp_path, scale, seed, device="cpu")
    for f in ck.GRAPH_FIELDS:
        assert torch.equal(getattr(g, f), getattr(h, f)), f
    with pytest.raises(ValueError):  # the key must name the graph's own scale
        ck.save_graph(tmp_path, scale + 1, seed, g)
    u = torch.from_numpy(rng.integers(0, 1 << scale, M).astype(np.int32))
    v = torch.from_numpy(rng.integers(0, 1 << scale, M).astype(np.int32))
    ck.save_edges(tmp_path, scale, seed, u, v, "sorted")
    u2, v2 = ck.load_edges(tmp_path, scale, seed, "sorted", device="cpu")
    assert torch.equal(u, u2) and torch.equal(v, v2)
    r = torch.from_numpy(rng.random(1 << scale))
    ck.save_ranks(tmp_path, scale, seed, r, 12)
    r2, k = ck.load_ranks(tmp_path, scale, seed, device="cpu")
    assert k == 12 and torch.equal(r, r2)
    # a file of another scale is refused
    import os

    os.replace(ck.stage_path(tmp_path, scale, seed, "graph"), ck.stage_path(tmp_path, scale + 2, seed, "graph"))
    with pytest.raises(ValueError):
        ck.load_graph(tmp_path, scale + 2, seed, device="cpu")


@pytest.mark.gpu
def test_reloaded_graph_and_resumed_ranks(ck, k0, tmp_path):
    import torch

    import paper_1603_01876_gb300 as pp

    scale, seed = 16, 9
    u, v = k0.edges_device(scale, seed)
    us, vs = pp.sort_edges(u, v, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    ck.save_edges(tmp_path, scale, seed, us, vs, "sorted")
    ck.save_graph(tmp_path, scale, seed, g)
    r0 = torch.from_numpy(k0.r0_host(1 << scale, seed)).cuda()
    h = ck.load_graph(tmp_path, scale, seed)
    us2, vs2 = ck.load_edges(tmp_path, scale, seed, "sorted")
    assert torch.equal(us, us2) and torch.equal(vs, vs2)
    for dt in ("fp64", "fp32"):
        a = pp.pagerank(g, r0, 20, 0.85, dt)
        assert torch.equal(a, pp.pagerank(h, r0, 20, 0.85, dt))
        r12 = pp.pagerank(h, r0, 12, 0.85, dt)
        ck.save_ranks(tmp_path, scale, seed, r12, 12, "ranks_" + dt)
        rk, k = ck.load_ranks(tmp_path, scale, seed, "ranks_" + dt)
        b = ck.pagerank_resume(h, rk, 20 - k, 0.85, dt)
        err = float((b.double() - a.double()).abs().sum() / a.double().abs().sum())
        assert err <= (1e-13 if dt == "fp64" else 2e-6), (dt, err)
    assert pp.last_device_error() == 0
