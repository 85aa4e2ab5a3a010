"""Batched Kernel 3 (several graphs x several start vectors, binary32) against
the oracle and the single-vector binary64 GPU path."""
import numpy as np
import pytest

from gpu_helpers import host_u32, rank_errors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp

    return pp


def build_batch(pp, k0, scales, seed):
    """Kernels 1-2 on the GPU for each graph; returns graphs and host edge lists."""
    graphs, edges = [], []
    for g, s in enumerate(scales):
        u, v = k0.edges_device(s, seed, graph=g)
        us, vs = pp.sort_edges(u, v, s)
        graphs.append(pp.build_filter_normalize(us, vs, s))
        edges.append((host_u32(us), host_u32(vs)))
    return graphs, edges


def start_vectors(k0, scales, nrhs, seed):
    return np.concatenate([np.stack([k0.r0_host(1 << s, seed, graph=g, rhs=j) for j in range(nrhs)], axis=1)
                           for g, s in enumerate(scales)])


def check_against_oracle(oracle_mod, got, scales, edges, r0, pairs):
    row = np.cumsum([0] + [1 << s for s in scales])
    for g, j in pairs:
        N = 1 << scales[g]
        R = oracle_mod.k2_filter(edges[g][0], edges[g][1], N)
        want = oracle_mod.k3_pagerank(R, r0[row[g]:row[g + 1], j], 20, 0.85)
        e = rank_errors(got[row[g]:row[g + 1], j], want)
        assert e["l1"] <= 1e-6 and e["max_rel"] <= 1e-4, (g, j, e)


@pytest.mark.parametrize("nrhs", [32, 5, 1])
def test_batched_small_vs_oracle(pp, k0, oracle_mod, nrhs):
    import torch

    scales = [6, 9, 10, 12, 8, 11, 10, 7]
    graphs, edges = build_batch(pp, k0, scales, 11)
    r0 = start_vectors(k0, scales, nrhs, 5)
    got = pp.pagerank_batched(graphs, torch.from_numpy(r0).cuda(), nrhs).cpu().numpy()
    assert pp.last_device_error() == 0
    check_against_oracle(oracle_mod, got, scales, edges, r0,
                         [(g, j) for g in range(len(scales)) for j in range(nrhs)])


def test_batched_deterministic_and_matches_single_vector_path(pp, k0):
    import torch

    scales = [10, 12, 9, 13]
    graphs, _ = build_batch(pp, k0, scales, 17)
    r0 = start_vectors(k0, scales, 32, 9)
    r0d = torch.from_numpy(r0).cuda()
    a = pp.pagerank_batched(graphs, r0d, 32)
    b = pp.pagerank_batched(graphs, r0d, 32)
    assert torch.equal(a, b)
    row = np.cumsum([0] + [1 << s for s in scales])
    for g in range(len(scales)):
        for j in (0, 13, 31):
            single = pp.pagerank(graphs[g], r0d[row[g]:row[g + 1], j].contiguous(), 20, 0.85, "fp64").cpu().numpy()
            e = rank_errors(a[row[g]:row[g + 1], j].cpu().numpy(), single)
            assert e["l1"] <= 1e-6 and e["max_rel"] <= 1e-4, (g, j, e)


def test_batched_iteration_counts(pp, k0, oracle_mod):
    import torch

    scales = [8, 7]
    graphs, edges = build_batch(pp, k0, scales, 3)
    r0 = start_vectors(k0, scales, 4, 2)
    row = np.cumsum([0] + [1 << s for s in scales])
    for iters in (0, 1, 3):
        got = pp.pagerank_batched(graphs, torch.from_numpy(r0).cuda(), 4, iters=iters).cpu().numpy()
        for g in range(2):
            R = oracle_mod.k2_filter(edges[g][0], edges[g][1], 1 << scales[g])
            for j in range(4):
                want = oracle_mod.k3_pagerank(R, r0[row[g]:row[g + 1], j], iters, 0.85)
                assert rank_errors(got[row[g]:row[g + 1], j], want)["l1"] <= 1e-6


@pytest.mark.slow
def test_batched_64_graphs_scales_12_to_18(pp, k0, oracle_mod):
    """The batch shape of the benchmark's batched configuration: 64 graphs,
    scales drawn from 12..18, 32 start vectors each."""
    import torch

    scales = k0.batch_scales(64, 12, 18, seed=1)
    graphs, edges = build_batch(pp, k0, scales, 1)
    r0 = start_vectors(k0, scales, 32, 1)
    r0d = torch.from_numpy(r0).cuda()
    got = pp.pagerank_batched(graphs, r0d, 32)
    assert pp.last_device_error() == 0
    gotn = got.cpu().numpy()
    row = np.cumsum([0] + [1 << s for s in scales])
    rng = np.random.default_rng(0)
    for g in rng.choice(64, size=6, replace=False):
        for j in rng.choice(32, size=3, replace=False):
            single = pp.pagerank(graphs[g], r0d[row[g]:row[g + 1], j].contiguous(), 20, 0.85, "fp64").cpu().numpy()
            e = rank_errors(gotn[row[g]:row[g + 1], j], single)
            assert e["l1"] <= 1e-6 and e["max_rel"] <= 1e-4, (g, j, e)
    small = int(np.argmin(scales))
    check_against_oracle(oracle_mod, gotn, scales, edges, r0, [(small, 0), (small, 31)])


def test_batched_cuda_graph_replay(pp, k0):
    """The captured stage gives the direct call's result bit for bit, and a
    replay after refilling r0 in place gives the direct call's result for the
    new start vectors."""
    import torch

    scales = [9, 12, 10]
    graphs, _ = build_batch(pp, k0, scales, 23)
    r0d = torch.from_numpy(start_vectors(k0, scales, 32, 4)).cuda()
    direct = pp.pagerank_batched(graphs, r0d, 32)
    before = pp.launch_count()
    ex = pp.BatchedExec(graphs, r0d, 32)
    assert pp.launch_count() == before, "capture must not count as launches"
    got = ex.launch().clone()
    torch.cuda.synchronize()
    assert pp.launch_count() > before
    assert torch.equal(got, direct)
    r0d.copy_(torch.from_numpy(start_vectors(k0, scales, 32, 8)))
    direct2 = pp.pagerank_batched(graphs, r0d, 32)
    got2 = ex.launch().clone()
    torch.cuda.synchronize()
    assert pp.last_device_error() == 0
    assert torch.equal(got2, direct2)
    assert not torch.equal(got2, got)
    ex.close()


def test_batched_capture_argument_error(pp, k0):
    import torch

    scales = [8]
    graphs, _ = build_batch(pp, k0, scales, 2)
    r0d = torch.from_numpy(start_vectors(k0, scales, 4, 1)).cuda()
    with pytest.raises(pp.PPError):
        pp.BatchedExec(graphs, r0d, 4, iters=20, c=1.5)
    # the failed capture leaves the stream usable
    out = pp.pagerank_batched(graphs, r0d, 4)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
