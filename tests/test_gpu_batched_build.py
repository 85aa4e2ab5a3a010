"""Batched Kernels 1 and 2 (one set of launches over every graph) against the
single-graph calls, bit for bit, and through them against the oracle; the
whole batched pipeline recorded as one CUDA graph against direct calls."""
import numpy as np
import pytest

from gpu_helpers import dev_u32, host_u32, rank_errors
from test_gpu_parity import check_k2

pytestmark = pytest.mark.gpu

GRAPH_FIELDS = ("colptr", "d_in", "d_out", "inv_dout32", "inv_dout64", "perm", "iperm")


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp

    return pp


def same_graph(a, b):
    import torch

    ia, ib = a.info_dict(), b.info_dict()
    assert ia == ib, (ia, ib)
    for f in GRAPH_FIELDS:
        assert torch.equal(getattr(a, f), getattr(b, f)), f
    nnz, novf = ia["nnz"], ia["novf"]
    assert torch.equal(a.rowc[:nnz], b.rowc[:nnz])
    assert torch.equal(a.ovf_key[:novf], b.ovf_key[:novf]) and torch.equal(a.ovf_cnt[:novf], b.ovf_cnt[:novf])


def batch_inputs(k0, scales, seed, Ms=None):
    us, vs = [], []
    for g, s in enumerate(scales):
        M = None if Ms is None else Ms[g]
        u, v = k0.edges_device(s, seed, graph=g, M=M) if M != 0 else (dev_u32([]), dev_u32([]))
        us.append(u)
        vs.append(v)
    return us, vs


@pytest.mark.parametrize("rule", ["lowest", "all_ties"])
def test_batched_k1_k2_equal_single_calls_and_oracle(pp, k0, oracle_mod, rule):
    import torch

    scales = [1, 4, 9, 12, 7, 14, 10, 5, 13, 3]
    Ms = [None, 37, 0, None, 1000, None, 16 * 1024 - 5, None, None, 9]
    us, vs = batch_inputs(k0, scales, 17, Ms)
    sorted_b = pp.sort_edges_batched(us, vs, scales)
    graphs_b = pp.build_filter_normalize_batched(sorted_b, scales, rule)
    assert pp.last_device_error() == 0
    for g, s in enumerate(scales):
        su, sv = pp.sort_edges(us[g], vs[g], s)
        assert torch.equal(sorted_b[g][0], su) and torch.equal(sorted_b[g][1], sv), g
        single = pp.build_filter_normalize(su, sv, s, rule)
        same_graph(graphs_b[g], single)
        ous, ovs = oracle_mod.k1_sort(host_u32(us[g]), host_u32(vs[g]))
        assert np.array_equal(host_u32(sorted_b[g][0]), ous) and np.array_equal(host_u32(sorted_b[g][1]), ovs)
        check_k2(pp, graphs_b[g], oracle_mod.k2_filter(ous, ovs, 1 << s, rule))
    assert pp.last_device_error() == 0


def test_batched_counts_beyond_the_union_and_graph_fields(pp, oracle_mod):
    """Duplicates counted past the union's count field (which is narrower)
    and past a graph's own field (its overflow table)."""
    import torch

    rng = np.random.default_rng(8)
    scales = [20, 16, 6]
    us, vs = [], []
    for s in scales:
        N = 1 << s
        cmax = (1 << (32 - s)) - 1
        u = list(rng.integers(0, N, 4000))
        v = list(rng.integers(0, N, 4000))
        u += list(rng.integers(0, N, 3 * cmax + 50))
        v += [N // 3] * (3 * cmax + 50)          # the supernode
        for a, b, c in ((1, 2, cmax + 2), (N - 1, 2, 600), (3, N - 2, cmax - 1)):
            u += [a] * c + [(a + 5) % N]
            v += [b] * c + [b]
        p = rng.permutation(len(u))
        us.append(dev_u32(np.array(u)[p]))
        vs.append(dev_u32(np.array(v)[p]))
    sorted_b = pp.sort_edges_batched(us, vs, scales)
    graphs_b = pp.build_filter_normalize_batched(sorted_b, scales)
    for g, s in enumerate(scales):
        su, sv = pp.sort_edges(us[g], vs[g], s)
        single = pp.build_filter_normalize(su, sv, s)
        same_graph(graphs_b[g], single)
        R = oracle_mod.k2_filter(host_u32(su), host_u32(sv), 1 << s)
        check_k2(pp, graphs_b[g], R)
        assert graphs_b[g].info_dict()["novf"] >= 1
    assert pp.last_device_error() == 0


def test_batched_64_graph_configuration(pp, k0, oracle_mod):
    """The batched benchmark's 64 graphs (scales 12..18): every graph equal to
    the single-graph calls; a few graphs' ranks from the batched Kernel 3 on
    the batched graphs against the oracle."""
    import torch

    scales = k0.batch_scales(64, 12, 18, seed=1)
    us, vs = batch_inputs(k0, scales, 1)
    sorted_b = pp.sort_edges_batched(us, vs, scales)
    graphs_b = pp.build_filter_normalize_batched(sorted_b, scales)
    for g, s in enumerate(scales):
        su, sv = pp.sort_edges(us[g], vs[g], s)
        assert torch.equal(sorted_b[g][0], su) and torch.equal(sorted_b[g][1], sv), g
        same_graph(graphs_b[g], pp.build_filter_normalize(su, sv, s))
    nrhs = 4
    r0 = np.concatenate([np.stack([k0.r0_host(1 << s, 1, graph=g, rhs=j) for j in range(nrhs)], axis=1)
                         for g, s in enumerate(scales)])
    got = pp.pagerank_batched(graphs_b, torch.from_numpy(r0).cuda(), nrhs).cpu().numpy()
    row = np.cumsum([0] + [1 << s for s in scales])
    for g in (0, 17, 63):
        R = oracle_mod.k2_filter(host_u32(sorted_b[g][0]), host_u32(sorted_b[g][1]), 1 << scales[g])
        for j in range(nrhs):
            want = oracle_mod.k3_pagerank(R, r0[row[g]:row[g + 1], j], 20, 0.85)
            e = rank_errors(got[row[g]:row[g + 1], j], want)
            assert e["l1"] <= 1e-6 and e["max_rel"] <= 1e-4, (g, j, e)
    assert pp.last_device_error() == 0


def test_batched_pipeline_graph_replay(pp, k0):
    """Kernels 1-3 of a batch as one CUDA graph: its replay equals the direct calls."""
    import torch

    scales = [9, 12, 10, 11, 8]
    us, vs = batch_inputs(k0, scales, 23)
    nrhs = 32
    r0 = np.concatenate([np.stack([k0.r0_host(1 << s, 23, graph=g, rhs=j) for j in range(nrhs)], axis=1)
                         for g, s in enumerate(scales)])
    r0d = torch.from_numpy(r0).cuda()
    ex = pp.BatchedPipelineExec(us, vs, scales, r0d, nrhs)
    for _ in range(2):
        got = ex.launch().clone()
    torch.cuda.synchronize()
    sorted_b = pp.sort_edges_batched(us, vs, scales)
    graphs_b = pp.build_filter_normalize_batched(sorted_b, scales)
    want = pp.pagerank_batched(graphs_b, r0d, nrhs)
    assert torch.equal(got, want)
    for g in range(len(scales)):
        same_graph(ex.graphs[g], graphs_b[g])
    ex.close()
    assert pp.last_device_error() == 0


def test_batched_out_of_range_id_is_reported(pp):
    us = [dev_u32([1, 2, 3]), dev_u32([0, 64, 5])]  # 64 >= 2^6
    vs = [dev_u32([0, 1, 2]), dev_u32([1, 2, 3])]
    pp.last_device_error()
    pp.sort_edges_batched(us, vs, [4, 6])
    assert pp.last_device_error() & pp.DEV_RANGE
