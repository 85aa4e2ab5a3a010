"""GPU parity on hand-built inputs: the degenerate cases of Kernels 1-3."""
import numpy as np
import pytest

from gpu_helpers import dev_u32, gpu_triples, host_u32, oracle_triples, rank_errors
from test_gpu_parity import check_k2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp

    return pp


def run_and_compare(pp, oracle_mod, u, v, scale, rules=("lowest", "all_ties"), dtypes=("fp64", "fp32"), iters=20):
    import torch

    u = np.asarray(u, dtype=np.uint32)
    v = np.asarray(v, dtype=np.uint32)
    N = 1 << scale
    us, vs = pp.sort_edges(dev_u32(u), dev_u32(v), scale)
    ous, ovs = oracle_mod.k1_sort(u, v)
    assert np.array_equal(host_u32(us), ous) and np.array_equal(host_u32(vs), ovs)
    r0 = np.random.default_rng(scale).random(N) + 0.05
    r0d = torch.from_numpy(r0).cuda()
    graphs = {}
    for rule in rules:
        g = pp.build_filter_normalize(us, vs, scale, rule)
        R = oracle_mod.k2_filter(ous, ovs, N, rule)
        check_k2(pp, g, R)
        want = oracle_mod.k3_pagerank(R, r0, iters, 0.85)
        for dt in dtypes:
            got = pp.pagerank(g, r0d, iters, 0.85, dt).cpu().numpy()
            e = rank_errors(got, want)
            assert e["l1"] <= (1e-12 if dt == "fp64" else 1e-6), (rule, dt, e)
            if dt == "fp32":
                assert e["max_rel"] <= 1e-4, (rule, e)
        graphs[rule] = (g, R)
    assert pp.last_device_error() == 0
    return graphs


def test_no_edges(pp, oracle_mod):
    graphs = run_and_compare(pp, oracle_mod, [], [], 5)
    g, R = graphs["lowest"]
    assert g.info_dict()["nnz"] == 0


def test_single_edge(pp, oracle_mod):
    run_and_compare(pp, oracle_mod, [3], [7], 4)


def test_all_edges_identical(pp, oracle_mod):
    run_and_compare(pp, oracle_mod, [9] * 5000, [4] * 5000, 10)


def test_self_loops_only(pp, oracle_mod):
    rng = np.random.default_rng(1)
    x = rng.integers(0, 256, 3000)
    run_and_compare(pp, oracle_mod, x, x, 8)


def test_every_in_degree_one(pp, oracle_mod):
    # a permutation: max(d_in) = 1, so every column is removed and A = 0
    p = np.random.default_rng(2).permutation(1 << 9)
    graphs = run_and_compare(pp, oracle_mod, np.arange(1 << 9), p, 9)
    assert graphs["lowest"][0].info_dict()["nnz"] == 0


def test_tied_maximum(pp, oracle_mod):
    rng = np.random.default_rng(3)
    u = list(rng.integers(0, 1024, 4000))
    v = list(rng.integers(0, 1024, 4000))
    # columns 100, 200 and 300 get exactly the same, largest in-degree
    for col in (300, 100, 200):
        extra = 400 - sum(1 for x in v if x == col)
        u += list(rng.integers(0, 1024, extra))
        v += [col] * extra
    graphs = run_and_compare(pp, oracle_mod, u, v, 10)
    assert graphs["all_ties"][1]["ties"] == 3 and graphs["all_ties"][1]["supernodes"] == 3
    assert graphs["lowest"][1]["supernodes"] == 1 and graphs["lowest"][1]["vmax"] == 100


@pytest.mark.parametrize("scale", [20, 24, 26, 27])
def test_counts_that_overflow_the_packed_field(pp, oracle_mod, scale):
    """Counts >= 2^(32-scale)-1 go to the overflow table; put some in kept columns."""
    rng = np.random.default_rng(scale)
    N = 1 << scale
    cmax = (1 << (32 - scale)) - 1
    heavy = min(cmax + 5, 5000)
    u = list(rng.integers(0, N, 3000))
    v = list(rng.integers(0, N, 3000))
    sup = 11
    u += list(rng.integers(0, N, 4 * heavy + 100))
    v += [sup] * (4 * heavy + 100)               # the supernode column, removed
    for k, (a, b) in enumerate([(5, 12), (6, 12), (N - 1, 13), (0, N - 1)]):
        u += [a] * (heavy + k)
        v += [b] * (heavy + k)
        u += [7, 8]
        v += [b, b]
    perm = rng.permutation(len(u))
    dts = ("fp64", "fp32") if scale < 27 else ("fp32",)
    graphs = run_and_compare(pp, oracle_mod, np.array(u)[perm], np.array(v)[perm], scale, rules=("lowest",),
                             dtypes=dts)
    g, R = graphs["lowest"]
    assert g.info_dict()["novf"] >= 4


def test_long_columns_span_many_tiles(pp, oracle_mod, k0):
    """Columns far longer than a Kernel 3 tile, next to each other and at both ends."""
    scale = 16
    N = 1 << scale
    rng = np.random.default_rng(4)
    bu, bv = k0.edges_host(scale, 9, M=200000)
    u, v = [bu], [bv]
    for col, n in ((77, 90000), (0, 40000), (1, 30000), (N - 1, 45000), (N - 2, 20000), (5000, 60000)):
        u.append(rng.integers(0, N, n).astype(np.uint32))
        v.append(np.full(n, col, dtype=np.uint32))
    run_and_compare(pp, oracle_mod, np.concatenate(u), np.concatenate(v), scale)


def test_out_of_range_id_is_reported(pp):
    import torch

    scale = 6
    u = dev_u32([1, 2, 64, 3])  # 64 >= N
    v = dev_u32([0, 1, 2, 3])
    pp.last_device_error()
    pp.sort_edges(u, v, scale)
    assert pp.last_device_error() & pp.DEV_RANGE
    assert pp.last_device_error() == 0  # the word is cleared once read


@pytest.mark.parametrize("scale,offset", [(20, 1), (20, 3), (12, 2)])
def test_unaligned_edge_arrays(pp, oracle_mod, k0, scale, offset):
    """Kernel 1 reads u and v four ids at a time when both are 16-byte
    aligned and one at a time otherwise: arrays starting 4, 8 or 12 bytes
    past an aligned address sort the same as the oracle; so do the outputs
    written to unaligned places."""
    import torch

    u, v = k0.edges_host(scale, 77)
    ud, vd = dev_u32(u), dev_u32(v)
    bu = torch.empty(len(u) + offset, dtype=torch.int32, device="cuda")
    bv = torch.empty(len(v) + offset, dtype=torch.int32, device="cuda")
    bu[offset:].copy_(ud)
    bv[offset:].copy_(vd)
    ou = torch.empty(len(u) + 1, dtype=torch.int32, device="cuda")
    ov = torch.empty(len(v) + 1, dtype=torch.int32, device="cuda")
    us, vs = pp.sort_edges(bu[offset:], bv[offset:], scale, out=(ou[1:], ov[1:]))
    ous, ovs = oracle_mod.k1_sort(u, v)
    assert np.array_equal(host_u32(us), ous) and np.array_equal(host_u32(vs), ovs)
    assert pp.last_device_error() == 0
