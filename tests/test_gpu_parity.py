"""GPU parity: Kernels 1-3 through the C-ABI against the CPU oracle.

Kernel 1 and Kernel 2 must match bit for bit; Kernel 3 within the stated
tolerances: binary64 L1 error <= 1e-12 ||r||_1; binary32 max relative error
<= 1e-4 per entry and L1 error <= 1e-6 ||r||_1; bfloat16-stored ranks are
reported and only checked loosely (L1 <= 2e-2).
"""
import numpy as np
import pytest

from gpu_helpers import check_row_order, dev_u32, gpu_triples, host_u32, oracle_triples, rank_errors

pytestmark = pytest.mark.gpu

# binary64, binary32 gated as stated; the bfloat16- and binary16-stored vectors reported with a loose bound
TOL = {"fp64": (1e-12, 1e-9), "fp32": (1e-6, 1e-4), "bf16": (2e-2, None), "fp16": (2e-3, None)}

# (scale, M or None for 16 N, seed): several tiles, ragged tails, 32- and 64-bit keys
CASES = [(1, None, 1), (2, None, 2), (4, None, 3), (5, 77, 4), (8, None, 5), (10, None, 1),
         (10, 16 * 1024 - 7, 6), (12, 3 * 4097, 7), (16, None, 8), (17, None, 9), (20, None, 1)]


@pytest.fixture(scope="module")
def pp():
    import torch

    assert torch.cuda.is_available()
    import paper_1603_01876_gb300 as pp

    return pp


def _inputs(k0, scale, M, seed):
    u, v = k0.edges_host(scale, seed, M=M)
    ud, vd = k0.edges_device(scale, seed, M=M)
    assert np.array_equal(host_u32(ud), u) and np.array_equal(host_u32(vd), v), "host/device generators differ"
    return u, v, ud, vd


def check_k2(pp, g, R):
    info = g.info_dict()
    for k in ("nnz0", "nnz", "dmax", "ties", "supernodes"):
        assert info[k] == R[k], k
    assert info["vmax"] == R["vmax"]
    assert np.array_equal(host_u32(g.d_in), R["d_in"])
    assert np.array_equal(host_u32(g.d_out), R["d_out"])
    gu, gv, gc, (cu, cv, colptr) = gpu_triples(g)
    ou, ov, oc = oracle_triples(R)
    assert np.array_equal(gu, ou) and np.array_equal(gv, ov) and np.array_equal(gc, oc)
    # inside each column the rows' vertex ids strictly ascend (the compressed-column layout)
    rows = host_u32(g.iperm)[: g.N][cu]
    same_col = cv[1:] == cv[:-1]
    assert (rows[1:][same_col] > rows[:-1][same_col]).all()
    d = R["d_out"]
    want32 = np.where(d > 0, np.float32(1) / np.maximum(d, 1).astype(np.float32), np.float32(0))
    want64 = np.where(d > 0, 1.0 / np.maximum(d, 1).astype(np.float64), 0.0)
    assert np.array_equal(g.inv_dout32.cpu().numpy(), want32)
    assert np.array_equal(g.inv_dout64.cpu().numpy(), want64)


@pytest.mark.parametrize("scale,M,seed", CASES, ids=["s%d_m%s" % (s, m) for s, m, _ in CASES])
def test_pipeline_parity(pp, k0, oracle_mod, scale, M, seed):
    import torch

    N = 1 << scale
    u, v, ud, vd = _inputs(k0, scale, M, seed)
    # Kernel 1
    us, vs = pp.sort_edges(ud, vd, scale)
    ous, ovs = oracle_mod.k1_sort(u, v)
    assert np.array_equal(host_u32(us), ous) and np.array_equal(host_u32(vs), ovs)
    # Kernel 2, both supernode rules
    r0 = k0.r0_host(N, seed)
    r0d = torch.from_numpy(r0).cuda()
    for rule in ("lowest", "all_ties"):
        g = pp.build_filter_normalize(us, vs, scale, rule)
        R = oracle_mod.k2_filter(ous, ovs, N, rule)
        check_k2(pp, g, R)
        check_row_order(g, ous)
        # Kernel 3
        want = oracle_mod.k3_pagerank(R, r0, 20, 0.85)
        for dt in ("fp64", "fp32", "bf16", "fp16"):
            got = pp.pagerank(g, r0d, 20, 0.85, dt).cpu().numpy()
            e = rank_errors(got, want)
            l1, mr = TOL[dt]
            assert e["l1"] <= l1, (dt, e)
            if mr is not None:
                assert e["max_rel"] <= mr, (dt, e)
    assert pp.last_device_error() == 0


def test_k3_iteration_counts_and_damping(pp, k0, oracle_mod):
    import torch

    scale = 11
    u, v, ud, vd = _inputs(k0, scale, None, 21)
    us, vs = pp.sort_edges(ud, vd, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    R = oracle_mod.k2_filter(u, v, 1 << scale)
    r0 = k0.r0_host(1 << scale, 5)
    r0d = torch.from_numpy(r0).cuda()
    for iters in (0, 1, 2, 7):
        for c in (0.0, 0.5, 0.85, 1.0):
            want = oracle_mod.k3_pagerank(R, r0, iters, c)
            got = pp.pagerank(g, r0d, iters, c, "fp64").cpu().numpy()
            assert rank_errors(got, want)["l1"] <= 1e-12, (iters, c)
    got, l1 = pp.pagerank(g, r0d, 20, 0.85, "fp64", want_l1=True)
    got = got.cpu().numpy()
    assert np.allclose(l1.cpu().numpy(), got / np.abs(got).sum(), rtol=1e-15, atol=0)


def test_determinism(pp, k0):
    import torch

    scale = 16
    _, _, ud, vd = _inputs(k0, scale, None, 31)
    r0d = torch.from_numpy(k0.r0_host(1 << scale, 3)).cuda()
    outs = []
    for _ in range(2):
        us, vs = pp.sort_edges(ud, vd, scale)
        g = pp.build_filter_normalize(us, vs, scale)
        rs = [pp.pagerank(g, r0d, 20, 0.85, dt) for dt in ("fp64", "fp32", "bf16", "fp16")]
        nnz = g.info_dict()["nnz"]
        outs.append([us.clone(), vs.clone(), g.colptr.clone(), g.rowc[:nnz].clone(), g.d_out.clone()] + rs)
    for a, b in zip(*outs):
        assert torch.equal(a, b)


def test_pipeline_host_matches_device_path(pp, k0):
    import torch

    scale = 14
    u, v, ud, vd = _inputs(k0, scale, None, 41)
    r0 = k0.r0_host(1 << scale, 41)
    for dt in ("fp64", "fp32"):
        uh = torch.from_numpy(u.view(np.int32)).pin_memory()
        vh = torch.from_numpy(v.view(np.int32)).pin_memory()
        r0h = torch.from_numpy(r0).pin_memory()
        r, info = pp.pipeline_host(uh, vh, scale, r0h, 20, 0.85, dt)
        torch.cuda.synchronize()
        us, vs = pp.sort_edges(ud, vd, scale)
        g = pp.build_filter_normalize(us, vs, scale)
        want = pp.pagerank(g, torch.from_numpy(r0).cuda(), 20, 0.85, dt).cpu()
        assert torch.equal(r, want)
        assert info.tolist()[:7] == g.info.cpu().tolist()[:7]


@pytest.mark.parametrize("scale,M", [(16, None), (18, None), (18, 16 * (1 << 18) - 3), (20, None)])
def test_pipeline_host_chunked_sort_matches_device_path(pp, k0, scale, M):
    """From 2^20 edges with 64-bit keys the host-buffer pipeline sorts the
    edge list in four chunks as they arrive and merges them: the sorted edges
    (through Kernel 2's output), the scalars and the ranks equal the device
    path's bit for bit, for ragged chunk boundaries too."""
    import torch

    u, v, ud, vd = _inputs(k0, scale, M, 47)
    N = 1 << scale
    r0 = k0.r0_host(N, 47)
    uh = torch.from_numpy(u.view(np.int32)).pin_memory()
    vh = torch.from_numpy(v.view(np.int32)).pin_memory()
    r0h = torch.from_numpy(r0).pin_memory()
    r, info = pp.pipeline_host(uh, vh, scale, r0h, 20, 0.85, "fp32")
    torch.cuda.synchronize()
    us, vs = pp.sort_edges(ud, vd, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    assert torch.equal(r, pp.pagerank(g, torch.from_numpy(r0).cuda(), 20, 0.85, "fp32").cpu())
    assert info.tolist()[:7] == g.info.cpu().tolist()[:7]
    assert pp.last_device_error() == 0


@pytest.mark.parametrize("scale", [16, 18])
def test_pipeline_host_back_to_back_calls_keep_their_start_vectors(pp, k0, scale):
    """Two host-buffer pipelines enqueued back to back on one stream with one
    workspace and different start vectors: the second call's copies (on a
    side stream) must not overtake the first call's kernels."""
    import torch

    u, v, ud, vd = _inputs(k0, scale, None, 43)
    N = 1 << scale
    uh = torch.from_numpy(u.view(np.int32)).pin_memory()
    vh = torch.from_numpy(v.view(np.int32)).pin_memory()
    r0s = [torch.from_numpy(k0.r0_host(N, s)).pin_memory() for s in (5, 6)]
    ws = torch.empty(pp.workspace_bytes("pipeline", len(u), scale, 20, "fp32"), dtype=torch.uint8, device="cuda")
    outs = [pp.pipeline_host(uh, vh, scale, r0, 20, 0.85, "fp32", workspace=ws)[0] for r0 in r0s]
    torch.cuda.synchronize()
    us, vs = pp.sort_edges(ud, vd, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    for r0, got in zip(r0s, outs):
        assert torch.equal(got, pp.pagerank(g, r0.cuda(), 20, 0.85, "fp32").cpu())


# other seeds, scales between the fixed cases, and other edge factors (M = 2N
# .. 64N: sparser graphs with more leaves and empty columns, denser ones with
# more duplicate edges and longer columns)
SWEEP = [(13, None, 101), (15, 5 * (1 << 15) + 3, 102), (16, 2 * (1 << 16), 103), (16, 64 * (1 << 16), 104),
         (18, None, 105), (19, 4 * (1 << 19) - 1, 106), (21, None, 107), (22, None, 108)]


@pytest.mark.parametrize("scale,M,seed", SWEEP, ids=["s%d_m%s_seed%d" % c for c in SWEEP])
def test_sweep_parity(pp, k0, oracle_mod, scale, M, seed):
    import torch

    N = 1 << scale
    u, v, ud, vd = _inputs(k0, scale, M, seed)
    us, vs = pp.sort_edges(ud, vd, scale)
    ous, ovs = oracle_mod.k1_sort(u, v)
    assert np.array_equal(host_u32(us), ous) and np.array_equal(host_u32(vs), ovs)
    del u, v
    g = pp.build_filter_normalize(us, vs, scale)
    R = oracle_mod.k2_filter(ous, ovs, N)
    check_k2(pp, g, R)
    r0 = k0.r0_host(N, seed)
    want = oracle_mod.k3_pagerank(R, r0, 20, 0.85)
    r0d = torch.from_numpy(r0).cuda()
    for dt in ("fp64", "fp32"):
        e = rank_errors(pp.pagerank(g, r0d, 20, 0.85, dt).cpu().numpy(), want)
        l1, mr = TOL[dt]
        assert e["l1"] <= l1 and e["max_rel"] <= mr, (dt, e)
    assert pp.last_device_error() == 0
