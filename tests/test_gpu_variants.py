"""Kernel 3 variants (pp_pagerank_ex) against the oracle: the dangling-node
term, the convergence test, both together, and flags = 0 against the plain
iteration.  Tolerances as for the plain path (binary64 L1 <= 1e-12; binary32
L1 <= 1e-6, max relative <= 1e-4), the binary32 ones scaled by k/20 when a
run takes k > 20 iterations (rounding accumulates about linearly); the
stopping iteration must be the oracle's exactly in binary64."""
import numpy as np
import pytest

from gpu_helpers import host_u32, rank_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-12, 1e-9), "fp32": (1e-6, 1e-4)}


@pytest.fixture(scope="module", params=[(10, 3), (16, 7)], ids=["s10", "s16"])
def case(request, k0, oracle_mod):
    import torch

    import paper_1603_01876_gb300 as pp

    scale, seed = request.param
    N = 1 << scale
    u, v = k0.edges_device(scale, seed)
    us, vs = pp.sort_edges(u, v, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    R = oracle_mod.k2_filter(host_u32(us), host_u32(vs), N)
    assert (R["d_out"] == 0).sum() > 0, "the case must have dangling rows"
    r0 = k0.r0_host(N, seed)
    return pp, g, R, r0, torch.from_numpy(r0).cuda()


@pytest.mark.parametrize("dtype", ["fp64", "fp32"])
@pytest.mark.parametrize("dangling,tol,iters", [(True, 0.0, 20), (False, 1e-7, 200), (True, 1e-9, 200),
                                                (True, 1e-3, 200), (False, 0.0, 20)])
def test_variant_vs_oracle(case, oracle_mod, dtype, dangling, tol, iters):
    pp, g, R, r0, r0d = case
    want, want_iters = oracle_mod.k3_pagerank_ex(R, r0, iters, 0.85, dangling=dangling, tol=tol)
    got, done = pp.pagerank_ex(g, r0d, iters, 0.85, dtype, dangling=dangling, tol=tol)
    got = got.cpu().numpy()
    assert pp.last_device_error() == 0
    if dtype == "fp64" or tol == 0.0:
        # binary32 may cross a tolerance one iteration apart from binary64
        assert int(done.item()) == want_iters
    e = rank_errors(got, want)
    l1, mr = TOL[dtype]
    if dtype == "fp32":
        grow = max(1.0, want_iters / 20.0)
        l1, mr = l1 * grow, mr * grow
    if int(done.item()) == want_iters:
        assert e["l1"] <= l1 and e["max_rel"] <= mr, e
    if dangling:
        assert abs(got.astype(np.float64).sum() - 1.0) <= (1e-12 if dtype == "fp64" else 1e-5)


def test_flags_zero_matches_plain_path(case):
    pp, g, R, r0, r0d = case
    for dtype in ("fp64", "fp32"):
        a = pp.pagerank(g, r0d, 20, 0.85, dtype).cpu().numpy()
        b, done = pp.pagerank_ex(g, r0d, 20, 0.85, dtype)
        assert int(done.item()) == 20
        e = rank_errors(b.cpu().numpy(), a)
        assert e["l1"] <= (1e-15 if dtype == "fp64" else 1e-7), (dtype, e)


def test_variant_deterministic_and_l1(case):
    pp, g, R, r0, r0d = case
    a, da, l1 = pp.pagerank_ex(g, r0d, 100, 0.85, "fp32", dangling=True, tol=1e-6, want_l1=True)
    b, db = pp.pagerank_ex(g, r0d, 100, 0.85, "fp32", dangling=True, tol=1e-6)
    import torch

    assert torch.equal(a, b) and int(da.item()) == int(db.item())
    a = a.cpu().numpy().astype(np.float64)
    assert np.allclose(l1.cpu().numpy(), a / np.abs(a).sum(), rtol=1e-15, atol=0)


def test_variant_argument_errors(case):
    pp, g, R, r0, r0d = case
    import ctypes

    L = pp.lib()
    out = r0d.clone()
    ws = pp._workspace(pp.workspace_bytes("pagerank_ex", g.M, g.scale, 20, "fp64"), r0d.device)
    call = lambda flags, tol: L.pp_pagerank_ex(ctypes.byref(g.c), pp._ptr(r0d), 20, 0.85, 0, flags, tol, pp._ptr(out),
                                               None, None, pp._ptr(ws), ws.numel(), None)
    assert call(4, 0.0) == pp.PP_ERR_INVALID_ARG      # unknown flag
    assert call(2, 0.0) == pp.PP_ERR_INVALID_ARG      # convergence test without a tolerance
    assert call(2, -1.0) == pp.PP_ERR_INVALID_ARG
