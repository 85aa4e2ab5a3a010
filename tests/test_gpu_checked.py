"""The bounds-checked build (libpp_checked.so) beside the plain one (libpp.so).

The checked build compares every index a kernel reads from memory, or
computes from what it read, with the length of the array it addresses; one
out of range sets PP_DEV_BOUNDS in the device error word and the access is
sent to element 0 instead of leaving the array.  It stands in for a memory
checker:

- the whole path (Kernels 1-3 in every precision, the variants, the export,
  the batched calls) runs through both libraries on the same inputs: the
  outputs must be bit-identical and the checked build's error word clear,
  i.e. no index of a correct run ever left its array;
- a graph with one planted bad entry (a storage position naming a vertex
  past N) goes through the checked build only: Kernel 3, plain, variant and
  batched, reports PP_DEV_BOUNDS and the context stays usable (a clean call
  afterwards gives the plain build's bits).  Every use of that array in
  those kernels is index-checked in this build; the plain build is never
  given the bad graph.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GRAPH_FIELDS = ("colptr", "d_in", "d_out", "inv_dout32", "inv_dout64", "perm", "iperm")
CASES = [(10, 1, None), (13, 5, 16 * 8192 - 77), (16, 2, None)]


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp
    from paper_1603_01876_gb300 import tune

    prev = pp.use_library("default")
    knobs = list(tune.SINGLE_KNOBS) + list(tune.BATCH_KNOBS) + ["k3_unroll_f64"]
    values = {k: pp.get_tuning(k) for k in knobs}
    pp.use_library("checked")
    assert pp.build_flags() & pp.BUILD_CHECKED
    for k, v in values.items():  # the same launch configuration in both
        pp.set_tuning(k, v)
    assert pp.last_device_error() == 0
    pp.use_library(prev)
    yield pp
    pp.use_library(prev)


def graph_arrays(g):
    info = g.info_dict()
    out = {f: getattr(g, f).clone() for f in GRAPH_FIELDS}
    out["rowc"] = g.rowc[: info["nnz"]].clone()
    out["ovf_key"] = g.ovf_key[: info["novf"]].clone()
    out["ovf_cnt"] = g.ovf_cnt[: info["novf"]].clone()
    out["info"] = g.info.clone()
    return out


def run_path(pp, k0, scale, seed, M):
    import torch

    N = 1 << scale
    u, v = k0.edges_device(scale, seed, M=M)
    us, vs = pp.sort_edges(u, v, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    g2 = pp.build_filter_normalize(us, vs, scale, "all_ties")
    r0 = torch.from_numpy(k0.r0_host(N, seed)).cuda()
    out = {"us": us, "vs": vs}
    out.update({"A." + k: t for k, t in graph_arrays(g).items()})
    out.update({"A2." + k: t for k, t in graph_arrays(g2).items()})
    for dt in ("fp64", "fp32", "bf16", "fp16"):
        out["r." + dt] = pp.pagerank(g, r0, 20, 0.85, dt)
    for dt in ("fp64", "fp32"):
        r, done, l1 = pp.pagerank_ex(g, r0, 300, 0.85, dt, dangling=True, tol=1e-9, want_l1=True)
        out.update({"rx." + dt: r, "rx_done." + dt: done, "rx_l1." + dt: l1})
    rowptr, col, cnt, v64, v32 = pp.export_csr(g)
    nnz = int(rowptr[-1].item())
    out.update({"csr.rowptr": rowptr, "csr.col": col[:nnz], "csr.cnt": cnt[:nnz], "csr.v64": v64[:nnz],
                "csr.v32": v32[:nnz]})
    torch.cuda.synchronize()
    return out


def run_batched(pp, k0):
    import torch

    scales = [9, 4, 12, 7, 11]
    us, vs = zip(*[k0.edges_device(s, 40, graph=i) for i, s in enumerate(scales)])
    sb = pp.sort_edges_batched(list(us), list(vs), scales)
    gb = pp.build_filter_normalize_batched(sb, scales)
    out = {}
    for i, (a, b) in enumerate(sb):
        out["b.us%d" % i], out["b.vs%d" % i] = a, b
    for i, g in enumerate(gb):
        out.update({"b.A%d.%s" % (i, k): t for k, t in graph_arrays(g).items()})
    rows = sum(1 << s for s in scales)
    for nrhs in (5, 32):
        r0 = torch.rand(rows, nrhs, dtype=torch.float64, device="cuda",
                        generator=torch.Generator("cuda").manual_seed(nrhs)) + 0.5
        out["b.r%d" % nrhs] = pp.pagerank_batched(gb, r0, nrhs, 20)
    torch.cuda.synchronize()
    return out


def same_bits(a, b):
    import torch

    assert a.keys() == b.keys()
    for k in a:
        x, y = a[k], b[k]
        assert x.dtype == y.dtype and x.shape == y.shape, k
        if x.is_floating_point():
            x, y = x.contiguous().view(torch.uint8), y.contiguous().view(torch.uint8)
        assert torch.equal(x, y), k


@pytest.mark.parametrize("scale,seed,M", CASES, ids=["s10", "s13_ragged", "s16"])
def test_checked_build_gives_the_same_bits(pp, k0, scale, seed, M):
    plain = run_path(pp, k0, scale, seed, M)
    assert pp.last_device_error() == 0
    prev = pp.use_library("checked")
    try:
        checked = run_path(pp, k0, scale, seed, M)
        assert pp.last_device_error() == 0, "an index left its array"
    finally:
        pp.use_library(prev)
    same_bits(plain, checked)


def test_checked_build_gives_the_same_bits_batched(pp, k0):
    plain = run_batched(pp, k0)
    assert pp.last_device_error() == 0
    prev = pp.use_library("checked")
    try:
        checked = run_batched(pp, k0)
        assert pp.last_device_error() == 0, "an index left its array"
    finally:
        pp.use_library(prev)
    same_bits(plain, checked)


def test_checked_build_reports_a_bad_index(pp, k0):
    import torch

    scale, seed = 12, 3
    N = 1 << scale
    u, v = k0.edges_device(scale, seed)
    us, vs = pp.sort_edges(u, v, scale)
    g = pp.build_filter_normalize(us, vs, scale)
    r0 = torch.from_numpy(k0.r0_host(N, seed)).cuda()
    want = pp.pagerank(g, r0, 20, 0.85, "fp32")
    assert pp.last_device_error() == 0
    bad = pp.Graph(g.M, scale, r0.device)
    for f in GRAPH_FIELDS + ("rowc", "ovf_key", "ovf_cnt", "info"):
        getattr(bad, f).copy_(getattr(g, f))
    bad.iperm[5] = N + 3  # position 5 names a vertex past the last one
    other = pp.build_filter_normalize(*pp.sort_edges(*k0.edges_device(9, 4), 9), 9)
    torch.cuda.synchronize()
    prev = pp.use_library("checked")
    try:
        for dt in ("fp64", "fp32", "bf16", "fp16"):
            pp.pagerank(bad, r0, 20, 0.85, dt)
            assert pp.last_device_error() & pp.DEV_BOUNDS, dt
        pp.pagerank_ex(bad, r0, 50, 0.85, "fp32", dangling=True, tol=1e-7)
        assert pp.last_device_error() & pp.DEV_BOUNDS
        rows = N + (1 << 9)
        for nrhs in (3, 32):
            pp.pagerank_batched([bad, other], torch.ones(rows, nrhs, dtype=torch.float64, device="cuda"), nrhs, 5)
            assert pp.last_device_error() & pp.DEV_BOUNDS, nrhs
        # the context is intact: a clean call gives the plain build's bits
        got = pp.pagerank(g, r0, 20, 0.85, "fp32")
        assert pp.last_device_error() == 0
    finally:
        pp.use_library(prev)
    assert torch.equal(got.view(torch.int32), want.view(torch.int32))
    assert np.isfinite(got.cpu().numpy()).all()
