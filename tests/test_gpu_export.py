"""Kernel 2's filtered A exported as compressed rows in vertex order
(pp_export_csr), against the oracle's rows (Sec. IV-C step 4).

Row pointers, columns and counts must equal the oracle's bit for bit; the
binary64 values are cnt / d_out(u) by IEEE division, as the oracle computes
them, so they must be identical too; the binary32 values are the binary32
quotient of the same (exactly converted) operands.
"""
import numpy as np
import pytest

from gpu_helpers import dev_u32, host_u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp

    return pp


def check_export(pp, g, R):
    rowptr, col, cnt, v64, v32 = pp.export_csr(g)
    assert pp.last_device_error() == 0
    nnz = R["nnz"]
    rp = rowptr.cpu().numpy()
    np.testing.assert_array_equal(rp, R["rowptr"].astype(np.int64))
    assert rp[-1] == nnz == g.info_dict()["nnz"]
    np.testing.assert_array_equal(host_u32(col)[:nnz], R["col"])
    np.testing.assert_array_equal(host_u32(cnt)[:nnz], R["cnt"])
    np.testing.assert_array_equal(v64.cpu().numpy()[:nnz].view(np.uint64), R["val"].view(np.uint64))
    u = np.repeat(np.arange(R["N"]), np.diff(R["rowptr"].astype(np.int64)))
    want32 = R["cnt"].astype(np.float32) / R["d_out"][u].astype(np.float32)
    np.testing.assert_array_equal(v32.cpu().numpy()[:nnz].view(np.uint32), want32.view(np.uint32))


def build(pp, oracle_mod, u, v, scale, rule):
    u = np.asarray(u, dtype=np.uint32)
    v = np.asarray(v, dtype=np.uint32)
    us, vs = pp.sort_edges(dev_u32(u), dev_u32(v), scale)
    g = pp.build_filter_normalize(us, vs, scale, rule)
    ous, ovs = oracle_mod.k1_sort(u, v)
    return g, oracle_mod.k2_filter(ous, ovs, 1 << scale, rule)


@pytest.mark.parametrize("scale,M", [(1, None), (4, 37), (10, None), (13, 100003), (16, None), (20, None)])
@pytest.mark.parametrize("rule", ["lowest", "all_ties"])
def test_export_kronecker(pp, oracle_mod, k0, scale, M, rule):
    u, v = k0.edges_host(scale, 30 + scale, M=M)
    g, R = build(pp, oracle_mod, u, v, scale, rule)
    check_export(pp, g, R)


def test_export_empty_matrix(pp, oracle_mod):
    # a permutation: every in-degree is 1, every column is removed
    p = np.random.default_rng(5).permutation(1 << 9)
    g, R = build(pp, oracle_mod, np.arange(1 << 9), p, 9, "lowest")
    assert R["nnz"] == 0
    check_export(pp, g, R)


@pytest.mark.parametrize("scale", [20, 24])
def test_export_counts_beyond_the_packed_field(pp, oracle_mod, scale):
    rng = np.random.default_rng(scale + 100)
    N = 1 << scale
    heavy = (1 << (32 - scale)) + 3
    u = list(rng.integers(0, N, 5000))
    v = list(rng.integers(0, N, 5000))
    u += list(rng.integers(0, N, 3 * heavy))
    v += [17] * (3 * heavy)  # the supernode
    for a, b in ((2, 9), (N - 1, 9), (3, N - 1)):
        u += [a] * heavy + [(a + 1) % N]
        v += [b] * heavy + [b]
    g, R = build(pp, oracle_mod, u, v, scale, "lowest")
    assert g.info_dict()["novf"] >= 3
    check_export(pp, g, R)


def test_export_too_small_output_is_reported(pp, oracle_mod, k0):
    import torch

    scale = 10
    u, v = k0.edges_host(scale, 3)
    g, R = build(pp, oracle_mod, u, v, scale, "lowest")
    nnz = R["nnz"]
    pp.last_device_error()
    rowptr, col, cnt, _, _ = pp.export_csr(g, cap=nnz - 1, values=False)
    assert pp.last_device_error() & pp.DEV_CAPACITY
    np.testing.assert_array_equal(rowptr.cpu().numpy(), R["rowptr"].astype(np.int64))
    rowptr, col, cnt, _, _ = pp.export_csr(g, cap=nnz, values=False)
    assert pp.last_device_error() == 0
    np.testing.assert_array_equal(host_u32(col)[:nnz], R["col"])
