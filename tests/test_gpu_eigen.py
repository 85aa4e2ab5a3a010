"""The eigenvector validation of Sec. IV-D, at scale 20.

The paper checks Kernel 3 by comparing r / norm(r,1) with the first
eigenvector of the Google matrix G = c*A^T + (1-c)/N (every entry of the
second term equal).  G is positive, so by Perron-Frobenius that eigenvector
is unique and positive.  Here the GPU's iteration is run to convergence and
its ranks are checked against G built on the host from the oracle's own
Kernel 2 matrix of the same graph (one sparse product, no GPU arithmetic):

- the plain iteration (mass leaks through the rows without entries, so each
  call restarts from r / norm(r,1), which the iteration does anyway): the
  normalised limit x satisfies G x = lambda x with lambda = sum(G x);
- the dangling-node variant (G made column-stochastic, lambda = 1): the
  converged ranks are a fixed point, and equal the oracle's converged vector,
  which stops at the same iteration.

After 20 iterations only the first (|lambda_2|/lambda_1)^20 of the error is
gone, so both checks use converged runs."""
import numpy as np
import pytest

from gpu_helpers import host_u32

pytestmark = pytest.mark.gpu

SCALE, SEED, C = 20, 2, 0.85


@pytest.fixture(scope="module")
def graph(k0, oracle_mod):
    import scipy.sparse as sp
    import torch

    import paper_1603_01876_gb300 as pp

    N = 1 << SCALE
    u, v = k0.edges_device(SCALE, SEED)
    us, vs = pp.sort_edges(u, v, SCALE)
    g = pp.build_filter_normalize(us, vs, SCALE)
    R = oracle_mod.k2_filter(host_u32(us), host_u32(vs), N)
    assert (R["d_out"] == 0).sum() > 0, "the graph must have rows without entries"
    At = sp.csr_matrix((R["val"], R["col"].astype(np.int64), R["rowptr"].astype(np.int64)), shape=(N, N)).T.tocsr()
    r0 = k0.r0_host(N, SEED)
    return pp, g, R, At, r0, torch.from_numpy(r0).cuda()


def _google(At, x, dangling_rows=None):
    """G x on the host, in binary64: c*A^T x + (1-c)/N * sum(x), plus
    c/N * (mass on the rows without entries) for the stochastic form."""
    N = len(x)
    y = C * (At @ x) + (1 - C) / N * x.sum()
    if dangling_rows is not None:
        y += C / N * x[dangling_rows].sum()
    return y


def test_plain_iteration_converges_to_the_perron_vector(graph):
    pp, g, R, At, r0, r0d = graph
    x = r0d
    prev = None
    for rounds in range(200):
        x = pp.pagerank(g, x, 50, C, "fp64")
        x = x / x.sum()
        if prev is not None and float((x - prev).abs().sum()) < 1e-13:
            break
        prev = x
    else:
        pytest.fail("no convergence in 10000 iterations")
    assert pp.last_device_error() == 0
    xh = x.cpu().numpy()
    assert (xh > 0).all()  # the Perron vector is positive
    y = _google(At, xh)
    lam = y.sum()
    assert 1 - C <= lam < 1.0, lam  # lambda = 1 - c * (mass on the rows without entries)
    assert np.abs(y / lam - xh).sum() <= 1e-11
    # one GPU step of the normalised vector is G x
    y_gpu = pp.pagerank(g, x, 1, C, "fp64").cpu().numpy()
    assert np.abs(y_gpu - y).sum() <= 1e-13


def test_dangling_variant_converges_to_the_stationary_vector(graph, oracle_mod):
    pp, g, R, At, r0, r0d = graph
    tol = 1e-12
    r, done = pp.pagerank_ex(g, r0d, 2000, C, "fp64", dangling=True, tol=tol)
    k = int(done.item())
    assert 20 < k < 2000
    rh = r.cpu().numpy()
    assert abs(rh.sum() - 1.0) <= 1e-12 and (rh > 0).all()
    # a fixed point of the stochastic G: r_k = G r_(k-1), so
    # norm(G r_k - r_k, 1) <= c * norm(r_k - r_(k-1), 1) < c * tol
    dangling_rows = np.flatnonzero(R["rowptr"][1:] == R["rowptr"][:-1])
    y = _google(At, rh, dangling_rows)
    assert np.abs(y - rh).sum() <= C * tol + 1e-14
    # the oracle's converged vector: same stopping iteration, same ranks
    want, wk = oracle_mod.k3_pagerank_ex(R, r0, 2000, C, dangling=True, tol=tol)
    assert wk == k
    assert np.abs(rh - want).sum() <= 1e-12
    # binary32 stops at its own tolerance within c/(1-c) * tol of the same
    # vector, plus its rounding (about 1e-6 in L1)
    r32, _ = pp.pagerank_ex(g, r0d, 2000, C, "fp32", dangling=True, tol=1e-6)
    assert np.abs(r32.cpu().numpy().astype(np.float64) - want).sum() <= C / (1 - C) * 1e-6 + 2e-6
    assert pp.last_device_error() == 0
