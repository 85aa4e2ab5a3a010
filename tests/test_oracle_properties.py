"""Property-based pins of the CPU oracle (no GPU): random small graphs drawn by
hypothesis, each kernel compared with a reference that is slow and obviously
right (Python's sorted, the dense Matlab statements of Sec. IV-C, the dense
Google matrix of Sec. IV-D).  The seeded pins in pins.py fix the cases;
these search around them.  hypothesis is a CPU-side test dependency only."""
import numpy as np
import pytest

import pins

hypothesis = pytest.importorskip("hypothesis")
st = hypothesis.strategies
given, settings = hypothesis.given, hypothesis.settings

SETTINGS = settings(max_examples=60, deadline=None, derandomize=True)


@pytest.fixture(scope="module")
def O():
    import oracle

    return oracle.default()


@st.composite
def edge_lists(draw, max_n=64, max_m=400):
    N = draw(st.integers(1, max_n))
    M = draw(st.integers(0, max_m))
    seed = draw(st.integers(0, 2**31))
    hub = draw(st.sampled_from([0.0, 0.3, 0.9]))
    u, v = pins.random_edges(N, M, seed, hub_bias=hub)
    return N, u, v


@SETTINGS
@given(data=st.data())
def test_k1_is_pythons_sort(O, data):
    M = data.draw(st.integers(0, 300))
    big = data.draw(st.booleans())
    hi = 2**32 - 1 if big else 7
    u = np.array(data.draw(st.lists(st.integers(0, hi), min_size=M, max_size=M)), dtype=np.uint32)
    v = np.array(data.draw(st.lists(st.integers(0, hi), min_size=M, max_size=M)), dtype=np.uint32)
    us, vs = O.k1_sort(u, v)
    assert list(zip(us.tolist(), vs.tolist())) == sorted(zip(u.tolist(), v.tolist()))


@SETTINGS
@given(g=edge_lists(), rule=st.sampled_from(["lowest", "all_ties"]))
def test_k2_is_the_dense_statements(O, g, rule):
    N, u, v = g
    R = O.k2_filter(u, v, N, rule)
    A, d_in, d_out = pins.dense_kernel2(u, v, N, rule)
    assert np.array_equal(R["d_in"].astype(np.float64), d_in)
    assert np.array_equal(R["d_out"].astype(np.float64), d_out)
    assert np.array_equal(pins.csr_to_dense(R), A)
    assert R["nnz"] == int((A != 0).sum())
    assert R["nnz0"] == len(set(zip(u.tolist(), v.tolist())))


@SETTINGS
@given(g=edge_lists(), c=st.sampled_from([0.0, 0.15, 0.5, 0.85, 1.0]), iters=st.integers(0, 25),
       rseed=st.integers(0, 2**31))
def test_k3_is_the_dense_google_iteration(O, g, c, iters, rseed):
    N, u, v = g
    R = O.k2_filter(u, v, N, "lowest")
    A, _, _ = pins.dense_kernel2(u, v, N, "lowest")
    r0 = np.random.default_rng(rseed).random(N) + 0.01
    got = O.k3_pagerank(R, r0, iters, c)
    want, _ = pins.google_power_iteration(A, r0, iters, c)
    assert np.abs(got - want).sum() <= 1e-13 * np.abs(want).sum()


@SETTINGS
@given(g=edge_lists(max_m=200), c=st.sampled_from([0.5, 0.85, 1.0]), iters=st.integers(0, 25),
       rseed=st.integers(0, 2**31))
def test_k3_dangling_is_the_stochastic_matrix(O, g, c, iters, rseed):
    N, u, v = g
    R = O.k2_filter(u, v, N, "lowest")
    A, _, _ = pins.dense_kernel2(u, v, N, "lowest")
    r0 = np.random.default_rng(rseed).random(N) + 0.01
    G = pins.google_dangling_matrix(A, c)
    want = r0 / np.abs(r0).sum()
    for _ in range(iters):
        want = G @ want
    got, done = O.k3_pagerank_ex(R, r0, iters, c, dangling=True)
    assert done == iters
    assert np.abs(got - want).sum() <= 1e-13 * np.abs(want).sum()
    assert abs(got.sum() - 1.0) <= 1e-13
