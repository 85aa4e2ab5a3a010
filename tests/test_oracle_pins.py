"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import pins


@pytest.fixture(scope="module")
def O():
    import oracle

    return oracle.default()


@pytest.mark.parametrize("name,check", pins.ALL_CHECKS, ids=[n for n, _ in pins.ALL_CHECKS])
def test_pin(O, name, check):
    check(O)


@pytest.fixture(scope="module")
def kron12(k0):
    return k0.edges_host(12, seed=5)


def test_k1_properties_kronecker(O, kron12):
    u, v = kron12
    pins.check_k1_properties(O, u, v)


def test_k1_edge_cases(O):
    for u, v in [([], []), ([3], [1]), ([2] * 50, [7] * 50), ([5, 5, 5, 1], [9, 3, 3, 0])]:
        pins.check_k1_properties(O, np.array(u, dtype=np.uint32), np.array(v, dtype=np.uint32))


def test_k2_invariants_kronecker(O, kron12):
    u, v = kron12
    pins.check_k2_invariants(O, u, v, 1 << 12)


def test_k2_no_edges(O):
    R = O.k2_filter(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 8, "lowest")
    assert R["nnz0"] == 0 and R["nnz"] == 0 and R["dmax"] == 0 and (R["d_in"] == 0).all()
    r = O.k3_pagerank(R, np.ones(8), 3, 0.85)
    assert np.allclose(r, 0.15 ** 3 / 8, rtol=1e-14, atol=0)


def test_k2_rejects_out_of_range(O):
    with pytest.raises(ValueError):
        O.k2_filter(np.array([0, 9], np.uint32), np.array([1, 1], np.uint32), 8)


def test_k3_mass_balance_kronecker(O, kron12):
    u, v = kron12
    pins.check_k3_mass_balance(O, u, v, 1 << 12)


def test_k3_sums_output(O, kron12):
    """The oracle's reported sum(r) per iteration is the sum of the vector it iterates."""
    u, v = kron12
    R = O.k2_filter(u, v, 1 << 12)
    r0 = np.random.default_rng(1).random(1 << 12)
    r, sums = O.k3_pagerank(R, r0, 4, 0.85, want_sums=True)
    assert abs(sums[0] - 1.0) < 1e-15
    assert abs(sums[4] - r.sum()) < 1e-14


def test_fullsize_script_matches_direct_oracle_calls(tmp_path, k0):
    """oracle/fullsize.py stores what the oracle itself returns (no other arithmetic)."""
    import hashlib

    import oracle
    from oracle import fullsize

    scale, seed = 12, 3
    path = fullsize.compute(scale, seed, out=str(tmp_path / "o.npz"))
    d = fullsize.load(path)
    u, v = k0.edges_host(scale, seed)
    us, vs = oracle.k1_sort(u, v)
    A = oracle.k2_filter(us, vs, 1 << scale)
    r = oracle.k3_pagerank(A, k0.r0_host(1 << scale, seed), 20, 0.85)
    sha = lambda a: hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()
    assert d["us_sha"] == sha(us) and d["vs_sha"] == sha(vs)
    assert d["col_sha"] == sha(A["col"]) and d["cnt_sha"] == sha(A["cnt"]) and d["val_sha"] == sha(A["val"])
    assert (d["nnz0"], d["nnz"], d["dmax"], d["vmax"]) == (A["nnz0"], A["nnz"], A["dmax"], A["vmax"])
    np.testing.assert_array_equal(d["d_in"], A["d_in"])
    np.testing.assert_array_equal(d["rowptr"], A["rowptr"])
    np.testing.assert_array_equal(d["r"], r)
