"""Independent checks ("pins") of the CPU oracle, reusable on any build of it.

Every check takes an ``oracle.Oracle`` instance and raises AssertionError when
the oracle disagrees with something the paper or the mathematics fixes.  The
pin tests run them on the oracle as built; the mutation tests run them on
copies of the oracle with a planted mistake and require that one of them fails.

Nothing here calls the GPU path, and nothing here restates the oracle's code:
each check uses a different formulation (brute force, dense matrices, closed
forms, hand-counted fixtures, conservation laws).
"""
import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _frac(s):
    return float(Fraction(s))


def random_edges(N, M, seed, hub_bias=0.0):
    """Small seeded edge lists with many duplicates (values kept small on purpose)."""
    rng = np.random.default_rng(seed)
    u = rng.integers(0, N, size=M).astype(np.uint32)
    v = rng.integers(0, N, size=M).astype(np.uint32)
    if hub_bias > 0:
        hub = rng.random(M) < hub_bias
        v[hub] = rng.integers(0, max(1, N // 8), size=int(hub.sum())).astype(np.uint32)
    return u, v


# ---------------------------------------------------------------- Kernel 1


def brute_force_sort(u, v):
    """Selection sort on (u, v) pairs in pure Python: slow and obviously right."""
    pairs = list(zip((int(x) for x in u), (int(x) for x in v)))
    out = []
    while pairs:
        k = min(range(len(pairs)), key=lambda i: pairs[i])
        out.append(pairs.pop(k))
    return out


def check_k1_brute_force(O, seed=0):
    for N, M in ((1, 1), (4, 17), (16, 120), (64, 200)):
        u, v = random_edges(N, M, seed + M)
        us, vs = O.k1_sort(u, v)
        assert list(zip(us.tolist(), vs.tolist())) == brute_force_sort(u, v)


def check_k1_properties(O, u, v):
    """u nondecreasing (Sec. IV-B), v nondecreasing within equal u, same multiset."""
    us, vs = O.k1_sort(u, v)
    assert len(us) == len(u)
    if len(u) == 0:
        return
    du = np.diff(us.astype(np.int64))
    assert (du >= 0).all()
    same = du == 0
    assert (np.diff(vs.astype(np.int64))[same] >= 0).all()
    a = np.sort((u.astype(np.uint64) << np.uint64(32)) | v.astype(np.uint64))
    b = (us.astype(np.uint64) << np.uint64(32)) | vs.astype(np.uint64)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------- Kernel 2


def dense_kernel2(u, v, N, rule):
    """Kernel 2's Matlab statements executed on a dense N x N float64 array."""
    A = np.zeros((N, N))
    np.add.at(A, (u.astype(np.int64), v.astype(np.int64)), 1.0)
    d_in = A.sum(axis=0)
    if rule == "all_ties":
        A[:, d_in == d_in.max()] = 0
    else:
        A[:, int(np.flatnonzero(d_in == d_in.max())[0])] = 0
    A[:, d_in == 1] = 0
    d_out = A.sum(axis=1)
    i = d_out > 0
    A[i, :] = A[i, :] / d_out[i][:, None]
    return A, d_in, d_out


def csr_to_dense(R):
    N = R["N"]
    D = np.zeros((N, N))
    rowptr = R["rowptr"].astype(np.int64)
    for r in range(N):
        for e in range(rowptr[r], rowptr[r + 1]):
            D[r, R["col"][e]] = R["val"][e]
    return D


def check_k2_dense(O, seed=0):
    cases = [(2, 5), (8, 40), (32, 150), (100, 900), (128, 3000)]
    for k, (N, M) in enumerate(cases):
        for rule in ("lowest", "all_ties"):
            u, v = random_edges(N, M, seed + 7 * k, hub_bias=0.3 if k % 2 else 0.0)
            R = O.k2_filter(u, v, N, rule)
            A, d_in, d_out = dense_kernel2(u, v, N, rule)
            assert np.array_equal(R["d_in"].astype(np.float64), d_in)
            assert np.array_equal(R["d_out"].astype(np.float64), d_out)
            assert np.array_equal(csr_to_dense(R), A)
            assert R["nnz"] == int((A != 0).sum())


def check_k2_golden(O):
    g = load_golden("k1_k2_k3_small_graph.json")
    e = np.array(g["edges"], dtype=np.uint32)
    N = 1 << g["scale"]
    us, vs = O.k1_sort(e[:, 0], e[:, 1])
    assert [[a, b] for a, b in zip(us.tolist(), vs.tolist())] == g["k1_sorted"]
    R = O.k2_filter(e[:, 0], e[:, 1], N, g["rule"])
    assert R["nnz0"] == g["nnz0"]
    assert R["d_in"].tolist() == g["d_in"]
    assert R["dmax"] == g["dmax"] and R["ties"] == g["ties"]
    assert R["d_out"].tolist() == g["d_out"]
    kept = []
    for r in range(N):
        for x in range(int(R["rowptr"][r]), int(R["rowptr"][r + 1])):
            kept.append([r, int(R["col"][x]), int(R["cnt"][x])])
            want = [t for t in g["val"] if t[0] == r and t[1] == int(R["col"][x])]
            assert len(want) == 1 and R["val"][x] == _frac(want[0][2])
    assert kept == g["kept"]

    t = load_golden("k2_supernode_ties.json")
    e = np.array(t["edges"], dtype=np.uint32)
    for rule, want in t["cases"].items():
        R = O.k2_filter(e[:, 0], e[:, 1], 1 << t["scale"], rule)
        assert R["d_in"].tolist() == t["d_in"] and R["dmax"] == t["dmax"] and R["ties"] == t["ties"]
        got = []
        for r in range(1 << t["scale"]):
            for x in range(int(R["rowptr"][r]), int(R["rowptr"][r + 1])):
                got.append([r, int(R["col"][x]), int(R["cnt"][x])])
        assert got == want["kept"] and R["d_out"].tolist() == want["d_out"]

    z = load_golden("k2_all_columns_removed.json")
    e = np.array(z["edges"], dtype=np.uint32)
    for rule in ("lowest", "all_ties"):
        R = O.k2_filter(e[:, 0], e[:, 1], 1 << z["scale"], rule)
        assert R["nnz"] == 0 and R["d_out"].tolist() == z["d_out"] and R["dmax"] == z["dmax"]


def check_k2_invariants(O, u, v, N):
    """Sec. IV-C: entries of A sum to M, nnz(A) <= M, normalised rows sum to 1,
    and no kept column has in-degree 1 or the maximum."""
    R = O.k2_filter(u, v, N, "lowest")
    M = len(u)
    assert int(R["d_in"].astype(np.int64).sum()) == M
    assert R["nnz"] <= R["nnz0"] <= M
    rowptr = R["rowptr"].astype(np.int64)
    rows = np.repeat(np.arange(N), np.diff(rowptr))
    rs = np.bincount(rows, weights=R["val"], minlength=N)
    nz = R["d_out"] > 0
    assert np.allclose(rs[nz], 1.0, rtol=0, atol=1e-12)
    assert (rs[~nz] == 0).all()
    kin = R["d_in"][R["col"]]
    assert (kin != 1).all()
    assert not ((kin == R["dmax"]) & (R["col"] == R["vmax"])).any()
    cs = np.bincount(rows, weights=R["cnt"].astype(np.float64), minlength=N)
    assert np.array_equal(cs, R["d_out"].astype(np.float64))


# ---------------------------------------------------------------- Kernel 3


def google_power_iteration(A, r0, iters, c):
    """Dense Google matrix G = c A' + (1-c)/N (Sec. IV-D validation form):
    the column vector r_k' evolves as r_{k+1}' = G r_k'."""
    N = A.shape[0]
    G = c * A.T + (1.0 - c) / N * np.ones((N, N))
    r = r0 / np.abs(r0).sum()
    for _ in range(iters):
        r = G @ r
    return r, G


def check_k3_dense(O, seed=0):
    for k, (N, M) in enumerate([(4, 12), (16, 80), (64, 500), (128, 1500)]):
        u, v = random_edges(N, M, seed + 11 * k, hub_bias=0.2)
        R = O.k2_filter(u, v, N, "lowest")
        A, _, _ = dense_kernel2(u, v, N, "lowest")
        r0 = np.random.default_rng(seed + k).random(N) + 0.01
        for c in (0.85, 0.5):
            got = O.k3_pagerank(R, r0, 20, c)
            want, _ = google_power_iteration(A, r0, 20, c)
            assert np.abs(got - want).sum() <= 1e-13 * np.abs(want).sum()


def check_k3_eigenvector(O, seed=0):
    """Sec. IV-D validation: r/norm(r,1) equals the normalised Perron vector of
    c A' + (1-c)/N once the iteration has converged."""
    for k, (N, M) in enumerate([(8, 40), (48, 400)]):
        u, v = random_edges(N, M, seed + 3 * k, hub_bias=0.3)
        R = O.k2_filter(u, v, N, "lowest")
        A, _, _ = dense_kernel2(u, v, N, "lowest")
        c = 0.85
        G = c * A.T + (1.0 - c) / N * np.ones((N, N))
        w, V = np.linalg.eig(G)
        p = np.real(V[:, int(np.argmax(np.abs(w)))])
        p = p / p.sum()
        r0 = np.random.default_rng(seed + 5 * k).random(N) + 0.01
        r = O.k3_pagerank(R, r0, 200, c)
        r = r / np.abs(r).sum()
        assert np.abs(r - p).sum() <= 1e-10


def check_k3_closed_forms(O):
    # A = 0 (every column is a leaf): r_k = (1-c)^k / N.
    z = load_golden("k2_all_columns_removed.json")
    e = np.array(z["edges"], dtype=np.uint32)
    N = 1 << z["scale"]
    R = O.k2_filter(e[:, 0], e[:, 1], N, "lowest")
    r0 = np.array([0.3, 0.1, 0.4, 0.2])
    for k in (1, 2, 20):
        r = O.k3_pagerank(R, r0, k, 0.85)
        assert np.allclose(r, 0.15 ** k / N, rtol=1e-13, atol=0)
    # c = 0 (appendix, uniform random walk): one step gives sum(r)/N = 1/N.
    g = load_golden("k1_k2_k3_small_graph.json")
    e = np.array(g["edges"], dtype=np.uint32)
    N = 1 << g["scale"]
    R = O.k2_filter(e[:, 0], e[:, 1], N, "lowest")
    r = O.k3_pagerank(R, np.arange(1.0, N + 1.0), 1, 0.0)
    assert np.allclose(r, 1.0 / N, rtol=1e-15, atol=0)
    # zero iterations: r0 / norm(r0, 1)
    r0 = np.arange(1.0, N + 1.0)
    assert np.allclose(O.k3_pagerank(R, r0, 0, 0.85), r0 / r0.sum(), rtol=1e-15, atol=0)


def check_k3_golden(O):
    g = load_golden("k1_k2_k3_small_graph.json")
    e = np.array(g["edges"], dtype=np.uint32)
    N = 1 << g["scale"]
    R = O.k2_filter(e[:, 0], e[:, 1], N, g["rule"])
    c = _frac(g["k3_c"])
    r0 = np.array(g["k3_r0"], dtype=np.float64)
    r1 = O.k3_pagerank(R, r0, 1, c)
    r2 = O.k3_pagerank(R, r0, 2, c)
    assert r1.tolist() == [_frac(x) for x in g["k3_r1"]]
    assert r2.tolist() == [_frac(x) for x in g["k3_r2"]]


def check_k3_mass_balance(O, u, v, N, seed=0, iters=6, c=0.85):
    """Summing the update over v: sum(r') = c * sum of r(u) over rows with
    d_out(u) > 0 + (1-c) * sum(r), since every such row of A sums to 1."""
    R = O.k2_filter(u, v, N, "lowest")
    r0 = np.random.default_rng(seed).random(N) + 0.01
    live = R["d_out"] > 0
    prev = r0 / np.abs(r0).sum()
    for k in range(1, iters + 1):
        r = O.k3_pagerank(R, r0, k, c)
        want = c * prev[live].sum() + (1 - c) * prev.sum()
        assert abs(r.sum() - want) <= 1e-13 * want
        prev = r


def google_dangling_matrix(A, c):
    """Dense Google matrix with the dangling rows made uniform before damping:
    G = c (A + d 1'/N)' + (1-c)/N, d the indicator of rows without entries.
    Every column of G sums to 1 (a stochastic matrix)."""
    N = A.shape[0]
    S = A.copy()
    S[A.sum(axis=1) == 0, :] = 1.0 / N
    return c * S.T + (1.0 - c) / N * np.ones((N, N))


def check_k3ex_dense_dangling(O, seed=0):
    """The dangling-node variant against the dense stochastic Google matrix."""
    for k, (N, M) in enumerate([(8, 6), (16, 20), (64, 120), (128, 300)]):
        u, v = random_edges(N, M, seed + 17 * k, hub_bias=0.3)
        R = O.k2_filter(u, v, N, "lowest")
        A, _, _ = dense_kernel2(u, v, N, "lowest")
        assert (A.sum(axis=1) == 0).sum() >= 2, "the case must have dangling rows"
        r0 = np.random.default_rng(seed + k).random(N) + 0.01
        for c in (0.85, 0.5):
            G = google_dangling_matrix(A, c)
            want = r0 / np.abs(r0).sum()
            for _ in range(20):
                want = G @ want
            got, done = O.k3_pagerank_ex(R, r0, 20, c, dangling=True)
            assert done == 20
            assert np.abs(got - want).sum() <= 1e-13 * np.abs(want).sum()


def check_k3ex_conservation(O, seed=0):
    """With the dangling term every row of the update passes all its mass on,
    so sum(r) stays 1 at every iteration, for every graph (also when columns
    are removed: the removed columns' entries are gone before d_out is taken)."""
    for k, (N, M) in enumerate([(32, 200), (256, 1500)]):
        u, v = random_edges(N, M, seed + 7 * k, hub_bias=0.4)
        for rule in ("lowest", "all_ties"):
            R = O.k2_filter(u, v, N, rule)
            r0 = np.random.default_rng(seed + k).random(N) + 0.01
            for iters in (1, 5, 20):
                r, _ = O.k3_pagerank_ex(R, r0, iters, 0.85, dangling=True)
                assert abs(r.sum() - 1.0) <= 1e-14
    # A = 0: every row dangles, so one step gives the uniform vector 1/N
    z = load_golden("k2_all_columns_removed.json")
    e = np.array(z["edges"], dtype=np.uint32)
    N = 1 << z["scale"]
    R = O.k2_filter(e[:, 0], e[:, 1], N, "lowest")
    r, _ = O.k3_pagerank_ex(R, np.array([0.3, 0.1, 0.4, 0.2]), 3, 0.85, dangling=True)
    assert np.allclose(r, 1.0 / N, rtol=1e-15, atol=0)


def check_k3ex_convergence(O, seed=0):
    """The convergence test stops at the first k with norm(r_k - r_(k-1), 1) < tol,
    found independently by the dense iteration; the converged vector is the
    Perron vector of the stochastic Google matrix (Sec. IV-D validation)."""
    for k, (N, M) in enumerate([(24, 120), (96, 700)]):
        u, v = random_edges(N, M, seed + 5 * k, hub_bias=0.3)
        R = O.k2_filter(u, v, N, "lowest")
        A, _, _ = dense_kernel2(u, v, N, "lowest")
        r0 = np.random.default_rng(seed + 9 * k).random(N) + 0.01
        for dangling in (False, True):
            G = google_dangling_matrix(A, 0.85) if dangling else 0.85 * A.T + 0.15 / N * np.ones((N, N))
            for tol in (1e-4, 1e-9):
                r = r0 / np.abs(r0).sum()
                first = None
                for it in range(1, 400):
                    nxt = G @ r
                    if np.abs(nxt - r).sum() < tol:
                        first, r = it, nxt
                        break
                    r = nxt
                got, done = O.k3_pagerank_ex(R, r0, 400, 0.85, dangling=dangling, tol=tol)
                assert done == first, (dangling, tol, done, first)
                assert np.abs(got - r).sum() <= 1e-13 * np.abs(r).sum()
            # tol = 0 runs every iteration
            assert O.k3_pagerank_ex(R, r0, 7, 0.85, dangling=dangling, tol=0.0)[1] == 7
        # converged to 1e-13, the dangling variant is the normalised Perron vector
        G = google_dangling_matrix(A, 0.85)
        w, V = np.linalg.eig(G)
        p = np.real(V[:, int(np.argmax(np.abs(w)))])
        p = p / p.sum()
        got, _ = O.k3_pagerank_ex(R, r0, 1000, 0.85, dangling=True, tol=1e-13)
        assert np.abs(got - p).sum() <= 1e-11


def check_tsv_golden(O):
    """The edge-file text of Sec. IV-A/B against a hand-written fixture, and
    hand-written malformed lines that must be flagged."""
    g = load_golden("edges_tsv_small.json")
    text = g["text"].encode()
    assert O.format_tsv(np.array(g["u"], dtype=np.uint32), np.array(g["v"], dtype=np.uint32)) == text
    u, v, m, bad = O.parse_tsv(text)
    assert not bad and m == len(g["u"]) and u.tolist() == g["u"] and v.tolist() == g["v"]
    for t, why in g["malformed"]:
        assert O.parse_tsv(t.encode())[3], why
    # more lines than the room given
    assert O.parse_tsv(text, cap=2)[3]


def check_tsv_round_trip(O, seed=0):
    """Formatting agrees with Python's own decimal formatting; parsing inverts it."""
    rng = np.random.default_rng(seed)
    for n in (0, 1, 7, 1000):
        u = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
        v = (rng.integers(0, 1 << 12, n)).astype(np.uint32)
        text = O.format_tsv(u, v)
        assert text == "".join("%d\t%d\n" % (a, b) for a, b in zip(u.tolist(), v.tolist())).encode()
        pu, pv, m, bad = O.parse_tsv(text)
        assert not bad and m == n and np.array_equal(pu, u) and np.array_equal(pv, v)


ALL_CHECKS = [
    ("k1_brute_force", check_k1_brute_force),
    ("k3ex_dense_dangling", check_k3ex_dense_dangling),
    ("k3ex_conservation", check_k3ex_conservation),
    ("k3ex_convergence", check_k3ex_convergence),
    ("tsv_golden", check_tsv_golden),
    ("tsv_round_trip", check_tsv_round_trip),
    ("k2_dense", check_k2_dense),
    ("k2_golden", check_k2_golden),
    ("k3_dense", check_k3_dense),
    ("k3_eigenvector", check_k3_eigenvector),
    ("k3_closed_forms", check_k3_closed_forms),
    ("k3_golden", check_k3_golden),
]
