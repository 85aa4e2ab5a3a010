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


def _ref_parse(text):
    """The edge-file grammar written out: one "digits<TAB>digits" per line,
    each field 1-10 digits and at most 2^32-1, a line (with its newline) at
    most 22 bytes, the text ending with a newline; a malformed line reads as
    (0, 0)."""
    lines = text.split(b"\n")
    bad = lines[-1] != b""
    out = []
    for ln in lines[:-1]:
        parts = ln.split(b"\t")
        ok = (len(ln) + 1 <= 22 and len(parts) == 2
              and all(p and p.isdigit() and len(p) <= 10 and int(p) <= 2**32 - 1 for p in parts))
        bad |= not ok
        out.append((int(parts[0]), int(parts[1])) if ok else (0, 0))
    return out, bad


_field = st.one_of(st.integers(0, 2**32 - 1).map(lambda x: b"%d" % x),
                   st.text(alphabet="0123456789", min_size=0, max_size=12).map(str.encode),
                   st.text(alphabet="0123456789 +-a\t", min_size=0, max_size=6).map(str.encode))
_line = st.one_of(st.tuples(st.integers(0, 2**32 - 1), st.integers(0, 2**32 - 1)).map(lambda t: b"%d\t%d" % t),
                  st.tuples(_field, _field).map(lambda t: t[0] + b"\t" + t[1]),
                  _field)


@SETTINGS
@given(lines=st.lists(_line, max_size=40), tail=st.booleans(), room=st.integers(0, 45))
def test_parse_tsv_is_the_grammar(O, lines, tail, room):
    text = b"\n".join(lines) + (b"\n" if lines and tail else b"")
    want, want_bad = _ref_parse(text)
    u, v, m, bad = O.parse_tsv(text, cap=room)
    assert m == len(want)
    assert bad == (want_bad or len(want) > room)
    k = min(m, room)
    assert list(zip(u[:k].tolist(), v[:k].tolist())) == want[:k]


@SETTINGS
@given(edges=st.lists(st.tuples(st.integers(0, 2**32 - 1), st.integers(0, 2**32 - 1)), max_size=200))
def test_format_tsv_is_pythons_decimal(O, edges):
    u = np.array([a for a, _ in edges], dtype=np.uint32)
    v = np.array([b for _, b in edges], dtype=np.uint32)
    text = O.format_tsv(u, v)
    assert text == b"".join(b"%d\t%d\n" % e for e in edges)
    pu, pv, m, bad = O.parse_tsv(text)
    assert not bad and m == len(edges) and pu.tolist() == u.tolist() and pv.tolist() == v.tolist()
