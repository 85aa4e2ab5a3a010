"""The seeded input generator (Kernel 0 shape) on the host: no GPU needed."""
import numpy as np
import pytest


def test_philox_known_answers(k0):
    # Known-answer vectors published with the Philox4x32-10 reference (Salmon et al., SC'11).
    kat = [
        ([0, 0, 0, 0], [0, 0], [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]),
        ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2, [0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]),
        ([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344], [0xA4093822, 0x299F31D0],
         [0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]),
    ]
    for ctr, key, want in kat:
        assert k0.philox(ctr, key).tolist() == want


@pytest.mark.parametrize("scale", [1, 2, 5, 10, 16])
def test_relabel_is_bijection(k0, scale):
    p = k0.params(scale, seed=123)
    x = k0.relabel(p, np.arange(1 << scale, dtype=np.uint32))
    assert np.array_equal(np.sort(x), np.arange(1 << scale, dtype=np.uint32))


def test_edges_in_range_and_deterministic(k0):
    u, v = k0.edges_host(10, seed=1)
    assert len(u) == 16 << 10 and u.max() < 1024 and v.max() < 1024
    u2, v2 = k0.edges_host(10, seed=1, threads=1)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    u3, _ = k0.edges_host(10, seed=2)
    assert not np.array_equal(u, u3)
    # a slice of the stream equals the same edges generated on their own
    us, vs = k0.edges_host(10, seed=1, M=1000, e0=5000)
    assert np.array_equal(us, u[5000:6000]) and np.array_equal(vs, v[5000:6000])


def test_quadrant_frequencies(k0):
    """Without the relabel, bit l of (u, v) follows the initiator: P(0,0)=A, (0,1)=B, (1,0)=C, (1,1)=D."""
    S, M = 8, 200000
    p = k0.params(S, seed=9)
    p.mul[0] = p.mul[1] = p.mul[2] = 1
    p.add[0] = p.add[1] = p.add[2] = 0
    p.shift = 31
    u = np.empty(M, np.uint32)
    v = np.empty(M, np.uint32)
    import ctypes

    assert k0.lib().k0_gen_edges_host(ctypes.byref(p), 0, M, u.ctypes.data, v.ctypes.data, 0) == 0
    A, B, C, D = k0.INITIATOR
    for level in range(S):
        ib = (u >> level) & 1
        jb = (v >> level) & 1
        freq = np.bincount(ib * 2 + jb, minlength=4) / M
        # 5 standard deviations of a binomial proportion
        for f, pr in zip(freq, (A, B, C, D)):
            assert abs(f - pr) < 5 * np.sqrt(pr * (1 - pr) / M)


def test_r0_range(k0):
    r = k0.r0_host(100000, seed=3)
    assert (r > 0).all() and (r < 1).all()
    assert abs(r.mean() - 0.5) < 0.01
    assert not np.array_equal(r, k0.r0_host(100000, seed=3, rhs=1))
    assert np.array_equal(r, k0.r0_host(100000, seed=3, threads=1))


def test_batch_scales(k0):
    s = k0.batch_scales(64, 12, 18, seed=1)
    assert len(s) == 64 and min(s) >= 12 and max(s) <= 18
