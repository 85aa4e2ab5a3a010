"""The edge files of Kernels 0-2 (Sec. IV-A, IV-B) on the GPU: formatting and
parsing against the oracle, byte for byte and value for value, including
malformed text that must be flagged without any access out of bounds."""
import numpy as np
import pytest

from gpu_helpers import host_u32

pytestmark = pytest.mark.gpu

PP_DEV_PARSE = 4


@pytest.fixture(scope="module")
def pp():
    import paper_1603_01876_gb300 as pp

    return pp


def _dev_bytes(b):
    import torch

    t = torch.zeros(max(1, len(b)), dtype=torch.uint8)
    t[: len(b)] = torch.frombuffer(bytearray(b), dtype=torch.uint8) if len(b) else t[:0]
    return t.cuda()


@pytest.mark.parametrize("scale,M,seed", [(4, 1, 1), (8, 1000, 2), (10, None, 3), (16, 1023 * 1024 + 5, 4),
                                          (20, None, 5)])
def test_format_and_parse_vs_oracle(pp, k0, oracle_mod, scale, M, seed):
    import torch

    u, v = k0.edges_device(scale, seed, M=M)
    text, n = pp.format_tsv(u, v)
    L = int(n.item())
    want = oracle_mod.format_tsv(host_u32(u), host_u32(v))
    assert L == len(want)
    assert text[:L].cpu().numpy().tobytes() == want
    pu, pv, m = pp.parse_tsv(text, L, u.numel())
    torch.cuda.synchronize()
    assert pp.last_device_error() == 0
    assert int(m.item()) == u.numel()
    assert torch.equal(pu[: u.numel()], u) and torch.equal(pv[: v.numel()], v)


def test_extreme_values_and_golden(pp, oracle_mod):
    import json
    import os

    import torch

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "edges_tsv_small.json")))
    u = torch.tensor(np.array(g["u"], dtype=np.uint32).view(np.int32)).cuda()
    v = torch.tensor(np.array(g["v"], dtype=np.uint32).view(np.int32)).cuda()
    text, n = pp.format_tsv(u, v)
    assert text[: int(n.item())].cpu().numpy().tobytes() == g["text"].encode()
    pu, pv, m = pp.parse_tsv(_dev_bytes(g["text"].encode()), len(g["text"]), 16)
    assert pp.last_device_error() == 0 and int(m.item()) == len(g["u"])
    assert host_u32(pu)[: len(g["u"])].tolist() == g["u"] and host_u32(pv)[: len(g["v"])].tolist() == g["v"]


def test_malformed_text_is_flagged(pp, oracle_mod):
    import json
    import os

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "edges_tsv_small.json")))
    for t, why in g["malformed"]:
        b = t.encode()
        pu, pv, m = pp.parse_tsv(_dev_bytes(b), len(b), 8)
        err = pp.last_device_error()
        assert err & PP_DEV_PARSE, why
        ou, ov, om, bad = oracle_mod.parse_tsv(b, cap=8)
        assert bad and int(m.item()) == om, why
        assert host_u32(pu)[:om].tolist() == ou.tolist() and host_u32(pv)[:om].tolist() == ov.tolist(), why
    # more lines than room: flagged, the first m_cap lines kept
    b = g["text"].encode()
    pu, pv, m = pp.parse_tsv(_dev_bytes(b), len(b), 2)
    assert pp.last_device_error() & PP_DEV_PARSE
    assert host_u32(pu)[:2].tolist() == g["u"][:2]


def test_long_line_across_chunks(pp, oracle_mod):
    """Lines straddling the 32-byte chunks and 8192-byte tiles of the parser."""
    rng = np.random.default_rng(7)
    u = rng.integers(0, 1 << 32, 20000, dtype=np.uint64).astype(np.uint32)
    v = rng.integers(0, 1 << 32, 20000, dtype=np.uint64).astype(np.uint32)
    b = oracle_mod.format_tsv(u, v)
    pu, pv, m = pp.parse_tsv(_dev_bytes(b), len(b), len(u))
    assert pp.last_device_error() == 0 and int(m.item()) == len(u)
    assert np.array_equal(host_u32(pu), u) and np.array_equal(host_u32(pv), v)
    # the same text at an odd address (unaligned loads)
    import torch

    t = torch.zeros(len(b) + 1, dtype=torch.uint8)
    t[1:] = torch.frombuffer(bytearray(b), dtype=torch.uint8)
    t = t.cuda()
    pu, pv, m = pp.parse_tsv(t[1:], len(b), len(u))
    assert pp.last_device_error() == 0 and np.array_equal(host_u32(pu), u) and np.array_equal(host_u32(pv), v)
