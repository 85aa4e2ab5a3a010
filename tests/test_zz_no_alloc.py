"""The allocation-free Kernel 1 entry point (pp_sort_edges_static).

Some callers cannot allocate device memory: their GPU memory is owned by
another allocator, or cudaMalloc's implicit synchronisation would stall their
other streams.  pp_sort_edges_static serves them from a fixed device array.
These tests call it through the C-ABI, twice in a row (the array keeps the
previous call's contents), and require the same bits as pp_sort_edges.  The
file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_fn():
    import paper_1603_01876_gb300 as pp

    f = pp.lib().pp_sort_edges_static
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp]
    f.restype = ctypes.c_int
    return f


@pytest.mark.parametrize("scale,M", [(16, 1 << 20), (20, 1000003), (10, 4097)])
def test_static_sort_matches_sort_edges_twice(k0, scale, M):
    import torch

    import paper_1603_01876_gb300 as pp

    f = _static_fn()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed in (3, 4):  # two calls in a row with different inputs
        u, v = k0.edges_device(scale, seed, M=M)
        want_u, want_v = pp.sort_edges(u, v, scale)
        got_u = torch.empty_like(u)
        got_v = torch.empty_like(v)
        rc = f(u.data_ptr(), v.data_ptr(), M, scale, got_u.data_ptr(), got_v.data_ptr(), stream)
        assert rc == pp.PP_OK
        torch.cuda.synchronize()
        assert torch.equal(got_u, want_u) and torch.equal(got_v, want_v)
    assert pp.last_device_error() == 0


def test_static_sort_rejects_too_many_edges():
    import paper_1603_01876_gb300 as pp

    f = _static_fn()
    fake = ctypes.c_void_p(4096)
    assert f(fake, fake, (1 << 20) + 1, 20, fake, fake, None) == pp.PP_ERR_INVALID_ARG
