"""Host-side fault injection (pp_inject_fault), on the CPU: an armed entry
point returns the chosen status at once, before any argument check or CUDA
call, for exactly the armed number of calls; the binding turns it into
PPError; "*" arms every entry point; count 0 disarms."""
import ctypes

import pytest


@pytest.fixture
def pp():
    import paper_1603_01876_gb300 as pp

    yield pp
    pp.inject_fault("*", pp.PP_ERR_CUDA, 0)
    pp.inject_fault("pp_sort_edges", pp.PP_ERR_CUDA, 0)
    pp.inject_fault("pp_last_device_error", pp.PP_ERR_CUDA, 0)


def test_armed_call_fails_the_given_number_of_times(pp):
    L = pp.lib()
    # unarmed: the argument check answers (no CUDA call is made)
    assert L.pp_sort_edges(None, None, 10, 5, None, None, None, 0, None) == pp.PP_ERR_INVALID_ARG
    pp.inject_fault("pp_sort_edges", pp.PP_ERR_CUDA, 2)
    assert L.pp_sort_edges(None, None, 10, 5, None, None, None, 0, None) == pp.PP_ERR_CUDA
    # other entry points are not affected
    g = pp.CGraph()
    assert L.pp_build_filter_normalize(None, None, 10, 0, 0, ctypes.byref(g), None, 0, None) == pp.PP_ERR_INVALID_ARG
    assert L.pp_sort_edges(None, None, 10, 5, None, None, None, 0, None) == pp.PP_ERR_CUDA
    assert L.pp_sort_edges(None, None, 10, 5, None, None, None, 0, None) == pp.PP_ERR_INVALID_ARG


def test_binding_raises_the_injected_status(pp):
    import torch

    import types

    pp.inject_fault("pp_sort_edges", pp.PP_ERR_WORKSPACE, 1)
    u = torch.zeros(8, dtype=torch.int32)
    no_gpu_stream = types.SimpleNamespace(cuda_stream=0)  # the call fails before using it
    with pytest.raises(pp.PPError) as e:
        pp.sort_edges(u, u, 3, out=(u, u), workspace=torch.zeros(1 << 16, dtype=torch.uint8), stream=no_gpu_stream)
    assert e.value.status == pp.PP_ERR_WORKSPACE


def test_wildcard_device_error_and_disarm(pp):
    L = pp.lib()
    pp.inject_fault("*", pp.PP_ERR_DEVICE, 3)
    assert L.pp_pagerank(None, None, 20, 0.85, 1, None, None, None, 0, None) == pp.PP_ERR_DEVICE
    code = ctypes.c_uint32(7)
    assert L.pp_last_device_error(None, ctypes.byref(code)) == pp.PP_ERR_DEVICE
    assert code.value == 7  # outputs untouched
    pp.inject_fault("*", pp.PP_ERR_DEVICE, 0)
    assert L.pp_pagerank(None, None, 20, 0.85, 1, None, None, None, 0, None) == pp.PP_ERR_INVALID_ARG


def test_injection_argument_errors(pp):
    L = pp.lib()
    assert L.pp_inject_fault(None, pp.PP_ERR_CUDA, 1) == pp.PP_ERR_INVALID_ARG
    assert L.pp_inject_fault(b"x" * 64, pp.PP_ERR_CUDA, 1) == pp.PP_ERR_INVALID_ARG
    assert L.pp_inject_fault(b"pp_sort_edges", pp.PP_OK, 1) == pp.PP_ERR_INVALID_ARG
    assert L.pp_inject_fault(b"pp_sort_edges", 9, 1) == pp.PP_ERR_INVALID_ARG
    assert L.pp_inject_fault(b"pp_sort_edges", pp.PP_OK, 0) == pp.PP_OK  # disarming what is not armed
    names = [b"pp_fake_%d" % i for i in range(16)]
    try:
        for n in names:
            assert L.pp_inject_fault(n, pp.PP_ERR_CUDA, 1) == pp.PP_OK
        assert L.pp_inject_fault(b"pp_one_more", pp.PP_ERR_CUDA, 1) == pp.PP_ERR_INVALID_ARG  # table full
    finally:
        for n in names:
            L.pp_inject_fault(n, pp.PP_ERR_CUDA, 0)
