"""Failure detection on the GPU: a bounded cross-block wait that runs out.

The wait is made to expire by a status word that nothing writes (the first
tile of a scatter pass is never processed); no fault, trap or endless loop is
involved.  The kernel must record the timeout in the device error word and
return, and the context must stay usable for the next call.
"""
import numpy as np
import pytest

from gpu_helpers import host_u32

pytestmark = pytest.mark.gpu

PP_DEV_TIMEOUT = 2


def test_lookback_wait_expires_and_context_survives(k0, oracle_mod):
    import torch

    import paper_1603_01876_gb300 as pp

    assert pp.last_device_error() == 0
    err = pp.selftest_lookback_timeout(1000)
    assert err & PP_DEV_TIMEOUT, "expired wait not reported (error bits %#x)" % err
    assert pp.last_device_error() == 0, "the error word is cleared once read"

    # the next call on the same context sorts correctly
    scale = 10
    u, v = k0.edges_device(scale, 3, device="cuda")
    us, vs = pp.sort_edges(u, v, scale)
    torch.cuda.synchronize()
    assert pp.last_device_error() == 0
    exp_u, exp_v = oracle_mod.k1_sort(host_u32(u), host_u32(v))
    np.testing.assert_array_equal(host_u32(us), exp_u)
    np.testing.assert_array_equal(host_u32(vs), exp_v)


def test_selftest_argument_errors():
    import paper_1603_01876_gb300 as pp

    with pytest.raises(pp.PPError):
        pp.selftest_lookback_timeout(0)
