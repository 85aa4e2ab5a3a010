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


_RESET_SCRIPT = r"""
import ctypes, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import kernel0
import os
_rt = "/usr/local/cuda/lib64/libcudart.so.13"
rt = ctypes.CDLL(_rt if os.path.exists(_rt) else "libcudart.so.13", mode=ctypes.RTLD_GLOBAL)
pp = ctypes.CDLL(sys.argv[2])
vp = ctypes.c_void_p
pp.pp_sort_edges_static.argtypes = [vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp]
pp.pp_sort_edges_static.restype = ctypes.c_int
scale, M = 12, 50000
u, v = kernel0.edges_host(scale, 7, M=M)
order = np.lexsort((v, u))

def run_once():
    ptrs = []
    for _ in range(4):
        p = vp()
        assert rt.cudaMalloc(ctypes.byref(p), ctypes.c_size_t(4 * M)) == 0
        ptrs.append(p)
    for src, dst in ((u, ptrs[0]), (v, ptrs[1])):
        assert rt.cudaMemcpy(dst, src.ctypes.data_as(vp), ctypes.c_size_t(4 * M), 1) == 0
    assert pp.pp_sort_edges_static(ptrs[0], ptrs[1], M, scale, ptrs[2], ptrs[3], None) == 0
    assert rt.cudaDeviceSynchronize() == 0
    out = []
    for p in ptrs[2:]:
        h = np.empty(M, dtype=np.uint32)
        assert rt.cudaMemcpy(h.ctypes.data_as(vp), p, ctypes.c_size_t(4 * M), 2) == 0
        out.append(h)
    for p in ptrs:
        rt.cudaFree(p)
    return out

for k in range(3):
    gu, gv = run_once()
    assert np.array_equal(gu, u[order]) and np.array_equal(gv, v[order]), k
    # ends this process's context; the next call must find the array anew
    assert rt.cudaDeviceReset() == 0
print("ok")
"""


def test_static_sort_after_device_reset(tmp_path):
    """A device reset replaces the context and reloads the library's module,
    so the scratch array's address may change; calls after the reset must
    look it up again.  Runs in a child process, whose reset ends only its own
    context."""
    import os
    import subprocess
    import sys

    import paper_1603_01876_gb300 as pp

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "reset_child.py"
    script.write_text(_RESET_SCRIPT)
    r = subprocess.run([sys.executable, str(script), root, pp.LIB_PATH], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
