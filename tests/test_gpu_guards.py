"""Guard zones around every array the path writes.

Each output array and each workspace of the path is placed inside a larger
buffer whose surrounding bytes hold a fixed pattern; after the calls the
pattern must be intact: nothing is written before an array or past its
declared length (the graph arrays' lengths from pp_graph_lengths, the
workspace size the size query returned, N ranks, the edge count).  This and
the bounds-checked build stand in for a memory checker.
"""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

GUARD = 4096  # bytes on each side; a multiple of 256 keeps every array's alignment
PATTERN = 0xA5


class Guards:
    def __init__(self, device="cuda"):
        self.device = device
        self.bufs = []

    def empty(self, n, dtype):
        import torch

        nbytes = n * torch.empty(0, dtype=dtype).element_size()
        raw = torch.full((nbytes + 2 * GUARD,), PATTERN, dtype=torch.uint8, device=self.device)
        self.bufs.append((raw, nbytes))
        return raw[GUARD:GUARD + nbytes].view(dtype)

    def intact(self):
        bad = []
        for i, (raw, nb) in enumerate(self.bufs):
            if not (bool((raw[:GUARD] == PATTERN).all()) and bool((raw[GUARD + nb:] == PATTERN).all())):
                bad.append(i)
        return bad


def _size(fn, *args):
    import paper_1603_01876_gb300 as pp

    n = ctypes.c_size_t(0)
    assert getattr(pp.lib(), fn)(*args, ctypes.byref(n)) == pp.PP_OK
    return n.value


@pytest.mark.parametrize("scale,M", [(11, 16 * 2048 - 13), (14, None)], ids=["s11_ragged", "s14"])
def test_single_graph_calls_stay_inside_their_arrays(k0, scale, M):
    import torch

    import paper_1603_01876_gb300 as pp

    N = 1 << scale
    u, v = k0.edges_device(scale, 6, M=M)
    M = u.numel()
    gd = Guards()
    us, vs = gd.empty(M, torch.int32), gd.empty(M, torch.int32)
    pp.sort_edges(u, v, scale, out=(us, vs), workspace=gd.empty(pp.workspace_bytes("sort", M, scale), torch.uint8))
    g = pp.Graph(M, scale, u.device, alloc=gd.empty)
    pp.build_filter_normalize(us, vs, scale, graph=g,
                              workspace=gd.empty(pp.workspace_bytes("build", M, scale), torch.uint8))
    r0 = torch.from_numpy(k0.r0_host(N, 6)).cuda()
    for dt in ("fp64", "fp32", "bf16", "fp16"):
        out = gd.empty(N, torch.float64 if dt == "fp64" else torch.float32)
        pp.pagerank(g, r0, 20, 0.85, dt, out=out,
                    workspace=gd.empty(pp.workspace_bytes("pagerank", M, scale, 20, dt), torch.uint8))
        out = gd.empty(N, torch.float64 if dt == "fp64" else torch.float32)
        if dt in ("fp64", "fp32"):
            pp.pagerank_ex(g, r0, 100, 0.85, dt, dangling=True, tol=1e-8, out=out,
                           workspace=gd.empty(pp.workspace_bytes("pagerank_ex", M, scale, 100, dt), torch.uint8))
    pp.export_csr(g, workspace=gd.empty(_size("pp_export_csr_workspace", M, scale), torch.uint8))
    assert pp.last_device_error() == 0
    assert gd.intact() == []


def test_batched_calls_stay_inside_their_arrays(k0):
    import torch

    import paper_1603_01876_gb300 as pp

    scales = [10, 3, 12, 7]
    us, vs = zip(*[k0.edges_device(s, 8, graph=i) for i, s in enumerate(scales)])
    n = len(scales)
    gd = Guards()
    Ms = (ctypes.c_uint64 * n)(*[u.numel() for u in us])
    Ss = (ctypes.c_uint32 * n)(*scales)
    outs = [(gd.empty(u.numel(), torch.int32), gd.empty(u.numel(), torch.int32)) for u in us]
    pp.sort_edges_batched(list(us), list(vs), scales, outs=outs,
                          workspace=gd.empty(_size("pp_sort_edges_batched_workspace", n, Ms, Ss), torch.uint8))
    graphs = [pp.Graph(u.numel(), s, u.device, alloc=gd.empty) for u, s in zip(us, scales)]
    pp.build_filter_normalize_batched(outs, scales, graphs=graphs, workspace=gd.empty(
        _size("pp_build_filter_normalize_batched_workspace", n, Ms, Ss), torch.uint8))
    rows = sum(1 << s for s in scales)
    arr = (pp.CGraph * n)(*[g.c for g in graphs])
    for nrhs in (4, 32):
        r0 = torch.ones(rows, nrhs, dtype=torch.float64, device="cuda")
        pp.pagerank_batched(graphs, r0, nrhs, 20, out=gd.empty(rows * nrhs, torch.float32).view(rows, nrhs),
                            workspace=gd.empty(_size("pp_pagerank_batched_workspace", arr, n, nrhs, 20),
                                               torch.uint8))
    assert pp.last_device_error() == 0
    assert gd.intact() == []
