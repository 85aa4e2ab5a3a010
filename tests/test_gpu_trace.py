"""Call tracing in the binding (paper_1603_01876_gb300.trace): CUDA events
around each entry-point call while a trace is open, in call order, nothing
recorded outside it, and the per-call times adding up to the time of the
whole sequence measured around it."""
import pytest

pytestmark = pytest.mark.gpu


def test_trace_records_each_call(k0):
    import torch

    import paper_1603_01876_gb300 as pp

    scale = 16
    u, v = k0.edges_device(scale, 2)
    r0 = torch.from_numpy(k0.r0_host(1 << scale, 2)).cuda()
    pp.pagerank(pp.build_filter_normalize(*pp.sort_edges(u, v, scale), scale), r0, 20)  # warm-up
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with pp.trace() as t:
        e[0].record()
        us, vs = pp.sort_edges(u, v, scale)
        g = pp.build_filter_normalize(us, vs, scale)
        pp.pagerank(g, r0, 20, 0.85, "fp32")
        e[1].record()
    pp.sort_edges(u, v, scale)  # after the block: not recorded
    rep = t.report()
    assert [n for n, _ in rep] == ["sort_edges", "build_filter_normalize", "pagerank"]
    assert all(ms > 0 for _, ms in rep)
    whole = e[0].elapsed_time(e[1])
    assert sum(ms for _, ms in rep) <= whole * 1.05 + 0.05
    assert t.totals()["pagerank"][0] == 1
