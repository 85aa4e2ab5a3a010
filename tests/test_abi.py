"""The C-ABI libraries load and export every declared entry point (no GPU needed).

Only host-side behaviour is exercised here: size queries and argument checks
that return before any CUDA call.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    text = re.sub(r"typedef\s+(struct|enum)\s*\{.*?\}\s*\w+\s*;", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b((?:pp|k0)_\w+)\s*\(", text)))


@pytest.mark.parametrize("header,lib", [("pagerank_pipeline.h", "paper_1603_01876_gb300/libpp.so"),
                                        ("pagerank_pipeline.h", "paper_1603_01876_gb300/libpp_checked.so"),
                                        ("kernel0.h", "kernel0/libkernel0.so")])
def test_every_declared_symbol_is_exported(header, lib):
    names = declared_functions(header)
    assert len(names) >= 5
    L = ctypes.CDLL(os.path.join(ROOT, lib))
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_pp_declarations_cover_the_three_kernels():
    names = declared_functions("pagerank_pipeline.h")
    for n in ("pp_sort_edges", "pp_build_filter_normalize", "pp_pagerank", "pp_pipeline_host",
              "pp_last_device_error", "pp_status_string", "pp_launch_count"):
        assert n in names


def test_workspace_queries_and_lengths():
    import paper_1603_01876_gb300 as pp

    for kind in ("sort", "build", "pagerank", "pipeline"):
        assert pp.workspace_bytes(kind, 16 << 10, 10) > 0
    assert pp.workspace_bytes("pagerank", 16 << 10, 10, dtype="fp64") > pp.workspace_bytes("pagerank", 16 << 10, 10)
    lens = pp.graph_lengths(16 << 10, 10)
    assert lens[0] == 1025 and lens[1] == 16 << 10 and lens[4] == 1024 and lens[8] == pp.INFO_LEN
    assert len(lens) == pp.GRAPH_ARRAYS and lens[9] == lens[10] == 1024
    # the overflow table bound: each overflow entry needs >= 2^(32-scale)-1 duplicate edges
    assert pp.graph_lengths(1 << 30, 26)[2] == (1 << 30) // 63 + 1


def test_host_side_argument_errors():
    import paper_1603_01876_gb300 as pp

    L = pp.lib()
    n = ctypes.c_size_t(0)
    assert L.pp_sort_edges_workspace(10, 0, ctypes.byref(n)) == pp.PP_ERR_INVALID_ARG
    assert L.pp_sort_edges_workspace(10, 28, ctypes.byref(n)) == pp.PP_ERR_INVALID_ARG
    assert L.pp_sort_edges_workspace((1 << 31) + 1, 20, ctypes.byref(n)) == pp.PP_ERR_INVALID_ARG
    assert L.pp_pagerank_workspace(10, 5, 20, 7, ctypes.byref(n)) == pp.PP_ERR_INVALID_ARG
    out = (ctypes.c_uint64 * pp.GRAPH_ARRAYS)()
    assert L.pp_graph_lengths(10, 30, out) == pp.PP_ERR_INVALID_ARG
    # null pointers and missing workspace are rejected before anything is enqueued
    assert L.pp_sort_edges(None, None, 10, 5, None, None, None, 0, None) == pp.PP_ERR_INVALID_ARG
    fake = ctypes.c_void_p(4096)
    assert L.pp_sort_edges(fake, fake, 10, 5, fake, fake, None, 0, None) == pp.PP_ERR_WORKSPACE
    assert L.pp_sort_edges(fake, fake, 10, 5, fake, fake, ctypes.c_void_p(4096 + 8), 1 << 30, None) == pp.PP_ERR_WORKSPACE
    g = pp.CGraph()
    g.scale, g.M = 5, 10
    assert L.pp_build_filter_normalize(fake, fake, 10, 5, 0, ctypes.byref(g), None, 0, None) == pp.PP_ERR_INVALID_ARG
    assert L.pp_build_filter_normalize(fake, fake, 10, 5, 9, ctypes.byref(g), None, 0, None) == pp.PP_ERR_INVALID_ARG
    assert L.pp_pagerank(ctypes.byref(g), fake, 20, 1.5, 1, fake, None, None, 0, None) == pp.PP_ERR_INVALID_ARG
    for s in range(5):
        assert L.pp_status_string(s)


def test_binding_fails_loudly_without_library(monkeypatch):
    import paper_1603_01876_gb300 as pp

    monkeypatch.setattr(pp, "LIB_PATHS", {"default": "/nonexistent/libpp.so", "checked": "/nonexistent/x.so"})
    monkeypatch.setattr(pp, "_LIBS", {})
    with pytest.raises(ImportError):
        pp.lib()
    monkeypatch.setattr(pp, "_ACTIVE", "checked")
    with pytest.raises(ImportError):
        pp.lib()


def test_build_flags_of_both_libraries():
    """libpp.so is the plain build, libpp_checked.so the bounds-checked one;
    both open NVTX ranges.  Selecting a library changes which one the
    binding calls."""
    import paper_1603_01876_gb300 as pp

    prev = pp.use_library("default")
    try:
        assert pp.build_flags() == pp.BUILD_NVTX
        pp.use_library("checked")
        assert pp.build_flags() == pp.BUILD_CHECKED | pp.BUILD_NVTX
        with pytest.raises(ValueError):
            pp.use_library("fast")
    finally:
        pp.use_library(prev)


def test_tuning_knobs():
    import paper_1603_01876_gb300 as pp

    old = pp.get_tuning("k3_unroll_f32")
    try:
        for v in (4, 8):
            pp.set_tuning("k3_unroll_f32", v)
            assert pp.get_tuning("k3_unroll_f32") == v
        with pytest.raises(pp.PPError):
            pp.set_tuning("k3_unroll_f32", 7)
        with pytest.raises(pp.PPError):
            pp.set_tuning("no_such_knob", 1)
    finally:
        pp.set_tuning("k3_unroll_f32", old)


def test_stored_tuning_file_is_accepted():
    """Every knob the stored GB300 tuning file sets (what bench.py and the
    full-size tests apply) is a knob the library knows, with an allowed value;
    the autotuner searches only allowed values."""
    import json

    import paper_1603_01876_gb300 as pp
    from paper_1603_01876_gb300 import tune

    with open(tune.DEFAULT_PATH) as f:
        data = json.load(f)
    entries = [data["single"]] if "knobs" in data["single"] else list(data["single"].values())
    entries.append(data["batched"])
    searched = dict(tune.SINGLE_KNOBS, **tune.BATCH_KNOBS, k3_unroll_f64=[4, 8])
    for ent in entries:
        knobs = ent["knobs"]
        assert set(knobs) <= set(searched), set(knobs) - set(searched)
        for k, values in searched.items():
            old = pp.get_tuning(k)
            try:
                for v in values:
                    pp.set_tuning(k, v)
                if k in knobs:
                    pp.set_tuning(k, knobs[k])
                    assert pp.get_tuning(k) == knobs[k]
            finally:
                pp.set_tuning(k, old)


def test_tuning_entry_for_scale():
    """The stored entry applied to a graph is that of its scale, else of the
    nearest searched scale below it (the smallest for smaller graphs)."""
    from paper_1603_01876_gb300 import tune

    data = {"single": {"20": {"knobs": {"a": 20}}, "24": {"knobs": {"a": 24}}, "26": {"knobs": {"a": 26}}}}
    assert tune.entry_for_scale(data, 24)["knobs"]["a"] == 24
    assert tune.entry_for_scale(data, 25)["knobs"]["a"] == 24
    assert tune.entry_for_scale(data, 27)["knobs"]["a"] == 26
    assert tune.entry_for_scale(data, 12)["knobs"]["a"] == 20
    assert tune.entry_for_scale(data, None)["knobs"]["a"] == 24
    assert tune.entry_for_scale({"single": {"knobs": {"a": 1}}}, 20)["knobs"]["a"] == 1
