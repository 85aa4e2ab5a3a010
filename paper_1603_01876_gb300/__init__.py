"""Python binding of libpp: the GB300 CUDA path of the PageRank pipeline.

Argument marshalling only.  Every step of Kernels 1-3 runs in the CUDA
kernels behind include/pagerank_pipeline.h; this module passes device
pointers (from torch tensors) and sizes through ctypes, and raises if the
library is missing: there is no CPU fallback.

    sort_edges(u, v, scale)                      Kernel 1 (Sec. IV-B)
    build_filter_normalize(us, vs, scale, rule)  Kernel 2 (Sec. IV-C) -> Graph
    export_csr(graph)                            Kernel 2's A in vertex-order rows
    pagerank(graph, r0, iters, c, dtype)         Kernel 3 (Sec. IV-D)
    pipeline_host(u, v, scale, r0, ...)          Kernels 1-3 from host buffers

Vertex ids travel as torch.int32 tensors holding uint32 bit patterns.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpp.so")
# The bounds-checked build of the same sources (PP_DEV_BOUNDS instead of an
# out-of-range access); PP_LIBRARY=checked in the environment selects it.
LIB_PATHS = {"default": LIB_PATH, "checked": os.path.join(HERE, "libpp_checked.so")}
BUILD_CHECKED, BUILD_NVTX = 1, 2

PP_OK, PP_ERR_INVALID_ARG, PP_ERR_WORKSPACE, PP_ERR_CUDA, PP_ERR_DEVICE = range(5)
DTYPES = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
RULES = {"lowest": 0, "all_ties": 1}
INFO = {"nnz0": 0, "nnz": 1, "dmax": 2, "vmax": 3, "ties": 4, "novf": 5, "supernodes": 6}
INFO_LEN = 8
GRAPH_ARRAYS = 11
DEV_RANGE, DEV_TIMEOUT, DEV_PARSE, DEV_CAPACITY, DEV_BOUNDS = 1, 2, 4, 8, 16


class PPError(RuntimeError):
    def __init__(self, fn, status, detail=""):
        msg = "%s failed: %s" % (fn, _lib().pp_status_string(status).decode())
        super().__init__(msg + (" " + detail if detail else ""))
        self.status = status


class CGraph(ctypes.Structure):
    _fields_ = [
        ("scale", ctypes.c_uint32), ("reserved", ctypes.c_uint32), ("M", ctypes.c_uint64),
        ("colptr", ctypes.c_void_p), ("rowc", ctypes.c_void_p), ("ovf_key", ctypes.c_void_p),
        ("ovf_cnt", ctypes.c_void_p), ("d_in", ctypes.c_void_p), ("d_out", ctypes.c_void_p),
        ("inv_dout32", ctypes.c_void_p), ("inv_dout64", ctypes.c_void_p), ("info", ctypes.c_void_p),
        ("perm", ctypes.c_void_p), ("iperm", ctypes.c_void_p),
    ]


_LIBS = {}
_ACTIVE = os.environ.get("PP_LIBRARY", "default")


def use_library(kind):
    """Selects the library later calls go through: "default" (libpp.so) or
    "checked" (libpp_checked.so); returns the previous choice.  Graphs and
    workspaces are plain device memory and may be passed between the two;
    tuning knobs are kept per library."""
    global _ACTIVE
    if kind not in LIB_PATHS:
        raise ValueError("unknown library %r" % (kind,))
    prev, _ACTIVE = _ACTIVE, kind
    return prev


def _lib():
    L = _LIBS.get(_ACTIVE)
    if L is None:
        path = LIB_PATHS.get(_ACTIVE)
        if path is None:
            raise ImportError("PP_LIBRARY=%r names no library (default or checked)" % (_ACTIVE,))
        if not os.path.exists(path):
            raise ImportError("%s is not built (run __graft_entry__.build()); there is no CPU fallback"
                              % os.path.basename(path))
        L = ctypes.CDLL(path)
        vp, u32, u64, sz = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_size_t)
        i32, dbl = ctypes.c_int, ctypes.c_double
        sig = {
            "pp_graph_lengths": [u64, u32, vp],
            "pp_sort_edges_workspace": [u64, u32, sz],
            "pp_sort_edges": [vp, vp, u64, u32, vp, vp, vp, ctypes.c_size_t, vp],
            "pp_build_filter_normalize_workspace": [u64, u32, sz],
            "pp_build_filter_normalize": [vp, vp, u64, u32, i32, ctypes.POINTER(CGraph), vp, ctypes.c_size_t, vp],
            "pp_pagerank_workspace": [u64, u32, u32, i32, sz],
            "pp_pagerank": [ctypes.POINTER(CGraph), vp, u32, dbl, i32, vp, vp, vp, ctypes.c_size_t, vp],
            "pp_pipeline_workspace": [u64, u32, u32, i32, sz],
            "pp_pipeline_host": [vp, vp, u64, u32, vp, u32, dbl, i32, i32, vp, vp, vp, ctypes.c_size_t, vp],
            "pp_last_device_error": [vp, ctypes.POINTER(ctypes.c_uint32)],
            "pp_pagerank_batched_workspace": [ctypes.POINTER(CGraph), u32, u32, u32, sz],
            "pp_pagerank_batched": [ctypes.POINTER(CGraph), u32, vp, u32, u32, dbl, vp, vp, ctypes.c_size_t, vp],
            "pp_selftest_lookback_timeout": [u32, vp, ctypes.c_size_t, sz, vp],
            "pp_pagerank_ex_workspace": [u64, u32, u32, i32, sz],
            "pp_format_tsv_workspace": [u64, sz],
            "pp_format_tsv": [vp, vp, u64, vp, u64, vp, vp, ctypes.c_size_t, vp],
            "pp_parse_tsv_workspace": [u64, sz],
            "pp_parse_tsv": [vp, u64, vp, vp, u64, vp, vp, ctypes.c_size_t, vp],
            "pp_pagerank_ex": [ctypes.POINTER(CGraph), vp, u32, dbl, i32, u32, dbl, vp, vp, vp, vp, ctypes.c_size_t,
                               vp],
            "pp_pagerank_batched_capture": [ctypes.POINTER(CGraph), u32, vp, u32, u32, dbl, vp, vp, ctypes.c_size_t,
                                            vp, ctypes.POINTER(vp)],
            "pp_exec_launch": [vp, vp],
            "pp_export_csr_workspace": [u64, u32, sz],
            "pp_export_csr": [ctypes.POINTER(CGraph), vp, vp, vp, vp, vp, u64, vp, ctypes.c_size_t, vp],
            "pp_exec_destroy": [vp],
            "pp_gather_probe": [vp, u64, u32, vp, vp, vp],
            "pp_range_counts": [vp, u64, vp, u32, vp, vp],
            "pp_in_degree": [vp, u64, u32, vp, vp],
            "pp_build_filter_normalize_rows": [vp, vp, u64, u32, i32, vp, ctypes.POINTER(CGraph), vp, ctypes.c_size_t,
                                               vp],
            "pp_rank_update": [vp, u64, dbl, dbl, vp, vp, i32, vp, ctypes.c_size_t, vp],
            "pp_sort_edges_batched_workspace": [u32, vp, vp, sz],
            "pp_sort_edges_batched": [u32, vp, vp, vp, vp, vp, vp, vp, ctypes.c_size_t, vp],
            "pp_build_filter_normalize_batched_workspace": [u32, vp, vp, sz],
            "pp_build_filter_normalize_batched": [u32, vp, vp, i32, ctypes.POINTER(CGraph), vp, ctypes.c_size_t, vp],
            "pp_pipeline_batched_workspace": [u32, ctypes.POINTER(CGraph), u32, u32, sz],
            "pp_pipeline_batched_capture": [u32, vp, vp, vp, vp, i32, ctypes.POINTER(CGraph), vp, u32, u32, dbl, vp,
                                            vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.pp_status_string.argtypes = [ctypes.c_int]
        L.pp_status_string.restype = ctypes.c_char_p
        L.pp_set_tuning.argtypes = [ctypes.c_char_p, ctypes.c_int64]
        L.pp_set_tuning.restype = ctypes.c_int
        L.pp_get_tuning.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64)]
        L.pp_get_tuning.restype = ctypes.c_int
        L.pp_launch_count.argtypes = []
        L.pp_launch_count.restype = ctypes.c_uint64
        L.pp_build_flags.argtypes = []
        L.pp_build_flags.restype = ctypes.c_uint32
        L.pp_inject_fault.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.c_uint32]
        L.pp_inject_fault.restype = ctypes.c_int
        _LIBS[_ACTIVE] = L
    return L


def lib():
    return _lib()


def inject_fault(call, status=PP_ERR_CUDA, count=1):
    """Arms a host-side failure: the next `count` calls of the C entry point
    `call` ("*": any) return `status` at once (count 0 disarms it)."""
    _check("pp_inject_fault", _lib().pp_inject_fault(call.encode(), int(status), int(count)))


def build_flags():
    """BUILD_CHECKED | BUILD_NVTX bits of the library in use."""
    return int(_lib().pp_build_flags())


def _check(fn, st):
    if st != PP_OK:
        raise PPError(fn, st)


def _stream(stream, device=None):
    if stream is None:
        stream = torch.cuda.current_stream(device)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _workspace(nbytes, device):
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def set_tuning(key, value):
    """Set a library tuning knob (see pp_set_tuning in include/pagerank_pipeline.h)."""
    _check("pp_set_tuning(%s=%r)" % (key, value), _lib().pp_set_tuning(key.encode(), int(value)))


def get_tuning(key):
    v = ctypes.c_int64(0)
    _check("pp_get_tuning(%s)" % key, _lib().pp_get_tuning(key.encode(), ctypes.byref(v)))
    return int(v.value)


def launch_count():
    return int(_lib().pp_launch_count())


def last_device_error(stream=None):
    """Synchronise and return (and clear) the device error bits (0 = none)."""
    code = ctypes.c_uint32(0)
    st = _lib().pp_last_device_error(_stream(stream), ctypes.byref(code))
    if st not in (PP_OK, PP_ERR_DEVICE):
        raise PPError("pp_last_device_error", st)
    return int(code.value)


def selftest_lookback_timeout(spin_limit, device=None, stream=None):
    """Run the bounded-wait self-test; returns the device error bits it left."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    need = ctypes.c_size_t(0)
    _check("pp_selftest_lookback_timeout",
           _lib().pp_selftest_lookback_timeout(spin_limit, None, 0, ctypes.byref(need), None))
    ws = torch.empty(need.value, dtype=torch.uint8, device=dev)
    _check("pp_selftest_lookback_timeout",
           _lib().pp_selftest_lookback_timeout(spin_limit, _ptr(ws), ws.numel(), None, _stream(stream, dev)))
    return last_device_error(stream)


def graph_lengths(M, scale):
    out = (ctypes.c_uint64 * GRAPH_ARRAYS)()
    _check("pp_graph_lengths", _lib().pp_graph_lengths(M, scale, out))
    return list(out)


def workspace_bytes(kind, M, scale, iters=20, dtype="fp32"):
    n = ctypes.c_size_t(0)
    L = _lib()
    if kind == "sort":
        st = L.pp_sort_edges_workspace(M, scale, ctypes.byref(n))
    elif kind == "build":
        st = L.pp_build_filter_normalize_workspace(M, scale, ctypes.byref(n))
    elif kind == "pagerank":
        st = L.pp_pagerank_workspace(M, scale, iters, DTYPES[dtype], ctypes.byref(n))
    elif kind == "pagerank_ex":
        st = L.pp_pagerank_ex_workspace(M, scale, iters, DTYPES[dtype], ctypes.byref(n))
    elif kind == "pipeline":
        st = L.pp_pipeline_workspace(M, scale, iters, DTYPES[dtype], ctypes.byref(n))
    else:
        raise ValueError(kind)
    _check("workspace query", st)
    return int(n.value)


class Graph:
    """Kernel 2's output (device tensors) and the C struct that points at them."""

    def __init__(self, M, scale, device, alloc=None):
        """alloc(n, dtype) -> device tensor of n elements, if given, provides
        the arrays (e.g. placed inside larger buffers)."""
        lens = graph_lengths(M, scale)
        i32, i64 = torch.int32, torch.int64
        new = alloc or (lambda n, dt: torch.empty(n, dtype=dt, device=device))
        self.M, self.scale, self.N = M, scale, 1 << scale
        self.colptr = new(lens[0], i32)
        self.rowc = new(lens[1], i32)
        self.ovf_key = new(lens[2], i64)
        self.ovf_cnt = new(lens[3], i32)
        self.d_in = new(lens[4], i32)
        self.d_out = new(lens[5], i32)
        self.inv_dout32 = new(lens[6], torch.float32)
        self.inv_dout64 = new(lens[7], torch.float64)
        self.info = new(lens[8], i64)
        self.info.zero_()
        self.perm = new(lens[9], i32)
        self.iperm = new(lens[10], i32)
        self.c = CGraph(scale, 0, M, self.colptr.data_ptr(), self.rowc.data_ptr(), self.ovf_key.data_ptr(),
                        self.ovf_cnt.data_ptr(), self.d_in.data_ptr(), self.d_out.data_ptr(),
                        self.inv_dout32.data_ptr(), self.inv_dout64.data_ptr(), self.info.data_ptr(),
                        self.perm.data_ptr(), self.iperm.data_ptr())

    def info_dict(self):
        v = self.info.cpu().tolist()
        return {k: int(v[i]) for k, i in INFO.items()}


def sort_edges(u, v, scale, out=None, workspace=None, stream=None):
    """Kernel 1: (u_out, v_out) sorted by (u, v)."""
    M = u.numel()
    dev = u.device
    if out is None:
        out = (torch.empty_like(u), torch.empty_like(v))
    need = workspace_bytes("sort", M, scale)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    st = _lib().pp_sort_edges(_ptr(u), _ptr(v), M, scale, _ptr(out[0]), _ptr(out[1]), _ptr(ws), ws.numel(),
                              _stream(stream, dev))
    _check("pp_sort_edges", st)
    return out


def build_filter_normalize(us, vs, scale, rule="lowest", graph=None, workspace=None, stream=None):
    """Kernel 2: the filtered, normalised matrix as a Graph."""
    M = us.numel()
    dev = us.device
    g = graph if graph is not None else Graph(M, scale, dev)
    need = workspace_bytes("build", M, scale)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    st = _lib().pp_build_filter_normalize(_ptr(us), _ptr(vs), M, scale, RULES[rule], ctypes.byref(g.c), _ptr(ws),
                                          ws.numel(), _stream(stream, dev))
    _check("pp_build_filter_normalize", st)
    return g


def export_csr(graph, cap=None, values=True, workspace=None, stream=None):
    """Kernel 2's filtered A in compressed rows, vertex order (pp_export_csr):
    (rowptr int64[N+1], col int32[cap], cnt int32[cap], val64 float64[cap],
    val32 float32[cap]); the first rowptr[N] entries are valid.  The value
    arrays are None with values=False."""
    dev = graph.colptr.device
    cap = graph.M if cap is None else int(cap)
    rowptr = torch.empty(graph.N + 1, dtype=torch.int64, device=dev)
    col = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    cnt = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    v64 = torch.empty(max(cap, 1), dtype=torch.float64, device=dev) if values else None
    v32 = torch.empty(max(cap, 1), dtype=torch.float32, device=dev) if values else None
    need = ctypes.c_size_t(0)
    _check("pp_export_csr_workspace", _lib().pp_export_csr_workspace(graph.M, graph.scale, ctypes.byref(need)))
    ws = workspace if workspace is not None and workspace.numel() >= need.value else _workspace(need.value, dev)
    st = _lib().pp_export_csr(ctypes.byref(graph.c), _ptr(rowptr), _ptr(col), _ptr(cnt), _ptr(v64), _ptr(v32), cap,
                              _ptr(ws), ws.numel(), _stream(stream, dev))
    _check("pp_export_csr", st)
    return rowptr, col, cnt, v64, v32


def pagerank(graph, r0, iters=20, c=0.85, dtype="fp32", out=None, want_l1=False, workspace=None, stream=None):
    """Kernel 3: r after `iters` iterations (float64 for fp64, float32 otherwise)."""
    dev = r0.device
    if out is None:
        out = torch.empty(graph.N, dtype=torch.float64 if dtype == "fp64" else torch.float32, device=dev)
    l1 = torch.empty(graph.N, dtype=torch.float64, device=dev) if want_l1 else None
    need = workspace_bytes("pagerank", graph.M, graph.scale, iters, dtype)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    st = _lib().pp_pagerank(ctypes.byref(graph.c), _ptr(r0), iters, c, DTYPES[dtype], _ptr(out), _ptr(l1), _ptr(ws),
                            ws.numel(), _stream(stream, dev))
    _check("pp_pagerank", st)
    return (out, l1) if want_l1 else out


def gather_probe(graph, x, out, n=None, stream=None):
    """Gathers x at the row positions of the graph's first n packed entries
    (pp_gather_probe, a measurement aid); adds their sum to out[0]."""
    n = graph.info_dict()["nnz"] if n is None else n
    _check("pp_gather_probe", _lib().pp_gather_probe(_ptr(graph.rowc), n, graph.scale, _ptr(x), _ptr(out),
                                                     _stream(stream, x.device)))
    return out


BATCH_MAX_GRAPHS, BATCH_MAX_RHS = 128, 32


def range_counts(us, bounds, stream=None):
    """Edges of the sorted list us whose start vertex lies in each
    [bounds[p], bounds[p+1]) (pp_range_counts); int64 device tensor."""
    parts = bounds.numel() - 1
    counts = torch.empty(parts, dtype=torch.int64, device=us.device)
    _check("pp_range_counts", _lib().pp_range_counts(_ptr(us), us.numel(), _ptr(bounds), parts, _ptr(counts),
                                                     _stream(stream, us.device)))
    return counts


def in_degree(vs, scale, out=None, stream=None):
    """In-degree of an edge list, int32[2^scale] (pp_in_degree)."""
    out = out if out is not None else torch.empty(1 << scale, dtype=torch.int32, device=vs.device)
    _check("pp_in_degree", _lib().pp_in_degree(_ptr(vs), vs.numel(), scale, _ptr(out), _stream(stream, vs.device)))
    return out


def build_filter_normalize_rows(us, vs, scale, d_in_all, rule="lowest", graph=None, workspace=None, stream=None):
    """Kernel 2 on a share of a graph's rows with the in-degree of every
    column supplied (pp_build_filter_normalize_rows)."""
    M = us.numel()
    dev = us.device
    g = graph if graph is not None else Graph(M, scale, dev)
    need = workspace_bytes("build", M, scale)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    st = _lib().pp_build_filter_normalize_rows(_ptr(us), _ptr(vs), M, scale, RULES[rule], _ptr(d_in_all),
                                               ctypes.byref(g.c), _ptr(ws), ws.numel(), _stream(stream, dev))
    _check("pp_build_filter_normalize_rows", st)
    return g


def rank_update(y, a, b, r, workspace=None, stream=None):
    """r = a * y + b elementwise (pp_rank_update, binary64 or binary32 by
    dtype); returns sum(r) as a float64 device tensor of one element."""
    dt = {torch.float64: 0, torch.float32: 1}[y.dtype]
    out = torch.empty(1, dtype=torch.float64, device=y.device)
    ws = workspace if workspace is not None and workspace.numel() >= 2048 else _workspace(2048, y.device)
    _check("pp_rank_update", _lib().pp_rank_update(_ptr(y), y.numel(), float(a), float(b), _ptr(r), _ptr(out), dt,
                                                   _ptr(ws), ws.numel(), _stream(stream, y.device)))
    return out


def _ptr_array(tensors):
    return (ctypes.c_void_p * len(tensors))(*[t.data_ptr() if t is not None else 0 for t in tensors])


def sort_edges_batched(us, vs, scales, outs=None, workspace=None, stream=None):
    """Kernel 1 for a batch of graphs (pp_sort_edges_batched): one sort of all
    their edges; returns [(u_out, v_out)] per graph."""
    n = len(us)
    dev = us[0].device
    if outs is None:
        outs = [(torch.empty_like(u), torch.empty_like(v)) for u, v in zip(us, vs)]
    M = (ctypes.c_uint64 * n)(*[u.numel() for u in us])
    S = (ctypes.c_uint32 * n)(*scales)
    need = ctypes.c_size_t(0)
    _check("pp_sort_edges_batched_workspace", _lib().pp_sort_edges_batched_workspace(n, M, S, ctypes.byref(need)))
    ws = workspace if workspace is not None and workspace.numel() >= need.value else _workspace(need.value, dev)
    st = _lib().pp_sort_edges_batched(n, _ptr_array(us), _ptr_array(vs), M, S, _ptr_array([o[0] for o in outs]),
                                      _ptr_array([o[1] for o in outs]), _ptr(ws), ws.numel(), _stream(stream, dev))
    _check("pp_sort_edges_batched", st)
    return outs


def build_filter_normalize_batched(sorted_edges, scales, rule="lowest", graphs=None, workspace=None, stream=None):
    """Kernel 2 for a batch of graphs (pp_build_filter_normalize_batched);
    sorted_edges: [(us, vs)] per graph; returns a Graph per graph."""
    n = len(sorted_edges)
    dev = sorted_edges[0][0].device
    if graphs is None:
        graphs = [Graph(u.numel(), s, dev) for (u, _), s in zip(sorted_edges, scales)]
    arr = (CGraph * n)(*[g.c for g in graphs])
    M = (ctypes.c_uint64 * n)(*[g.M for g in graphs])
    S = (ctypes.c_uint32 * n)(*[g.scale for g in graphs])
    need = ctypes.c_size_t(0)
    _check("pp_build_filter_normalize_batched_workspace",
           _lib().pp_build_filter_normalize_batched_workspace(n, M, S, ctypes.byref(need)))
    ws = workspace if workspace is not None and workspace.numel() >= need.value else _workspace(need.value, dev)
    st = _lib().pp_build_filter_normalize_batched(n, _ptr_array([e[0] for e in sorted_edges]),
                                                  _ptr_array([e[1] for e in sorted_edges]), RULES[rule], arr,
                                                  _ptr(ws), ws.numel(), _stream(stream, dev))
    _check("pp_build_filter_normalize_batched", st)
    return graphs


class BatchedPipelineExec:
    """Kernels 1-3 for a batch of graphs recorded as one CUDA graph
    (pp_pipeline_batched_capture); launch() replays the whole pipeline."""

    def __init__(self, us, vs, scales, r0, nrhs, iters=20, c=0.85, rule="lowest", stream=None):
        n = len(us)
        dev = us[0].device
        self.sorted = [(torch.empty_like(u), torch.empty_like(v)) for u, v in zip(us, vs)]
        self.graphs = [Graph(u.numel(), s, dev) for u, s in zip(us, scales)]
        self._arr = (CGraph * n)(*[g.c for g in self.graphs])
        rows = sum(g.N for g in self.graphs)
        assert r0.shape == (rows, nrhs) and r0.dtype == torch.float64 and r0.is_contiguous()
        self.out = torch.empty(rows, nrhs, dtype=torch.float32, device=dev)
        need = ctypes.c_size_t(0)
        _check("pp_pipeline_batched_workspace",
               _lib().pp_pipeline_batched_workspace(n, self._arr, nrhs, iters, ctypes.byref(need)))
        self.ws = _workspace(need.value, dev)
        self._keep = (list(us), list(vs), r0)
        self._dev = dev
        h = ctypes.c_void_p(None)
        _check("pp_pipeline_batched_capture",
               _lib().pp_pipeline_batched_capture(n, _ptr_array(us), _ptr_array(vs),
                                                  _ptr_array([o[0] for o in self.sorted]),
                                                  _ptr_array([o[1] for o in self.sorted]), RULES[rule], self._arr,
                                                  _ptr(r0), nrhs, iters, c, _ptr(self.out), _ptr(self.ws),
                                                  self.ws.numel(), _stream(stream, dev), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check("pp_exec_launch", _lib().pp_exec_launch(self._h, _stream(stream, self._dev)))
        return self.out

    def close(self):
        if self._h is not None and self._h.value:
            _lib().pp_exec_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TSV_MAX_LINE = 22


def format_tsv(u, v, out=None, stream=None):
    """The edge-file text of (u, v) ("u\\tv\\n" per edge), formatted on the device.
    Returns (text uint8 tensor with room for M * TSV_MAX_LINE bytes, length as a
    device int64 tensor)."""
    M = u.numel()
    dev = u.device
    if out is None:
        out = torch.empty(max(1, M * TSV_MAX_LINE), dtype=torch.uint8, device=dev)
    n = torch.zeros(1, dtype=torch.int64, device=dev)
    need = ctypes.c_size_t(0)
    _check("pp_format_tsv_workspace", _lib().pp_format_tsv_workspace(M, ctypes.byref(need)))
    ws = _workspace(need.value, dev)
    st = _lib().pp_format_tsv(_ptr(u), _ptr(v), M, _ptr(out), out.numel(), _ptr(n), _ptr(ws), ws.numel(),
                              _stream(stream, dev))
    _check("pp_format_tsv", st)
    return out, n


def parse_tsv(text, length, m_cap, out=None, stream=None):
    """Edges (u, v) from edge-file text (device uint8 tensor, `length` bytes);
    returns (u, v, number of lines as a device int64 tensor).  Malformed text
    sets PP_DEV_PARSE (see last_device_error)."""
    dev = text.device
    if out is None:
        out = (torch.empty(max(1, m_cap), dtype=torch.int32, device=dev),
               torch.empty(max(1, m_cap), dtype=torch.int32, device=dev))
    m = torch.zeros(1, dtype=torch.int64, device=dev)
    need = ctypes.c_size_t(0)
    _check("pp_parse_tsv_workspace", _lib().pp_parse_tsv_workspace(length, ctypes.byref(need)))
    ws = _workspace(need.value, dev)
    st = _lib().pp_parse_tsv(_ptr(text), length, _ptr(out[0]), _ptr(out[1]), m_cap, _ptr(m), _ptr(ws), ws.numel(),
                             _stream(stream, dev))
    _check("pp_parse_tsv", st)
    return out[0], out[1], m


K3_DANGLING = 1
K3_CONVERGE = 2


def pagerank_ex(graph, r0, iters=20, c=0.85, dtype="fp32", dangling=False, tol=0.0, out=None, want_l1=False,
                workspace=None, stream=None):
    """Kernel 3 variants (pp_pagerank_ex): the dangling-node term and/or the
    convergence test norm(r_k - r_(k-1), 1) < tol.  Returns (r, iterations
    run as a device uint32 tensor[, r / norm(r,1)])."""
    dev = r0.device
    if out is None:
        out = torch.empty(graph.N, dtype=torch.float64 if dtype == "fp64" else torch.float32, device=dev)
    l1 = torch.empty(graph.N, dtype=torch.float64, device=dev) if want_l1 else None
    done = torch.zeros(1, dtype=torch.int32, device=dev)
    flags = (K3_DANGLING if dangling else 0) | (K3_CONVERGE if tol > 0 else 0)
    need = workspace_bytes("pagerank_ex", graph.M, graph.scale, iters, dtype)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, dev)
    st = _lib().pp_pagerank_ex(ctypes.byref(graph.c), _ptr(r0), iters, c, DTYPES[dtype], flags, float(tol),
                               _ptr(out), _ptr(l1), _ptr(done), _ptr(ws), ws.numel(), _stream(stream, dev))
    _check("pp_pagerank_ex", st)
    return (out, done, l1) if want_l1 else (out, done)


def pagerank_batched(graphs, r0, nrhs, iters=20, c=0.85, out=None, workspace=None, stream=None):
    """Kernel 3 for several graphs and nrhs start vectors each (binary32 ranks).

    r0: device float64 tensor of shape (sum of N_g, nrhs), the graphs' rows
    one after another; returns a float32 tensor of the same shape."""
    n = len(graphs)
    arr = (CGraph * n)(*[g.c for g in graphs])
    rows = sum(g.N for g in graphs)
    assert r0.shape == (rows, nrhs) and r0.dtype == torch.float64 and r0.is_contiguous()
    dev = r0.device
    if out is None:
        out = torch.empty(rows, nrhs, dtype=torch.float32, device=dev)
    need = ctypes.c_size_t(0)
    _check("pp_pagerank_batched_workspace", _lib().pp_pagerank_batched_workspace(arr, n, nrhs, iters,
                                                                               ctypes.byref(need)))
    ws = workspace if workspace is not None and workspace.numel() >= need.value else _workspace(need.value, dev)
    st = _lib().pp_pagerank_batched(arr, n, _ptr(r0), nrhs, iters, c, _ptr(out), _ptr(ws), ws.numel(),
                                    _stream(stream, dev))
    _check("pp_pagerank_batched", st)
    return out


class BatchedExec:
    """Batched Kernel 3 captured as one CUDA graph (pp_pagerank_batched_capture).

    launch() replays the stage; it reads r0 and writes out as they are at
    launch time.  Keeps references to every buffer it was captured with."""

    def __init__(self, graphs, r0, nrhs, iters=20, c=0.85, out=None, workspace=None, stream=None):
        n = len(graphs)
        self._arr = (CGraph * n)(*[g.c for g in graphs])
        rows = sum(g.N for g in graphs)
        assert r0.shape == (rows, nrhs) and r0.dtype == torch.float64 and r0.is_contiguous()
        dev = r0.device
        self.out = out if out is not None else torch.empty(rows, nrhs, dtype=torch.float32, device=dev)
        need = ctypes.c_size_t(0)
        _check("pp_pagerank_batched_workspace",
               _lib().pp_pagerank_batched_workspace(self._arr, n, nrhs, iters, ctypes.byref(need)))
        self.ws = workspace if workspace is not None and workspace.numel() >= need.value else _workspace(need.value,
                                                                                                      dev)
        self._keep = (list(graphs), r0)
        self._dev = dev
        h = ctypes.c_void_p(None)
        _check("pp_pagerank_batched_capture",
               _lib().pp_pagerank_batched_capture(self._arr, n, _ptr(r0), nrhs, iters, c, _ptr(self.out),
                                                  _ptr(self.ws), self.ws.numel(), _stream(stream, dev),
                                                  ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check("pp_exec_launch", _lib().pp_exec_launch(self._h, _stream(stream, self._dev)))
        return self.out

    def close(self):
        if self._h is not None and self._h.value:
            _lib().pp_exec_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pipeline_host(u, v, scale, r0, iters=20, c=0.85, dtype="fp32", rule="lowest", out=None, info=None,
                  workspace=None, stream=None, device="cuda"):
    """Kernels 1-3 from host tensors (pin them for asynchronous copies); returns (r, info)."""
    M = u.numel()
    N = 1 << scale
    if out is None:
        out = torch.empty(N, dtype=torch.float64 if dtype == "fp64" else torch.float32).pin_memory()
    if info is None:
        info = torch.zeros(INFO_LEN, dtype=torch.int64).pin_memory()
    need = workspace_bytes("pipeline", M, scale, iters, dtype)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, device)
    st = _lib().pp_pipeline_host(_ptr(u), _ptr(v), M, scale, _ptr(r0), iters, c, DTYPES[dtype], RULES[rule],
                                 _ptr(out), _ptr(info), _ptr(ws), ws.numel(), _stream(stream, ws.device))
    _check("pp_pipeline_host", st)
    return out, info


# ------------------------------------------------------------------ tracing
# CUDA events around each call of the kernels' entry points while a trace is
# open: trace() records, per call, the device time between an event recorded
# on the call's stream before it and one after it (the NVTX ranges of the
# library name the same calls for external profilers).
_TRACE = None
_TRACED = ("sort_edges", "build_filter_normalize", "pagerank", "pagerank_ex", "export_csr", "sort_edges_batched",
           "build_filter_normalize_batched", "pagerank_batched", "pipeline_host", "format_tsv", "parse_tsv",
           "build_filter_normalize_rows", "rank_update", "range_counts", "in_degree")


class Trace:
    """The calls recorded by `with trace() as t:`; t.report() (after the
    block) synchronises and lists (call, device ms) in call order."""

    def __init__(self):
        self.calls = []

    def report(self):
        if self.calls:
            torch.cuda.synchronize()
        return [(name, a.elapsed_time(b)) for name, a, b in self.calls]

    def totals(self):
        out = {}
        for name, ms in self.report():
            n, t = out.get(name, (0, 0.0))
            out[name] = (n + 1, t + ms)
        return out


class trace:
    def __enter__(self):
        global _TRACE
        self.prev, _TRACE = _TRACE, Trace()
        return _TRACE

    def __exit__(self, *exc):
        global _TRACE
        _TRACE = self.prev
        return False


def _traced(fn):
    import functools
    import inspect

    sig = inspect.signature(fn)

    @functools.wraps(fn)
    def wrapper(*args, **kwargs):
        if _TRACE is None:
            return fn(*args, **kwargs)
        stream = sig.bind_partial(*args, **kwargs).arguments.get("stream") or torch.cuda.current_stream()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        result = fn(*args, **kwargs)
        b.record(stream)
        _TRACE.calls.append((fn.__name__, a, b))
        return result

    return wrapper


for _name in _TRACED:
    globals()[_name] = _traced(globals()[_name])
del _name
