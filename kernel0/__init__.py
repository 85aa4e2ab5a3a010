"""Seeded synthetic inputs for the PageRank pipeline (Kernel 0, Sec. IV-A).

This module is shared by the CPU oracle's tests and the GPU path, and holds
none of the arithmetic of Kernels 1-3.  It makes

* Kronecker edge lists of the Graph500 shape: scale S, N = 2^S vertices,
  M = 16 N edges (edge factor k = 16), initiator probabilities
  A/B/C/D = 0.57/0.19/0.19/0.05, one 32-bit Philox4x32-10 draw per edge and
  bit level, then one seeded bijective relabel of [0, N) applied to both
  endpoints.  Duplicate edges, self-loops, empty rows/columns and a heavy
  in/out-degree tail all occur, as the paper expects (Sec. IV-C);
* the start vector r = rand(1,N) of Kernel 3 (Sec. IV-D): uniform (0, 1)
  binary64 values from the same counter-based generator.

The host and device generators run the same integer code and agree bit for
bit (checked by the tests), so a GPU run and an oracle run see the same graph.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkernel0.so")

#: Graph500 initiator probabilities (A, B, C, D).
INITIATOR = (0.57, 0.19, 0.19, 0.05)
#: Average number of edges per vertex, k (Sec. IV-A).
EDGE_FACTOR = 16


class Params(ctypes.Structure):
    _fields_ = [
        ("key0", ctypes.c_uint32), ("key1", ctypes.c_uint32), ("graph", ctypes.c_uint32),
        ("scale", ctypes.c_uint32), ("t_a", ctypes.c_uint32), ("t_ab", ctypes.c_uint32),
        ("t_abc", ctypes.c_uint32), ("mul", ctypes.c_uint32 * 3), ("add", ctypes.c_uint32 * 3),
        ("shift", ctypes.c_uint32),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            from . import build as _b
            _b.build()
        L = ctypes.CDLL(LIB_PATH)
        L.k0_params_init.argtypes = [ctypes.POINTER(Params), ctypes.c_uint32, ctypes.c_uint64,
                                     ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double]
        L.k0_gen_edges_host.argtypes = [ctypes.POINTER(Params), ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        L.k0_gen_edges_device.argtypes = [ctypes.POINTER(Params), ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.k0_gen_r0_host.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                     ctypes.c_uint64, ctypes.c_void_p, ctypes.c_int]
        L.k0_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.k0_relabel_host.argtypes = [ctypes.POINTER(Params), ctypes.c_void_p, ctypes.c_uint64]
        for f in (L.k0_params_init, L.k0_gen_edges_host, L.k0_gen_edges_device, L.k0_gen_r0_host,
                  L.k0_philox, L.k0_relabel_host):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


def params(scale, seed, graph=0, initiator=INITIATOR):
    p = Params()
    rc = lib().k0_params_init(ctypes.byref(p), scale, seed, graph, *initiator)
    if rc != 0:
        raise ValueError("bad Kronecker parameters: scale=%r graph=%r initiator=%r" % (scale, graph, initiator))
    return p


def num_edges(scale, edge_factor=EDGE_FACTOR):
    return edge_factor << scale


def edges_host(scale, seed, graph=0, M=None, edge_factor=EDGE_FACTOR, e0=0, threads=0,
               initiator=INITIATOR):
    """Edges e0 .. e0+M-1 as two host uint32 arrays (u, v)."""
    if M is None:
        M = num_edges(scale, edge_factor)
    p = params(scale, seed, graph, initiator)
    u = np.empty(M, dtype=np.uint32)
    v = np.empty(M, dtype=np.uint32)
    rc = lib().k0_gen_edges_host(ctypes.byref(p), e0, M, u.ctypes.data, v.ctypes.data, threads)
    if rc != 0:
        raise RuntimeError("k0_gen_edges_host failed: %d" % rc)
    return u, v


def edges_device(scale, seed, graph=0, M=None, edge_factor=EDGE_FACTOR, e0=0, device="cuda",
                 initiator=INITIATOR, out=None):
    """The same edges generated on the GPU, as two torch.int32 tensors holding uint32 bits."""
    import torch

    if M is None:
        M = num_edges(scale, edge_factor)
    p = params(scale, seed, graph, initiator)
    if out is None:
        u = torch.empty(M, dtype=torch.int32, device=device)
        v = torch.empty(M, dtype=torch.int32, device=device)
    else:
        u, v = out
    stream = torch.cuda.current_stream(u.device).cuda_stream
    rc = lib().k0_gen_edges_device(ctypes.byref(p), e0, M, u.data_ptr(), v.data_ptr(), stream)
    if rc != 0:
        raise RuntimeError("k0_gen_edges_device failed: %d" % rc)
    return u, v


def r0_host(n, seed, graph=0, rhs=0, threads=0):
    """Start vector rand(1,n): binary64 uniform in (0, 1)."""
    out = np.empty(n, dtype=np.float64)
    rc = lib().k0_gen_r0_host(seed, graph, rhs, n, out.ctypes.data, threads)
    if rc != 0:
        raise RuntimeError("k0_gen_r0_host failed: %d" % rc)
    return out


def batch_scales(n_graphs, lo, hi, seed):
    """Scales of a batch of graphs drawn uniformly from lo..hi (inclusive)."""
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.integers(lo, hi + 1, size=n_graphs)]


def philox(ctr, key):
    """One Philox4x32-10 block (test hook)."""
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().k0_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def relabel(p, x):
    """The relabel bijection of graph parameters p applied to the ids x (test hook)."""
    x = np.array(x, dtype=np.uint32)
    lib().k0_relabel_host(ctypes.byref(p), x.ctypes.data, len(x))
    return x
