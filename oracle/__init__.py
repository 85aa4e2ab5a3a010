"""CPU oracle for Kernels 1-3 of the PageRank pipeline — TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg (and its
``--impl reference`` arm) may import this package.  The product path never
does.  The arithmetic lives in pp_oracle.c (plain single-threaded C, binary64);
this file only marshals numpy arrays.

Parity status of each function (what pins it is listed in tests/):
  k1_sort      pinned: brute-force sort, permutation/multiset checks.
  k2_filter    pinned: dense literal Matlab statements, hand-counted graphs,
               sum/row-sum invariants.
  k3_pagerank  pinned: dense Google-matrix power iteration, Perron eigenvector,
               closed forms (A = 0, c = 0, one hand-worked example), the
               per-iteration mass balance.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
RULES = {"lowest": 0, "all_ties": 1}


class Oracle:
    """Bindings to one build of the oracle library (the default one or a test variant)."""

    def __init__(self, path=None):
        if path is None:
            from . import build as _b
            path = _b.build()
        L = ctypes.CDLL(path)
        vp, u64, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32
        L.oracle_k1_sort.argtypes = [vp, vp, u64, vp, vp]
        L.oracle_k2_filter.argtypes = [vp, vp, u64, u32, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_k3_pagerank.argtypes = [u32, vp, vp, vp, vp, u32, ctypes.c_double, vp, vp]
        L.oracle_k3_pagerank_ex.argtypes = [u32, vp, vp, vp, vp, u32, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                            vp, vp]
        L.oracle_format_tsv.argtypes = [vp, vp, u64, vp, u64]
        L.oracle_format_tsv.restype = ctypes.c_int64
        L.oracle_parse_tsv.argtypes = [vp, u64, vp, vp, u64, vp, vp]
        for f in (L.oracle_k1_sort, L.oracle_k2_filter, L.oracle_k3_pagerank, L.oracle_k3_pagerank_ex,
                  L.oracle_parse_tsv):
            f.restype = ctypes.c_int
        self.lib = L

    def k1_sort(self, u, v):
        """Kernel 1: edges sorted by start vertex, ties by end vertex."""
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        uo = np.empty_like(u)
        vo = np.empty_like(v)
        if self.lib.oracle_k1_sort(u.ctypes.data, v.ctypes.data, len(u), uo.ctypes.data, vo.ctypes.data):
            raise MemoryError("oracle_k1_sort failed")
        return uo, vo

    def k2_filter(self, u, v, N, rule="lowest"):
        """Kernel 2: filtered, row-normalised adjacency matrix by rows (see pp_oracle.c)."""
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        M = len(u)
        cap = max(M, 1)
        rowptr = np.empty(N + 1, dtype=np.uint64)
        col = np.empty(cap, dtype=np.uint32)
        cnt = np.empty(cap, dtype=np.uint32)
        val = np.empty(cap, dtype=np.float64)
        d_in = np.empty(N, dtype=np.uint32)
        d_out = np.empty(N, dtype=np.uint32)
        stats = np.zeros(8, dtype=np.uint64)
        rc = self.lib.oracle_k2_filter(u.ctypes.data, v.ctypes.data, M, N, RULES[rule], rowptr.ctypes.data,
                                       col.ctypes.data, cnt.ctypes.data, val.ctypes.data, d_in.ctypes.data,
                                       d_out.ctypes.data, stats.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_k2_filter failed: %d" % rc)
        nnz = int(stats[1])
        return {
            "N": N, "rowptr": rowptr, "col": col[:nnz].copy(), "cnt": cnt[:nnz].copy(),
            "val": val[:nnz].copy(), "d_in": d_in, "d_out": d_out, "nnz0": int(stats[0]),
            "nnz": nnz, "dmax": int(stats[2]), "ties": int(stats[3]), "vmax": int(stats[4]),
            "supernodes": int(stats[5]),
        }

    def k3_pagerank(self, A, r0, iters=20, c=0.85, want_sums=False):
        """Kernel 3: `iters` damped iterations from r0 (normalised to unit L1 norm first)."""
        N = A["N"]
        r0 = np.ascontiguousarray(r0, dtype=np.float64)
        assert len(r0) == N
        rowptr = np.ascontiguousarray(A["rowptr"], dtype=np.uint64)
        col = np.ascontiguousarray(A["col"], dtype=np.uint32)
        val = np.ascontiguousarray(A["val"], dtype=np.float64)
        r = np.empty(N, dtype=np.float64)
        sums = np.empty(iters + 1, dtype=np.float64)
        rc = self.lib.oracle_k3_pagerank(N, rowptr.ctypes.data, col.ctypes.data if len(col) else None,
                                         val.ctypes.data if len(val) else None, r0.ctypes.data, iters, c,
                                         r.ctypes.data, sums.ctypes.data)
        if rc != 0:
            raise MemoryError("oracle_k3_pagerank failed")
        return (r, sums) if want_sums else r

    def k3_pagerank_ex(self, A, r0, iters=20, c=0.85, dangling=False, tol=0.0):
        """Kernel 3 with the dangling-node term and/or the convergence test;
        returns (r, iterations run)."""
        N = A["N"]
        r0 = np.ascontiguousarray(r0, dtype=np.float64)
        assert len(r0) == N
        rowptr = np.ascontiguousarray(A["rowptr"], dtype=np.uint64)
        col = np.ascontiguousarray(A["col"], dtype=np.uint32)
        val = np.ascontiguousarray(A["val"], dtype=np.float64)
        r = np.empty(N, dtype=np.float64)
        done = ctypes.c_uint32(0)
        rc = self.lib.oracle_k3_pagerank_ex(N, rowptr.ctypes.data, col.ctypes.data if len(col) else None,
                                            val.ctypes.data if len(val) else None, r0.ctypes.data, iters, c,
                                            1 if dangling else 0, float(tol), r.ctypes.data, ctypes.byref(done))
        if rc != 0:
            raise MemoryError("oracle_k3_pagerank_ex failed")
        return r, int(done.value)

    def format_tsv(self, u, v):
        """The edge file text of (u, v): one "u\\tv\\n" line per edge."""
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        cap = 22 * len(u)
        out = np.empty(max(cap, 1), dtype=np.uint8)
        n = self.lib.oracle_format_tsv(u.ctypes.data, v.ctypes.data, len(u), out.ctypes.data, cap)
        if n < 0:
            raise MemoryError("oracle_format_tsv failed")
        return out[:n].tobytes()

    def parse_tsv(self, text, cap=None):
        """(u, v, lines, malformed) read from edge file text."""
        buf = np.frombuffer(bytes(text), dtype=np.uint8)
        cap = len(buf) // 4 + 1 if cap is None else cap
        u = np.zeros(max(cap, 1), dtype=np.uint32)
        v = np.zeros(max(cap, 1), dtype=np.uint32)
        m = ctypes.c_uint64(0)
        bad = ctypes.c_int(0)
        self.lib.oracle_parse_tsv(buf.ctypes.data if len(buf) else None, len(buf), u.ctypes.data, v.ctypes.data, cap,
                                  ctypes.byref(m), ctypes.byref(bad))
        k = min(m.value, cap)
        return u[:k], v[:k], int(m.value), bool(bad.value)

    def pipeline(self, u, v, scale, r0, iters=20, c=0.85, rule="lowest"):
        """Kernels 1-3 in order, each finished before the next starts."""
        N = 1 << scale
        us, vs = self.k1_sort(u, v)
        A = self.k2_filter(us, vs, N, rule)
        r = self.k3_pagerank(A, r0, iters, c)
        return us, vs, A, r


_default = None


def default():
    global _default
    if _default is None:
        _default = Oracle()
    return _default


def k1_sort(u, v):
    return default().k1_sort(u, v)


def k2_filter(u, v, N, rule="lowest"):
    return default().k2_filter(u, v, N, rule)


def k3_pagerank(A, r0, iters=20, c=0.85, want_sums=False):
    return default().k3_pagerank(A, r0, iters, c, want_sums)


def k3_pagerank_ex(A, r0, iters=20, c=0.85, dangling=False, tol=0.0):
    return default().k3_pagerank_ex(A, r0, iters, c, dangling, tol)


def format_tsv(u, v):
    return default().format_tsv(u, v)


def parse_tsv(text, cap=None):
    return default().parse_tsv(text, cap)


def pipeline(u, v, scale, r0, iters=20, c=0.85, rule="lowest"):
    return default().pipeline(u, v, scale, r0, iters, c, rule)
