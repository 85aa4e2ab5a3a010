"""Helpers for the GPU parity tests: moving arrays and decoding Kernel 2's output.

The decode here is test code: it turns the GPU's compressed columns back into
(u, v, count) triples so they can be compared with the oracle's rows.
"""
import numpy as np


def dev_u32(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def host_u32(t):
    return t.cpu().numpy().view(np.uint32)


def row_buckets(u_sorted, N):
    """Kernel 2's row order key: clz(d | 1) of each row's edge count d before
    the filters (ascending key = descending floor(log2(d)))."""
    d = np.bincount(u_sorted.astype(np.int64), minlength=N).astype(np.uint64)
    return 31 - np.floor(np.log2(np.maximum(d, 1))).astype(np.int64)


def check_row_order(g, u_sorted):
    """perm / iperm are inverse permutations ordering the rows by bucket, then id."""
    N = g.N
    perm = host_u32(g.perm)[:N].astype(np.int64)
    iperm = host_u32(g.iperm)[:N].astype(np.int64)
    want = np.lexsort((np.arange(N), row_buckets(u_sorted, N)))
    assert np.array_equal(iperm, want)
    assert np.array_equal(perm[iperm], np.arange(N))


def gpu_triples(g):
    """(u, v, cnt) of the GPU's filtered A in (u, v) order, plus the CSC-order
    arrays (row positions, column positions, column pointers)."""
    info = g.info_dict()
    nnz, novf = info["nnz"], info["novf"]
    colptr = host_u32(g.colptr)[: g.N + 1].astype(np.int64)
    rowc = host_u32(g.rowc)[:nnz]
    assert colptr[0] == 0 and colptr[-1] == nnz and (np.diff(colptr) >= 0).all()
    iperm = host_u32(g.iperm)[: g.N]
    pos = rowc & np.uint32((1 << g.scale) - 1)
    u = iperm[pos]
    cf = (rowc >> np.uint32(g.scale)).astype(np.uint64)
    cpos = np.repeat(np.arange(g.N, dtype=np.uint32), np.diff(colptr))  # column positions
    v = iperm[cpos]
    cmax = (1 << (32 - g.scale)) - 1
    esc = cf == cmax
    if esc.any():
        ovk = g.ovf_key.cpu().numpy().view(np.uint64)[:novf]
        ovc = host_u32(g.ovf_cnt)[:novf]
        keys = (u[esc].astype(np.uint64) << np.uint64(32)) | v[esc].astype(np.uint64)
        idx = np.searchsorted(ovk, keys)
        assert (idx < novf).all() and (ovk[idx] == keys).all()
        cf[esc] = ovc[idx]
    order = np.lexsort((v, u))
    return u[order], v[order], cf[order], (pos, cpos, colptr)


def oracle_triples(R):
    N = R["N"]
    u = np.repeat(np.arange(N, dtype=np.uint32), np.diff(R["rowptr"].astype(np.int64)))
    return u, R["col"], R["cnt"].astype(np.uint64)


def rank_errors(got, want):
    got = np.asarray(got, dtype=np.float64)
    d = np.abs(got - want)
    nz = want != 0
    mr = float((d[nz] / np.abs(want[nz])).max()) if nz.any() else 0.0
    return {"l1": float(d.sum() / np.abs(want).sum()), "max_rel": mr, "zero_mismatch": float(d[~nz].max(initial=0))}
