"""A host stand-in for the local steps of the row-decomposed form
(paper_1603_01876_gb300.parallel.RowOps), used only by the two-rank CPU test
of the orchestration: each step written out directly in numpy from its
definition (Sec. IV-B to IV-D)."""
import numpy as np
import torch


def _u32(t):
    return t.numpy().view(np.uint32)


def _t32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32))


class NumpyRowOps:
    def __init__(self, scale):
        self.scale, self.N = scale, 1 << scale

    def sort(self, u, v):
        u, v = _u32(u), _u32(v)
        o = np.lexsort((v, u))
        return _t32(u[o]), _t32(v[o])

    def range_counts(self, us, bounds):
        u = _u32(us)
        b = np.asarray(bounds, dtype=np.int64)
        return torch.from_numpy(np.diff(np.searchsorted(u, b, side="left")).astype(np.int64))

    def in_degree(self, vs):
        return torch.from_numpy(np.bincount(_u32(vs), minlength=self.N).astype(np.int32))

    def build_rows(self, us, vs, d_in_all, rule):
        u, v = _u32(us).astype(np.int64), _u32(vs).astype(np.int64)
        d_in = d_in_all.numpy().astype(np.int64)
        dmax = int(d_in.max())
        kill = d_in == 1
        if rule == "lowest":
            kill[int(np.argmax(d_in))] = True
        else:
            kill |= d_in == dmax
        key = u * self.N + v
        k, cnt = np.unique(key, return_counts=True)
        ku, kv = k // self.N, k % self.N
        keep = ~kill[kv]
        ku, kv, cnt = ku[keep], kv[keep], cnt[keep]
        d_out = np.bincount(ku, weights=cnt, minlength=self.N).astype(np.int64)
        return {"u": ku, "v": kv, "cnt": cnt, "d_out": d_out, "d_in": d_in}

    def zeros(self, n):
        return torch.zeros(n, dtype=torch.float64)

    def update(self, y, a, b, r):
        r.copy_(a * y + b)
        return torch.tensor([float(r.sum())], dtype=torch.float64)

    def column_sums(self, g, r_full, r_local_sum):
        r = r_full.numpy()
        y = np.zeros(self.N)
        np.add.at(y, g["v"], g["cnt"] * (r[g["u"]] / g["d_out"][g["u"]]))
        return torch.from_numpy(y)
