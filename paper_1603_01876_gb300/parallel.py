"""Kernels 1-3 in the paper's row-decomposed parallel form (Sec. IV-B to
IV-D): every rank owns a contiguous range of vertices, the rows of A with
those start vertices and the ranks r of those vertices.

    Kernel 1  each rank sorts its share of the edge list, the edges move to
              the rank owning their start vertex (an all-to-all by start
              vertex range), and each rank sorts what it received: the
              ranks' lists, one after the other, are the sorted edge list.
    Kernel 2  each rank counts the in-degree of its edges; the counts are
              added over the ranks (the in-degree is a column sum, and
              columns span every rank), and each rank builds its own rows of
              the filtered, normalised A with that global in-degree deciding
              the supernode and leaf columns.
    Kernel 3  r is normalised by its L1 norm added over the ranks; each
              iteration every rank takes the column sums of its own rows,
              sum_u r(u) A(u,v) for every column v, these are added over the
              ranks, and each rank updates its own ranks r(v) = c * y(v) +
              ((1-c)/N) * sum(r), sum(r) added over the ranks in binary64.

Collectives: one all-to-all (Kernel 1), one sum of an N-vector (Kernel 2),
one sum of an N-vector and one of a scalar per iteration (Kernel 3); NCCL
for device tensors, gloo for host ones.  The local steps go through an
`ops` object; RowOps runs them in libpp's kernels on this rank's GPU.
Kernel 3 runs in binary64.
"""
import torch

import paper_1603_01876_gb300 as pp


def row_bounds(N, parts):
    """The first vertex of every rank's range, and N: [b_0 = 0, ..., b_parts = N]."""
    return [p * N // parts for p in range(parts + 1)]


class Comm:
    """The collectives of the row-decomposed form over a torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist

        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def exchange_counts(self, send):
        """send[q] = items for rank q; returns recv[q] = items from rank q (tensors on the same device)."""
        recv = torch.empty_like(send)
        self.dist.all_to_all_single(recv, send, group=self.group)
        return recv

    def all_to_all(self, x, send, recv):
        out = torch.empty(int(sum(recv)), dtype=x.dtype, device=x.device)
        self.dist.all_to_all_single(out, x, output_split_sizes=[int(c) for c in recv],
                                    input_split_sizes=[int(c) for c in send], group=self.group)
        return out

    def sum(self, x):
        self.dist.all_reduce(x, group=self.group)
        return x


class SingleComm:
    """One rank: every collective is the identity."""

    rank, size = 0, 1

    def exchange_counts(self, send):
        return send.clone()

    def all_to_all(self, x, send, recv):
        return x

    def sum(self, x):
        return x


class RowOps:
    """The local steps in libpp's kernels on this rank's GPU."""

    def __init__(self, scale, device):
        self.scale, self.N, self.device = scale, 1 << scale, device
        self.ws = torch.empty(4096, dtype=torch.uint8, device=device)

    def sort(self, u, v):
        return pp.sort_edges(u, v, self.scale)

    def range_counts(self, us, bounds):
        return pp.range_counts(us, torch.tensor(bounds, dtype=torch.int32, device=self.device))

    def in_degree(self, vs):
        return pp.in_degree(vs, self.scale)

    def build_rows(self, us, vs, d_in_all, rule):
        return pp.build_filter_normalize_rows(us, vs, self.scale, d_in_all, rule)

    def zeros(self, n):
        return torch.zeros(n, dtype=torch.float64, device=self.device)

    def scalar(self, x):
        return torch.tensor([float(x)], dtype=torch.float64, device=self.device)

    def update(self, y, a, b, r):
        """r = a * y + b (elementwise, binary64); returns sum(r) as a 1-element tensor."""
        return pp.rank_update(y, a, b, r, workspace=self.ws)

    def column_sums(self, g, r_full, r_local_sum):
        """y(v) = sum over this rank's rows u of r(u) A(u,v), every column v."""
        y = pp.pagerank(g, r_full, 1, 1.0, "fp64")  # Kernel 3 on r / norm(r, 1) of this rank's rows
        self.update(y, float(r_local_sum), 0.0, y)
        return y


def pipeline(ops, comm, u, v, scale, r0, iters=20, c=0.85, rule="lowest"):
    """The row-decomposed Kernels 1-3 on this rank.  u, v: this rank's share
    of the edge list (any share); r0: the start values of this rank's
    vertices (binary64).  Returns (us, vs, graph, d_in, r): this rank's
    sorted edges (the rows it owns), its rows of A, the global in-degree and
    its ranks after `iters` iterations."""
    N = 1 << scale
    bounds = row_bounds(N, comm.size)
    lo, hi = bounds[comm.rank], bounds[comm.rank + 1]
    # Kernel 1
    us, vs = ops.sort(u, v)
    send = ops.range_counts(us, bounds)
    recv = comm.exchange_counts(send)
    send_l, recv_l = send.tolist(), recv.tolist()
    us, vs = ops.sort(comm.all_to_all(us, send_l, recv_l), comm.all_to_all(vs, send_l, recv_l))
    # Kernel 2
    d_in = comm.sum(ops.in_degree(vs))
    g = ops.build_rows(us, vs, d_in, rule)
    # Kernel 3: r of every vertex of this rank, the other entries of r_full 0
    r_full = ops.zeros(N)
    mine = r_full[lo:hi]
    s = comm.sum(ops.update(r0, 1.0, 0.0, mine))
    s_local = ops.update(mine, 1.0 / float(s.item()), 0.0, mine)
    for _ in range(iters):
        total = comm.sum(s_local.clone())
        y = comm.sum(ops.column_sums(g, r_full, float(s_local.item())))
        s_local = ops.update(y[lo:hi], c, (1.0 - c) / N * float(total.item()), mine)
    return us, vs, g, d_in, mine.clone()
