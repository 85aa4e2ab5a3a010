"""The row-decomposed form of Kernels 1-3 (paper_1603_01876_gb300.parallel)
with its local steps in libpp's kernels on the GPU, against the oracle's
single-rank pipeline.  One GPU here: a single rank, and two ranks run as two
host threads over one stream whose collectives are done on the host between
the ranks' kernels (no kernel waits on another rank)."""
import threading

import numpy as np
import pytest

from gpu_helpers import host_u32

pytestmark = pytest.mark.gpu

SCALE, SEED, ITERS = 11, 9, 20


class ThreadComm:
    """The collectives of parallel.Comm between host threads (test stand-in)."""

    def __init__(self, rank, size, shared):
        self.rank, self.size, self.sh = rank, size, shared

    def _exchange(self, item, combine):
        self.sh["slots"][self.rank] = item
        self.sh["barrier"].wait()
        res = combine(list(self.sh["slots"]))
        self.sh["barrier"].wait()
        return res

    def exchange_counts(self, send):
        import torch

        return self._exchange(send, lambda all_: torch.stack([a[self.rank] for a in all_]))

    def all_to_all(self, x, send, recv):
        import torch

        def take(all_):
            parts = []
            for xq, sq in all_:
                off = int(sum(sq[:self.rank]))
                parts.append(xq[off:off + int(sq[self.rank])])
            return torch.cat(parts)

        return self._exchange((x, send), take)

    def sum(self, x):
        total = self._exchange(x, lambda all_: sum(a.clone() for a in all_))
        x.copy_(total)
        return x


def _run(pp, k0, parts, rule):
    import torch

    from paper_1603_01876_gb300 import parallel

    N = 1 << SCALE
    u, v = k0.edges_host(SCALE, SEED)
    M = len(u)
    r0 = k0.r0_host(N, SEED)
    bounds = parallel.row_bounds(N, parts)
    out = [None] * parts
    errors = []
    shared = {"slots": [None] * parts, "barrier": threading.Barrier(parts)}

    def rank_main(p):
        try:
            comm = parallel.SingleComm() if parts == 1 else ThreadComm(p, parts, shared)
            a, b = p * M // parts, (p + 1) * M // parts
            ud = torch.from_numpy(u[a:b].view(np.int32)).cuda()
            vd = torch.from_numpy(v[a:b].view(np.int32)).cuda()
            r0d = torch.from_numpy(r0[bounds[p]:bounds[p + 1]].copy()).cuda()
            out[p] = parallel.pipeline(parallel.RowOps(SCALE, ud.device), comm, ud, vd, SCALE, r0d, ITERS, 0.85, rule)
        except Exception as e:  # reported after the join
            errors.append(e)
            shared["barrier"].abort()

    threads = [threading.Thread(target=rank_main, args=(p,)) for p in range(parts)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    if errors:
        raise errors[0]
    torch.cuda.synchronize()
    return out, bounds


@pytest.mark.parametrize("parts,rule", [(1, "lowest"), (2, "lowest"), (2, "all_ties")])
def test_rows_on_the_gpu_equal_the_oracle(oracle_mod, k0, parts, rule):
    import paper_1603_01876_gb300 as pp

    out, bounds = _run(pp, k0, parts, rule)
    N = 1 << SCALE
    u, v = k0.edges_host(SCALE, SEED)
    ous, ovs = oracle_mod.k1_sort(u, v)
    R = oracle_mod.k2_filter(ous, ovs, N, rule)
    want = oracle_mod.k3_pagerank(R, k0.r0_host(N, SEED), ITERS, 0.85)
    assert np.array_equal(np.concatenate([host_u32(o[0]) for o in out]), ous)
    assert np.array_equal(np.concatenate([host_u32(o[1]) for o in out]), ovs)
    rowptr = R["rowptr"].astype(np.int64)
    for p, (us, vs, g, d_in, r) in enumerate(out):
        assert np.array_equal(host_u32(d_in), R["d_in"])
        lo, hi = bounds[p], bounds[p + 1]
        rp, col, cnt, val, _ = pp.export_csr(g)
        rp = rp.cpu().numpy()
        e0, e1 = rowptr[lo], rowptr[hi]
        assert np.array_equal(np.diff(rp)[lo:hi], np.diff(rowptr)[lo:hi])
        assert rp[N] == e1 - e0
        assert np.array_equal(host_u32(col)[:e1 - e0], R["col"][e0:e1])
        assert np.array_equal(host_u32(cnt)[:e1 - e0], R["cnt"][e0:e1])
        assert np.array_equal(val.cpu().numpy()[:e1 - e0].view(np.uint64), R["val"][e0:e1].view(np.uint64))
    r = np.concatenate([o[4].cpu().numpy() for o in out])
    assert np.abs(r - want).sum() / np.abs(want).sum() <= 1e-12
    assert pp.last_device_error() == 0
