"""The oracle on a whole benchmark-size graph — TEST INFRASTRUCTURE ONLY.

Only tests/ and bench.py (its accuracy report against the oracle) use this
module.  It runs the CPU oracle of pp_oracle.c (one thread, binary64) on the
full Kronecker graph of a given scale and seed, Kernels 1-3 in order, and
stores what the GPU results are compared with, keyed by (scale, seed):

  - Kernel 1: SHA-256 digests of the sorted u and v (the sort is unique, so
    equal digests mean equal arrays);
  - Kernel 2: nnz0, nnz, max(d_in), its lowest column, the tie count, the
    supernodes removed, d_in, d_out and the row pointers of the filtered A
    (arrays), and digests of its columns, counts and binary64 values;
  - Kernel 3: r after `iters` damped iterations (c = 0.85) from the seeded
    start vector, and sum(r) before each iteration;
  - the seconds each kernel took.

Every stored value comes from the oracle (nothing from the GPU path).  A
scale-24 run takes a few minutes and about 11 GB of host memory, so callers
start it in a child process early (start()) and collect it later (wait());
the result is cached in .oracle_cache/ at the repository root (ignored by
git) and reused while the oracle source is unchanged.

    python -m oracle.fullsize --scale 24 --seed 1
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CACHE_DIR = os.path.join(ROOT, ".oracle_cache")
DAMPING = 0.85
ITERS = 20


def _source_tag():
    with open(os.path.join(HERE, "pp_oracle.c"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


def digest(a):
    """SHA-256 of an array's bytes (contiguous, native little-endian)."""
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def cache_path(scale, seed, iters=ITERS, cache_dir=CACHE_DIR):
    return os.path.join(cache_dir, "oracle_s%d_seed%d_it%d_%s.npz" % (scale, seed, iters, _source_tag()))


def compute(scale, seed, iters=ITERS, out=None, log=None):
    """Runs the oracle pipeline and writes the result file; returns its path."""
    sys.path.insert(0, ROOT)
    import kernel0
    import oracle

    out = out or cache_path(scale, seed, iters)
    N = 1 << scale
    O = oracle.default()
    t = {}
    t0 = time.perf_counter()
    u, v = kernel0.edges_host(scale, seed)
    r0 = kernel0.r0_host(N, seed)
    t["gen"] = time.perf_counter() - t0
    M = len(u)
    t0 = time.perf_counter()
    us, vs = O.k1_sort(u, v)
    t["k1"] = time.perf_counter() - t0
    del u, v
    res = {"us_sha": digest(us), "vs_sha": digest(vs)}
    t0 = time.perf_counter()
    A = O.k2_filter(us, vs, N, "lowest")
    t["k2"] = time.perf_counter() - t0
    del us, vs
    res.update(col_sha=digest(A["col"]), cnt_sha=digest(A["cnt"]), val_sha=digest(A["val"]))
    t0 = time.perf_counter()
    r, sums = O.k3_pagerank(A, r0, iters, DAMPING, want_sums=True)
    t["k3"] = time.perf_counter() - t0
    meta = {"scale": scale, "seed": seed, "N": N, "M": M, "iters": iters, "c": DAMPING,
            "nnz0": A["nnz0"], "nnz": A["nnz"], "dmax": A["dmax"], "vmax": A["vmax"], "ties": A["ties"],
            "supernodes": A["supernodes"], "seconds": t, "oracle_source": _source_tag(), **res}
    os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
    tmp = out + ".tmp.%d.npz" % os.getpid()
    np.savez(tmp, meta=np.array(json.dumps(meta)), d_in=A["d_in"], d_out=A["d_out"],
             rowptr=A["rowptr"], r=r, sums=sums)
    os.replace(tmp, out)
    if log:
        log("oracle scale %d seed %d: %s" % (scale, seed, json.dumps(t)))
    return out


def load(path):
    with np.load(path) as z:
        d = {k: z[k] for k in z.files if k != "meta"}
        d.update(json.loads(str(z["meta"])))
    return d


class Pending:
    """An oracle run in a child process (or an already cached result)."""

    def __init__(self, scale, seed, iters=ITERS):
        self.path = cache_path(scale, seed, iters)
        self.proc = None
        self.log = self.path + ".log"
        if not os.path.exists(self.path):
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            with open(self.log, "w") as lf:
                # a fresh interpreter (not a fork of a process that may hold a CUDA context)
                self.proc = subprocess.Popen([sys.executable, "-m", "oracle.fullsize", "--scale", str(scale),
                                              "--seed", str(seed), "--iters", str(iters), "--out", self.path],
                                             cwd=ROOT, stdout=lf, stderr=subprocess.STDOUT)

    def wait(self, timeout=None):
        if self.proc is not None:
            rc = self.proc.wait(timeout=timeout)
            if rc != 0:
                with open(self.log) as lf:
                    raise RuntimeError("oracle run failed (rc %d): %s" % (rc, lf.read()[-2000:]))
            self.proc = None
        return load(self.path)

    def cancel(self):
        if self.proc is not None and self.proc.poll() is None:
            self.proc.kill()
            self.proc.wait()


def start(scale, seed, iters=ITERS):
    return Pending(scale, seed, iters)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)
    print(compute(args.scale, args.seed, args.iters, args.out, log=print))


if __name__ == "__main__":
    main()
