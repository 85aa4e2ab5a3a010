"""Build libpp.so (the sm_103a CUDA path behind include/pagerank_pipeline.h) in place.

Each .cu file is compiled by nvcc in parallel, then linked into one shared
library next to this file.  Only -gencode arch=compute_103a,code=sm_103a is
emitted; IEEE division and square root are kept (no fast-math).

libpp_checked.so is the same sources compiled with -DPP_CHECKED: every index
a kernel reads from memory, or computes from what it read, is compared with
the length of the array it addresses; one out of range sets PP_DEV_BOUNDS in
the device error word and the access is redirected to element 0 instead of
leaving the array (no trap, the context stays usable).  It stands in for a
memory checker; the tests run the pipeline through both libraries and
require bit-identical results and a clear error word.
"""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libpp.so")
OUT_CHECKED = os.path.join(HERE, "libpp_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _fresh(out, deps):
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(d) <= t for d in deps)


def build(force=False, verbose_ptxas=False, checked=True):
    """Builds libpp.so and (checked=True) libpp_checked.so; returns libpp.so's path."""
    srcs = sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "pagerank_pipeline.h")]
    variants = [(OUT, "_build", [])] + ([(OUT_CHECKED, "_build_checked", ["-DPP_CHECKED"])] if checked else [])
    if not force and not verbose_ptxas:
        variants = [v for v in variants if not _fresh(v[0], deps)]
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs, links = [], []
    for out, sub, defs in variants:
        bdir = os.path.join(HERE, sub)
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for s in srcs:
            obj = os.path.join(bdir, os.path.basename(s)[:-3] + ".o")
            jobs.append([NVCC, *ARCH, *FLAGS, *defs, *extra, "-c", s, "-o", obj])
            objs.append(obj)
        links.append((out, objs))
    if jobs:
        with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
            logs = list(ex.map(_run, jobs))
        if verbose_ptxas:
            print("\n".join(logs))
    for out, objs in links:
        tmp = out + ".tmp.%d" % os.getpid()
        _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64", "-ldl",
              *objs, "-o", tmp])
        os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
