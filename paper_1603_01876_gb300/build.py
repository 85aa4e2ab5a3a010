"""Build libpp.so (the sm_103a CUDA path behind include/pagerank_pipeline.h) in place.

Each .cu file is compiled by nvcc in parallel, then linked into one shared
library next to this file.  Only -gencode arch=compute_103a,code=sm_103a is
emitted; IEEE division and square root are kept (no fast-math).
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


def build(force=False, verbose_ptxas=False):
    srcs = sources()
    deps = srcs + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "pagerank_pipeline.h")]
    if not force and not verbose_ptxas and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(d) <= t for d in deps):
            return OUT
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    jobs = []
    for s in srcs:
        obj = os.path.join(bdir, os.path.basename(s)[:-3] + ".o")
        jobs.append((obj, [NVCC, *ARCH, *FLAGS, *extra, "-c", s, "-o", obj]))
    with ThreadPoolExecutor(max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        logs = list(ex.map(lambda j: _run(j[1]), jobs))
    if verbose_ptxas:
        print("\n".join(logs))
    tmp = OUT + ".tmp.%d" % os.getpid()
    _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
          *[j[0] for j in jobs], "-o", tmp])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
