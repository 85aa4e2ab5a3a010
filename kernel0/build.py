"""Build libkernel0.so (host + sm_103a device input generator) in place."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "libkernel0.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r


def build(force=False):
    srcs = [os.path.join(HERE, "csrc", f) for f in ("k0_host.c", "k0_device.cu")]
    deps = srcs + [os.path.join(HERE, "csrc", "k0_core.h"), os.path.join(ROOT, "include", "kernel0.h")]
    if not force and os.path.exists(OUT):
        t = os.path.getmtime(OUT)
        if all(os.path.getmtime(d) <= t for d in deps):
            return OUT
    bdir = os.path.join(HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    objs = [os.path.join(bdir, "k0_host.o"), os.path.join(bdir, "k0_device.o")]
    cmds = [
        ["gcc", "-O2", "-fPIC", "-std=c11", "-Wall", "-c", srcs[0], "-o", objs[0]],
        [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-c", srcs[1], "-o", objs[1]],
    ]
    with ThreadPoolExecutor(len(cmds)) as ex:
        list(ex.map(_run, cmds))
    tmp = OUT + ".tmp.%d" % os.getpid()
    _run([NVCC, *ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
          *objs, "-lpthread", "-o", tmp])
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
