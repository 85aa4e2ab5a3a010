"""Build the CPU oracle (test infrastructure only) as oracle/liboracle.so with gcc.

Plain -O2: no -ffast-math, no vectorisation flags that could reorder
floating-point sums.  Extra -D flags can be given to build a variant into
another file (the tests use this to plant mistakes and check that the pins
catch them).
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pp_oracle.c")
OUT = os.path.join(HERE, "liboracle.so")


def build(force=False, out=OUT, defines=()):
    if not force and not defines and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-Wall", "-ffp-contract=off",
           *["-D" + d for d in defines], SRC, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
