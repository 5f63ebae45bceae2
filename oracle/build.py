"""Build the C oracle (test infrastructure only) into oracle/_build/liboracle.so.

The oracle is compiled with contraction off and no fast-math, so each C
operator is one IEEE-754 operation rounded to nearest (the paper's Section 1
assumption).  On x86-64 the binary128 reference links libquadmath; on
AArch64 `long double` is binary128 and libm provides sqrtl/powl.
"""
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nrm_oracle.c")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")

CFLAGS = ["-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fno-finite-math-only",
          "-frounding-math", "-fPIC", "-shared", "-Wall", "-Wno-unused-function"]


def build(force=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    libs = ["-lm", "-lpthread"]
    if platform.machine() in ("x86_64", "AMD64"):
        libs.insert(0, "-lquadmath")
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + [SRC, "-o", tmp] + libs
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
