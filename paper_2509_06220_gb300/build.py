"""In-tree build of the CUDA library libnrm.so for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then
linked into paper_2509_06220_gb300/_build/libnrm.so.  Floating-point flags:
no fast-math, no FMA contraction (-fmad=false), IEEE division and square root,
no flush-to-zero -- every statement of the kernels is one correctly rounded
IEEE operation.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libnrm.so")
SOURCES = ["nrm_tree_d.cu", "nrm_tree_s.cu", "nrm_tree_mixed.cu", "nrm_kernels.cu", "nrm_runtime.cu", "nrm_gen.cu",
           "nrm_serve.cu", "nrm_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-prec-div=true", "-prec-sqrt=true",
                "-ftz=false", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-fast-math", "-Xptxas", "-warn-spills",
                "-I", INC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INC, "nrm.h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(src, verbose=False):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    cmd = [NVCC] + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose), srcs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
