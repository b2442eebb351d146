"""In-tree build of the KFBI CUDA library (libkfbim.so) for sm_103a.

Two translation units compiled in parallel: the host setup (g++, FP
contraction off so that every discrete choice of the setup is reproducible
across x86 and Arm hosts) and the CUDA solver (nvcc), linked by nvcc.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libkfbim.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC))


def build(force=False, verbose=False):
    """Compile libkfbim.so if any source is newer than it; return its path."""
    os.makedirs(OUT, exist_ok=True)
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        inc = os.path.join(os.path.dirname(HERE), "include", "kfbim.h")
        if all(os.path.getmtime(s) <= t for s in sources() + [inc]):
            return LIB
    nvcc = _nvcc()
    inc = "-I" + os.path.join(os.path.dirname(HERE), "include")
    o_setup = os.path.join(OUT, "setup.o")
    o_cu = os.path.join(OUT, "kfbim.o")
    cmds = [
        ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", inc, "-c",
         os.path.join(SRC, "setup.cpp"), "-o", o_setup],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", inc,
         "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(SRC, "kfbim.cu"), "-o", o_cu],
    ]
    with ThreadPoolExecutor(2) as ex:
        logs = list(ex.map(_run, cmds))
    logs.append(_run([nvcc, ARCH, "-shared", o_setup, o_cu, "-o", LIB + ".tmp", "-lcudart"]))
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
