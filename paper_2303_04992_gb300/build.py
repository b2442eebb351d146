"""In-tree build of the KFBI CUDA library (libkfbim.so) for sm_103a.

Translation units compiled in parallel: the host setup (g++, FP contraction
off so that every discrete choice of the setup is reproducible across x86 and
Arm hosts), the CUDA solver, the slab CG kernels and the four-step transform
passes of each grid size (nvcc), linked by nvcc.
"""
import hashlib
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


def source_digest():
    """SHA-256 over the sources and the header (names and contents)."""
    h = hashlib.sha256()
    for path in sources() + [os.path.join(os.path.dirname(HERE), "include", "kfbim.h")]:
        h.update(os.path.basename(path).encode())
        with open(path, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def build(force=False, verbose=False):
    """Compile libkfbim.so unless it was built from the current sources (a
    digest of them, taken before compiling, is kept beside the library);
    return its path."""
    os.makedirs(OUT, exist_ok=True)
    stamp = os.path.join(OUT, "sources.sha256")
    digest = source_digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    nvcc = _nvcc()
    inc = "-I" + os.path.join(os.path.dirname(HERE), "include")
    o_setup = os.path.join(OUT, "setup.o")
    cu_units = ["kfbim", "slab", "pass2_n32", "pass2_n64", "pass2_n96", "pass2_n128", "pass2_n256"]
    objs = [os.path.join(OUT, u + ".o") for u in cu_units]
    cmds = [
        ["g++", "-std=c++17", "-O2", "-fPIC", "-ffp-contract=off", inc, "-c",
         os.path.join(SRC, "setup.cpp"), "-o", o_setup],
    ] + [
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", inc,
         "-Xptxas", "-v" if verbose else "-O3", "-c", os.path.join(SRC, u + ".cu"), "-o", o]
        for u, o in zip(cu_units, objs)
    ]
    with ThreadPoolExecutor(len(cmds)) as ex:
        logs = list(ex.map(_run, cmds))
    logs.append(_run([nvcc, ARCH, "-shared", o_setup] + objs + ["-o", LIB + ".tmp", "-lcudart"]))
    os.replace(LIB + ".tmp", LIB)
    with open(stamp, "w") as f:
        f.write(digest + "\n")
    if verbose:
        sys.stdout.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
