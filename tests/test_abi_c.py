"""The C ABI from C: tests/abi_consumer.c includes include/kfbim.h, compiles
as strict C99 and as C++17 with warnings as errors, links against the built
library and runs its host-only entry points (no GPU).  Its output must match
the Python binding's view of the same context and the geometry: every control
point on the sphere, one primary flag per density unknown, and the same sphere
given as C callbacks (CALLBACK kind) reproduces the built-in setup."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import kfbim_inputs as ki
from paper_2303_04992_gb300 import build
from paper_2303_04992_gb300.binding import Options, Solver

HERE = os.path.dirname(os.path.abspath(__file__))
INC = os.path.join(os.path.dirname(HERE), "include")
SRC = os.path.join(HERE, "abi_consumer.c")


def run_consumer(tmp_path, compiler, std):
    lib = build()
    libdir = os.path.dirname(lib)
    exe = str(tmp_path / ("consumer_" + compiler.replace("+", "x")))
    lang = ["-x", "c++"] if compiler == "g++" else []
    cmd = ([compiler, "-std=" + std, "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", INC] + lang
           + [SRC, "-x", "none", "-L", libdir, "-l:" + os.path.basename(lib), "-Wl,-rpath," + libdir,
              "-lm", "-o", exe])
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=300).stdout
    return {k: float(v) for k, v in (line.split() for line in out.splitlines())}


@pytest.mark.parametrize("compiler,std", [("gcc", "c99"), ("g++", "c++17")])
def test_c_consumer_matches_binding(tmp_path, compiler, std):
    if shutil.which(compiler) is None:
        pytest.skip(compiler + " not found")
    got = run_consumer(tmp_path, compiler, std)
    s = Solver(ki.sphere(), ki.grid(32), device=False)
    fit, rows, nnz = s.table_sizes()
    assert got["N"] == 32
    # the binding's options struct is the header's (size, and the last field's default)
    assert got["options_size"] == ctypes.sizeof(Options)
    assert got["relax"] == s.options.relax == 0.1
    assert got["n_points"] == s.n_points and got["n_primary"] == s.n_primary
    assert (got["fit_nnz"], got["corr_rows"], got["corr_nnz"]) == (fit, rows, nnz)
    assert got["primary_flags"] == s.n_primary
    assert got["max_distance"] < 1e-12
    assert got["omega_cells"] == int(np.count_nonzero(s.sides(0)))
    assert got["status_apply"] == -1 and got["status_bad_grid"] == -1
    assert got["callback_equal"] == 1
    _, comp, _, prim = s.points()
    assert got["control_points_total"] == s.n_primary
    assert got["control_points_1"] == int(np.count_nonzero(prim & (comp == 1)))
    assert got["normal_deviation"] < 1e-12
    assert got["jump_points"] == s.n_points
