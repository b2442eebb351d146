"""The FP32 and MIXED_TF32 precision modes against the FP64 oracle.

* FP32: one FP32 grid solve per matvec (transforms and Schur CG to inner_tol,
  no FP64 refinement); jumps, corrections, traces and GMRES in FP64.  The
  matvec carries the FP32 solve's error (the CG stops at a relative residual
  of 3e-6), so it matches the oracle to 1e-4, and a solve with GMRES to 1e-6
  gives a density within 1e-3 of the oracle's.
* MIXED_TF32: MIXED refinement over the tensor-core (3xTF32) transform
  passes, N = 128 only; refined in FP64, its matvec matches the oracle to
  1e-8 like MIXED."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim as okfbim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP32, MIXED_TF32, KfbimError, Solver, build  # noqa: E402

build()


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_fp32_matvec_and_solve():
    geom, grid = ki.star(), ki.grid(64)
    o = okfbim.Setup(geom, grid)
    phi = ki.random_density(o.n, seed=23)
    s = Solver(geom, grid, precision=FP32, gmres_tol=1e-6)
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert rel(out.cpu().numpy(), o.apply(phi)) < 1e-4
    x = o.cp.xyz
    g = ki.stokes_velocity(x)[np.arange(o.cp.n), o.cp.comp - 1][o.primary]
    want = o.solve(g, tol=1e-10)["phi"]
    got = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.solve(cuda(g), got)
    assert s.last_stats["refine_sweeps"] == s.last_stats["interface_solves"]   # one FP32 pass each
    assert rel(got.cpu().numpy(), want) < 1e-3
    s.close()


def test_mixed_tf32_matvec_matches_oracle():
    geom, grid = ki.star(), ki.grid(128)
    o = okfbim.Setup(geom, grid)
    phi = ki.random_density(o.n, seed=29)
    s = Solver(geom, grid, precision=MIXED_TF32)
    info = s.transforms_info()
    assert info["plain"] == 1 and info["fused"] == 1
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert rel(out.cpu().numpy(), o.apply(phi)) < 1e-8
    s.close()


def test_mixed_tf32_needs_n128():
    with pytest.raises(KfbimError) as e:
        Solver(ki.star(), ki.grid(64), precision=MIXED_TF32)
    assert e.value.code == -1
