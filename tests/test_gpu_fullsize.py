"""The CUDA path at the benchmark size (star, N = 128) in the benchmark's
configuration, and the error paths of the C ABI.

* one matvec against the oracle's (FP64: <= 1e-10; MIXED: <= 1e-8);
* the constant-density identity A phi = phi, exact at any size;
* a full MIXED solve (the default relaxation of late matvecs) against the
  FP64 GPU solve (<= 1e-8; both solve the same discrete BIE, parity-tested
  against the oracle at smaller N);
* NaN data -> KFBIM_E_NONFINITE; GMRES cap -> KFBIM_E_NOCONV with the last
  iterate written; bad arguments -> KFBIM_E_INVALID."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim as okfbim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP64, MIXED, KfbimError, Solver, build  # noqa: E402

build()
GEOM, GRID = ki.WORKLOADS["star128"]


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max()


@pytest.fixture(scope="module")
def solvers():
    return {FP64: Solver(GEOM, GRID, precision=FP64), MIXED: Solver(GEOM, GRID, precision=MIXED)}


def test_apply_matches_oracle_at_128(solvers):
    o = okfbim.Setup(GEOM, GRID)
    phi = ki.random_density(o.n, seed=11)
    want = o.apply(phi)
    for prec, tol in ((FP64, 1e-10), (MIXED, 1e-8)):
        s = solvers[prec]
        assert s.n_primary == o.n
        out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
        s.apply(cuda(phi), out)
        assert rel(out.cpu().numpy(), want) < tol, prec


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (MIXED, 1e-10)])
def test_constant_density_identity_at_128(solvers, prec, tol):
    s = solvers[prec]
    _, comp, _, prim = s.points()
    phi = np.array([0.7, -1.3, 0.4])[comp[prim] - 1]
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert np.abs(out.cpu().numpy() - phi).max() < tol


def _inputs(s):
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    g = ki.stokes_velocity(xyz)[rows, comp - 1][prim]
    fpts = ki.stokes_forcing(xyz).T.copy()
    N, h = s.N, s.h
    idx = np.arange(N)
    fg = []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(s.lo + (idx + off[2]) * h, s.lo + (idx + off[1]) * h,
                              s.lo + (idx + off[0]) * h, indexing="ij")
        fg.append(ki.stokes_forcing(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
    return g, fpts, np.concatenate(fg)


def test_mixed_solve_matches_fp64_solve_at_128(solvers):
    out = {}
    for prec in (FP64, MIXED):
        s = solvers[prec]
        g, fpts, fg = _inputs(s)
        phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
        p = torch.zeros(s.N ** 3, dtype=torch.float64, device="cuda")
        s.solve(cuda(g), phi, cuda(fpts), cuda(fg), None, p)
        out[prec] = (phi.cpu().numpy(), p.cpu().numpy(), s.last_stats)
    assert rel(out[MIXED][0], out[FP64][0]) < 1e-8
    assert rel(out[MIXED][1], out[FP64][1]) < 1e-7
    # the inexact (refined FP32) matvec may take a few more GMRES steps near the
    # tolerance, and the relaxed refinement of late matvecs (relax = 0.1, the
    # default) some more: at most 15 % over the FP64 count
    it_m, it_64 = out[MIXED][2]["gmres_iters"], out[FP64][2]["gmres_iters"]
    assert it_64 - 3 <= it_m <= 1.15 * it_64 + 1, (it_m, it_64)


def test_nonfinite_data_is_reported(solvers):
    s = solvers[FP64]
    g = np.zeros(s.n_primary)
    g[5] = np.nan
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    with pytest.raises(KfbimError) as e:
        s.solve(cuda(g), phi)
    assert e.value.code == -4


def test_gmres_cap_reports_noconv_with_last_iterate():
    s = Solver(ki.sphere(), ki.grid(32), gmres_max=3)
    g, fpts, fg = _inputs(s)
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    with pytest.raises(KfbimError) as e:
        s.solve(cuda(g), phi, cuda(fpts), cuda(fg))
    assert e.value.code == -3
    assert float(phi.abs().max()) > 0.0


def test_bad_arguments_are_rejected(solvers):
    s = solvers[FP64]
    x = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    with pytest.raises(KfbimError) as e:
        s.apply(x, x)                    # aliasing input and output
    assert e.value.code == -1
    with pytest.raises(KfbimError) as e:
        s.poisson(4, x, x)               # no face grid 4
    assert e.value.code == -1
