"""The largest grid the solver accepts, N = 256 (the four-step transform
passes, whose DST-I takes a complex FFT of length 512 with its last radix-2
step between lane pairs).

The FP64 Poisson solve of each velocity component (DST-II along the two
tangential axes, DST-I along the normal one) against the oracle's at 256^3:
relative max-norm difference 1e-12, as at the smaller grids.

The star with the manufactured forced Stokes pair: MIXED against FP64, and
convergence from 128^3 to 256^3 towards the exact velocity.

MIXED against FP64 at the 128^3 bars (density and velocity 1e-8, pressure
1e-8), with both GMRES iterations run to a relative residual of 1e-12.  The
MIXED/FP64 gap has two parts.  One comes from where each GMRES stops and is
about kappa(A) times the stopping tolerance; at the workload tolerance 1e-10
it alone is of the order of the bar, so both solves go to 1e-12 here and the
gap that remains is that of the arithmetic.  The other comes from the FP64
refinement, which stops at a relative residual 1e-11 of the corrected MAC
system; the solution error that residual leaves grows with the system's
condition number (like h^-2).

The star r = 0.5 + 0.1 sin 3theta cos 4phi is Lipschitz but not C^1 at its
poles (r - 0.5 grows linearly in the distance from the axis, times cos 4phi),
and the maximum velocity error sits there; it falls slowly on coarse grids
(about 5.8e-2 at 32^3, 2.0e-2 at 128^3) and at second order from 128^3 to
256^3 (4.5e-3 at 256^3 on GB300), so the usual bar applies: a fall by more
than 2.5 per halving of h."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import mac

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP64, MIXED, Solver, build  # noqa: E402

build()


def face_nodes(s, c):
    N, lo, h = s.N, s.lo, s.h
    idx = np.arange(N)
    off = [0.5, 0.5, 0.5]
    off[c - 1] = 0.0
    Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                          lo + (idx + off[0]) * h, indexing="ij")
    return np.stack([X, Y, Z], -1)


def solve(s, tol=1e-10):
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    g = ki.stokes_velocity(xyz)[rows, comp - 1][prim]
    fp = ki.stokes_forcing(xyz).T.copy()
    fg = np.concatenate([ki.stokes_forcing(face_nodes(s, c))[..., c - 1].ravel() for c in (1, 2, 3)])
    N3 = s.N ** 3
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N3, dtype=torch.float64, device="cuda")
    gd, fpd, fgd = [torch.from_numpy(a).cuda() for a in (g, fp, fg)]
    s.solve(gd, phi, fpd, fgd, u, p)
    assert s.last_stats["gmres_residual"] < tol
    return phi.cpu().numpy(), u.cpu().numpy(), p.cpu().numpy()


def velocity_error(s, u):
    """Max error over the Omega face nodes of all components, relative to the
    largest exact value there."""
    N3 = s.N ** 3
    err, scale = 0.0, 0.0
    for c in (1, 2, 3):
        inside = s.sides(c).ravel()
        exact = ki.stokes_velocity(face_nodes(s, c))[..., c - 1].ravel()[inside]
        got = u[(c - 1) * N3:c * N3][inside]
        err = max(err, np.abs(got - exact).max())
        scale = max(scale, np.abs(exact).max())
    return err / scale


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module")
def sphere256():
    s = Solver(ki.sphere(), ki.grid(256), precision=FP64)
    yield s
    s.close()


@pytest.mark.parametrize("c", [1, 2, 3])
def test_poisson_256_matches_oracle(sphere256, c):
    s, N = sphere256, 256
    r = mac.zero_walls(np.random.default_rng(40 + c).standard_normal((N, N, N)), c)
    want = mac.poisson(r, c, s.h)
    got = s.poisson(c, torch.from_numpy(r.ravel()).cuda(), torch.zeros(N ** 3, dtype=torch.float64, device="cuda"))
    assert rel(got.cpu().numpy().reshape(N, N, N), want) < 1e-12


def test_star256_mixed_matches_fp64_and_converges():
    geom = ki.star()
    s128 = Solver(geom, ki.grid(128), precision=MIXED)
    e128 = velocity_error(s128, solve(s128)[1])
    s128.close()
    s = Solver(geom, ki.grid(256), precision=MIXED, gmres_tol=1e-12)
    phi, u, p = solve(s, 1e-12)
    e256 = velocity_error(s, u)
    s.close()
    s64 = Solver(geom, ki.grid(256), precision=FP64, gmres_tol=1e-12)
    phi64, u64, p64 = solve(s64, 1e-12)
    s64.close()
    got = {"phi": rel(phi, phi64), "u": rel(u, u64), "p": rel(p, p64), "e128": e128, "e256": e256}
    assert got["phi"] < 1e-8, got
    assert got["u"] < 1e-8, got
    assert got["p"] < 1e-8, got
    assert e256 < 1e-2, got
    assert e128 / e256 > 2.5, got
