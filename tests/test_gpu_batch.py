"""Batched solve (kfbim_solve_batch): B boundary-data instances on one
geometry.  Each instance must reproduce the single-instance solve of the same
context (same GMRES, refinement and CG iterations; results equal up to
rounding order) and, for one instance, the FP64 oracle at the MIXED tolerance
1e-8.  Instances are divergence-free harmonic fields (exact Stokes solutions
with f = 0), the manufactured forced pair, and zero data."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim as okfbim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP64, MIXED, KfbimError, Solver, build  # noqa: E402

build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def face_forcing(s, frc):
    N, lo, h = s.N, s.lo, s.h
    idx = np.arange(N)
    out = []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")
        out.append(frc(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
    return np.concatenate(out)


def instances(s, B, forced=True):
    """B instances: k % 3 == 0 harmonic curl field (f = 0), 1 the forced
    manufactured pair, 2 zero data (only the first such)."""
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    N3 = s.N ** 3
    g = np.zeros((B, s.n_primary))
    fp = np.zeros((B, 3 * s.n_points))
    fg = np.zeros((B, 3 * N3))
    for b in range(B):
        kind = b % 3 if b < 3 else (0 if b % 2 == 0 else 1)
        if kind == 0:
            g[b] = ki.harmonic_curl_field(100 + b)(xyz)[rows, comp - 1][prim]
        elif kind == 1 and forced:
            g[b] = ki.stokes_velocity(xyz)[rows, comp - 1][prim] * (1.0 + 0.1 * b)
            fp[b] = (ki.stokes_forcing(xyz) * (1.0 + 0.1 * b)).T.ravel()
            fg[b] = face_forcing(s, ki.stokes_forcing) * (1.0 + 0.1 * b)
        elif kind == 1:
            g[b] = ki.harmonic_curl_field(200 + b, degree=3)(xyz)[rows, comp - 1][prim]
    return g, fp, fg


def run_batch(s, g, fp, fg):
    B, N3 = g.shape[0], s.N ** 3
    phi = torch.zeros((B, s.n_primary), dtype=torch.float64, device="cuda")
    u = torch.zeros((B, 3 * N3), dtype=torch.float64, device="cuda")
    p = torch.zeros((B, N3), dtype=torch.float64, device="cuda")
    s.solve_batch(cuda(g), phi, None if fp is None else cuda(fp), None if fg is None else cuda(fg), u, p)
    return phi.cpu().numpy(), u.cpu().numpy(), p.cpu().numpy(), s.last_stats


def run_single(s, g, fp, fg):
    N3 = s.N ** 3
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N3, dtype=torch.float64, device="cuda")
    s.solve(cuda(g), phi, None if fp is None else cuda(fp), None if fg is None else cuda(fg), u, p)
    return phi.cpu().numpy(), u.cpu().numpy(), p.cpu().numpy(), s.last_stats


def check_against_single(s, g, fp, fg, tol):
    phis, us, ps, stats = run_batch(s, g, fp, fg)
    for b in range(g.shape[0]):
        phi1, u1, p1, st1 = run_single(s, g[b], None if fp is None else fp[b],
                                       None if fg is None else fg[b])
        if not np.any(g[b]) and (fp is None or not np.any(fp[b])):
            assert not np.any(phis[b]) and stats[b]["gmres_iters"] == 0
            continue
        assert stats[b]["gmres_iters"] == st1["gmres_iters"], b
        assert stats[b]["interface_solves"] == st1["interface_solves"], b
        assert rel(phis[b], phi1) <= tol, b
        assert rel(us[b], u1) <= tol, b
        assert rel(ps[b], p1) <= tol, b
    return phis, us, ps, stats


@pytest.mark.parametrize("B", [1, 3, 17])
def test_batch_matches_single_sphere32(B):
    # B = 17: 51 jobs per stage, i.e. one 48-job launch and one 3-job launch
    s = Solver(ki.sphere(), ki.grid(32), precision=MIXED)
    g, fp, fg = instances(s, B)
    check_against_single(s, g, fp, fg, 1e-12)


def test_batch_without_forcing_star64():
    s = Solver(ki.star(), ki.grid(64), precision=MIXED)
    g, _, _ = instances(s, 4, forced=False)
    check_against_single(s, g, None, None, 1e-12)


def test_batch_fp64_context_loops():
    s = Solver(ki.sphere(), ki.grid(32))
    assert s.options.precision == FP64
    g, fp, fg = instances(s, 2)
    check_against_single(s, g, fp, fg, 0.0)


def test_batch_instance_matches_oracle():
    o = okfbim.Setup(ki.sphere(), ki.grid(32))
    s = Solver(ki.sphere(), ki.grid(32), precision=MIXED)
    g, _, _ = instances(s, 3, forced=False)
    phis, us, ps, _ = run_batch(s, g, None, None)
    want = o.solve(g[0])
    N = 32
    assert rel(phis[0], want["phi"]) < 1e-8
    ug = us[0].reshape(3, N, N, N)
    for c in range(3):
        assert rel(ug[c], want["u"][c]) < 1e-8
    assert rel(ps[0].reshape(N, N, N), want["p"]) < 1e-8


def harmonic_error(N):
    s = Solver(ki.sphere(), ki.grid(N), precision=MIXED)
    g, _, _ = instances(s, 1, forced=False)
    _, us, _, _ = run_batch(s, g, None, None)
    field = ki.harmonic_curl_field(100)
    lo, h = s.lo, s.h
    idx = np.arange(N)
    err = 0.0
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")
        exact = field(np.stack([X, Y, Z], -1))[..., c - 1].ravel()
        inside = s.sides(c).ravel()
        got = us[0][(c - 1) * N ** 3:c * N ** 3]
        err = max(err, np.abs(got[inside] - exact[inside]).max() / np.abs(exact[inside]).max())
    return err


def test_batch_harmonic_instance_converges():
    """A harmonic curl field is an exact Stokes solution (p constant): the
    batched solve's velocity at the Omega face nodes converges to it at
    second order (error ratio near 4 per halving of h)."""
    e32, e64 = harmonic_error(32), harmonic_error(64)
    assert e64 < 1e-2
    assert e32 / e64 > 2.5, (e32, e64)


def test_batch_errors():
    s = Solver(ki.sphere(), ki.grid(32), precision=MIXED)
    n = s.n_primary
    phi = torch.zeros((65, n), dtype=torch.float64, device="cuda")
    with pytest.raises(KfbimError) as e:
        s.solve_batch(torch.zeros((65, n), dtype=torch.float64, device="cuda"), phi)
    assert e.value.code == -1
    with pytest.raises(KfbimError) as e:
        s.solve_batch(torch.zeros((0, n), dtype=torch.float64, device="cuda"), phi)
    assert e.value.code == -1
    g, _, _ = instances(s, 2, forced=False)
    g[1, 7] = np.nan
    with pytest.raises(KfbimError) as e:
        s.solve_batch(cuda(g), phi[:2].contiguous())
    assert e.value.code == -4
    # the context stays usable after the error
    g[1, 7] = 0.0
    phis, _, _, stats = run_batch(s, g, None, None)
    assert all(st["gmres_residual"] < 1e-10 for st in stats)
