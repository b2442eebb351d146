"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
inputs.  FP64 path: relative max-norm error <= 1e-10 (whole matvec / solve),
<= 1e-12 for single linear stages.  MIXED path: <= 1e-8 after refinement."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import interp, jumps as ojumps, kfbim as okfbim, mac

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import MIXED, Solver, build  # noqa: E402

build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


_ORACLE = {}


def oracle_setup(key, geom, N):
    if key not in _ORACLE:
        _ORACLE[key] = okfbim.Setup(geom, ki.grid(N))
    return _ORACLE[key]


CASES = [("sphere32", ki.sphere(), 32), ("star64", ki.star(), 64), ("torus64", ki.torus(0.2, 0.5), 64)]


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def pair(request):
    key, geom, N = request.param
    o = oracle_setup(key, geom, N)
    s = Solver(geom, ki.grid(N))
    return o, s


def test_control_points_match(pair):
    o, s = pair
    xyz, comp, axis, prim = s.points()
    assert np.array_equal(comp, o.cp.comp) and np.array_equal(axis, o.cp.axis)
    assert np.array_equal(prim, o.primary)
    assert np.abs(xyz - o.cp.xyz).max() < 1e-14


@pytest.mark.parametrize("c", [1, 2, 3])
def test_poisson(pair, c):
    o, s = pair
    N = s.N
    r = mac.zero_walls(np.random.default_rng(c).standard_normal((N, N, N)), c)
    want = mac.poisson(r, c, s.h)
    got = s.poisson(c, cuda(r), torch.zeros(N ** 3, dtype=torch.float64, device="cuda"))
    assert rel(got.cpu().numpy().reshape(N, N, N), want) < 1e-12


def test_schur_apply(pair):
    o, s = pair
    N = s.N
    d = np.random.default_rng(9).standard_normal((N, N, N))
    want = mac.schur_apply(d, 1.0, s.h, 1.0 * N ** 3)
    got = s.schur_apply(cuda(d), torch.zeros(N ** 3, dtype=torch.float64, device="cuda"))
    assert rel(got.cpu().numpy().reshape(N, N, N), want) < 1e-12


def test_jumps(pair):
    o, s = pair
    rng = np.random.default_rng(3)
    phi = rng.standard_normal(s.n_primary)
    fy = rng.standard_normal((s.n_points, 3))
    want = ojumps.jumps(o.jd, phi, fy, 1.0)
    J = torch.zeros(12 * s.n_points, dtype=torch.float64, device="cuda")
    s.jumps(cuda(phi), J, cuda(fy.T.copy()))
    got = J.cpu().numpy().reshape(12, s.n_points).T
    for k in range(12):
        assert rel(got[:, k], want[:, k]) < 1e-11, k


def test_trace(pair):
    o, s = pair
    N = s.N
    rng = np.random.default_rng(4)
    u = [mac.zero_walls(rng.standard_normal((N, N, N)), c) for c in (1, 2, 3)]
    J = rng.standard_normal((s.n_points, 12))
    want = interp.trace(o.grid, o.cp, o.S, u, J)[o.primary]
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.trace(cuda(np.concatenate([x.ravel() for x in u])), cuda(J.T.copy()), out)
    assert rel(out.cpu().numpy(), want) < 1e-12


def test_interface_solve(pair):
    o, s = pair
    N = s.N
    rng = np.random.default_rng(5)
    phi = rng.standard_normal(s.n_primary)
    x = o.cp.xyz
    fy = ki.stokes_forcing(x)
    ff = [ki.stokes_forcing(o.grid.node_xyz(c, o.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    u_w, p_w, _ = o.interface(phi, fy, ff)
    u = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    s.interface(cuda(phi), u, p, cuda(fy.T.copy()), cuda(np.concatenate([f.ravel() for f in ff])))
    ug = u.cpu().numpy().reshape(3, N, N, N)
    for c in range(3):
        assert rel(ug[c], u_w[c]) < 1e-10
    assert rel(p.cpu().numpy().reshape(N, N, N), p_w) < 1e-10


def test_pressure_trace(pair):
    o, s = pair
    N = s.N
    rng = np.random.default_rng(21)
    p = rng.standard_normal((N, N, N))
    J = rng.standard_normal((o.cp.n, 12))
    want = interp.pressure_trace(o.grid, o.cp, o.S, p, J)
    out = torch.zeros(o.cp.n, dtype=torch.float64, device="cuda")
    s.pressure_trace(cuda(p.ravel()), cuda(J.T.copy()), out)
    assert rel(out.cpu().numpy(), want) < 1e-13


def test_apply(pair):
    o, s = pair
    phi = np.random.default_rng(6).standard_normal(s.n_primary)
    want = o.apply(phi)
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert rel(out.cpu().numpy(), want) < 1e-10


def test_constant_density_identity(pair):
    o, s = pair
    _, comp, _, prim = s.points()
    phi = np.array([1.0, -0.5, 0.25])[comp[prim] - 1]
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert np.abs(out.cpu().numpy() - phi).max() < 1e-12


def _solve_inputs(o):
    x = o.cp.xyz
    rows = np.arange(o.cp.n)
    g = ki.stokes_velocity(x)[rows, o.cp.comp - 1][o.primary]
    fy = ki.stokes_forcing(x)
    ff = [ki.stokes_forcing(o.grid.node_xyz(c, o.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    return g, fy, ff


def test_solve_fp64_sphere32():
    o = oracle_setup("sphere32", ki.sphere(), 32)
    g, fy, ff = _solve_inputs(o)
    want = o.solve(g, fy, ff)
    s = Solver(ki.sphere(), ki.grid(32))
    N = 32
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    s.solve(cuda(g), phi, cuda(fy.T.copy()), cuda(np.concatenate([f.ravel() for f in ff])), u, p)
    assert rel(phi.cpu().numpy(), want["phi"]) < 1e-10
    ug = u.cpu().numpy().reshape(3, N, N, N)
    for c in range(3):
        assert rel(ug[c], want["u"][c]) < 1e-10
    assert rel(p.cpu().numpy().reshape(N, N, N), want["p"]) < 1e-10
    assert abs(s.last_stats["gmres_iters"] - want["iters"]) <= 1


def test_solve_mixed_sphere32():
    o = oracle_setup("sphere32", ki.sphere(), 32)
    g, fy, ff = _solve_inputs(o)
    want = o.solve(g, fy, ff)
    s = Solver(ki.sphere(), ki.grid(32), precision=MIXED)
    N = 32
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    s.solve(cuda(g), phi, cuda(fy.T.copy()), cuda(np.concatenate([f.ravel() for f in ff])), u, p)
    assert rel(phi.cpu().numpy(), want["phi"]) < 1e-8
    ug = u.cpu().numpy().reshape(3, N, N, N)
    for c in range(3):
        assert rel(ug[c], want["u"][c]) < 1e-8
    assert rel(p.cpu().numpy().reshape(N, N, N), want["p"]) < 1e-8


# ------------------------------------------------------------------ Navier
ELL = ki.ellipsoid((0.6, 0.45, 0.35), ki.seeded_rotation(3))


def _navier_pair(N=32):
    key = "navier_ell%d" % N
    if key not in _ORACLE:
        _ORACLE[key] = okfbim.Setup(ELL, ki.grid(N), mu=ki.LAME_MU, lam=ki.LAME_LAMBDA)
    return _ORACLE[key]


def _lame_inputs(o):
    x = o.cp.xyz
    rows = np.arange(o.cp.n)
    g = ki.lame_displacement(x)[rows, o.cp.comp - 1][o.primary]
    fy = ki.lame_forcing(x)
    ff = [ki.lame_forcing(o.grid.node_xyz(c, o.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    return g, fy, ff


def test_navier_jumps_and_apply():
    o = _navier_pair()
    rng = np.random.default_rng(21)
    phi = rng.standard_normal(o.n)
    fy = rng.standard_normal((o.cp.n, 3))
    want_J = ojumps.jumps(o.jd, phi, fy, ki.LAME_MU, ki.LAME_LAMBDA)
    want = o.apply(phi)
    for prec, tol in ((0, 1e-10), (MIXED, 1e-8)):
        s = Solver(ELL, ki.grid(32), mu=ki.LAME_MU, lam=ki.LAME_LAMBDA, precision=prec)
        J = torch.zeros(12 * s.n_points, dtype=torch.float64, device="cuda")
        s.jumps(cuda(phi), J, cuda(fy.T.copy()))
        got = J.cpu().numpy().reshape(12, s.n_points).T
        for k in range(12):
            assert rel(got[:, k], want_J[:, k]) < 1e-11, k
        out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
        s.apply(cuda(phi), out)
        assert rel(out.cpu().numpy(), want) < tol, prec
        s.close()


def test_navier_schur_apply():
    o = _navier_pair()
    N = 32
    d = np.random.default_rng(22).standard_normal((N, N, N))
    want = mac.schur_apply(d, ki.LAME_MU, o.grid.h, ki.LAME_MU * N ** 3, o.cpen)
    s = Solver(ELL, ki.grid(N), mu=ki.LAME_MU, lam=ki.LAME_LAMBDA)
    got = s.schur_apply(cuda(d), torch.zeros(N ** 3, dtype=torch.float64, device="cuda"))
    assert rel(got.cpu().numpy().reshape(N, N, N), want) < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (MIXED, 1e-8)])
def test_navier_solve(prec, tol):
    o = _navier_pair()
    g, fy, ff = _lame_inputs(o)
    key = "navier_solution"
    if key not in _ORACLE:
        _ORACLE[key] = o.solve(g, fy, ff)
    want = _ORACLE[key]
    N = 32
    s = Solver(ELL, ki.grid(N), mu=ki.LAME_MU, lam=ki.LAME_LAMBDA, precision=prec)
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * N ** 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(N ** 3, dtype=torch.float64, device="cuda")
    s.solve(cuda(g), phi, cuda(fy.T.copy()), cuda(np.concatenate([f.ravel() for f in ff])), u, p)
    assert rel(phi.cpu().numpy(), want["phi"]) < tol
    ug = u.cpu().numpy().reshape(3, N, N, N)
    for c in range(3):
        assert rel(ug[c], want["u"][c]) < tol
    assert rel(p.cpu().numpy().reshape(N, N, N), want["p"]) < 10 * tol
