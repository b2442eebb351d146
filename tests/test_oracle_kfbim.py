"""End-to-end pins of the oracle's BIE matvec and solve (Alg. 1)."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim
from tests import _fields


def _const_density(s, vals=(1.0, -0.5, 0.25)):
    return np.asarray(vals)[s.cp.comp - 1][s.primary]


@pytest.mark.parametrize("geom,N", [(ki.sphere(), 16), (ki.star(), 32)], ids=["sphere16", "star32"])
def test_constant_density_is_reproduced(geom, N):
    """phi = const: the interface problem is solved exactly by u = phi in
    Omega, 0 outside, p = 0, so (1/2 I - M_v) phi = phi at any N."""
    s = kfbim.Setup(geom, ki.grid(N))
    phi = _const_density(s)
    assert np.abs(s.apply(phi) - phi).max() < 1e-12


def test_rigid_motion_density_converges():
    om, c0 = np.array([0.3, -0.7, 0.5]), np.array([0.2, 0.1, -0.4])
    errs = []
    for N in (16, 32):
        s = kfbim.Setup(ki.sphere(), ki.grid(N))
        phi = _fields.component_values(lambda x: np.cross(om, x) + c0, s.cp)[s.primary]
        errs.append(np.abs(s.apply(phi) - phi).max())
    assert errs[0] / errs[1] > 4.0


def _exact_problem(N, R=0.5):
    s = kfbim.Setup(ki.sphere(R), ki.grid(N))
    g = _fields.component_values(lambda x: _fields.traction_free_W(x, R), s.cp)
    fy = _fields.traction_free_W_forcing(s.cp.xyz, R, s.mu)
    ff = [_fields.traction_free_W_forcing(s.grid.node_xyz(c, s.grid.all_idx()), R, s.mu)[..., c - 1]
          for c in (1, 2, 3)]
    return s, g, fy, ff


def test_exact_density_and_second_order_convergence():
    """Dirichlet data W|Gamma, forcing -mu Lap W: the exact solution is W in
    Omega, p = const, and the exact density is phi = W|Gamma (u- = 0 solves the
    exterior, IUS-4 holds because W is traction-free).  GMRES counts stay
    bounded (second-kind BIE, Sec. 3) and the velocity converges at second
    order (Sec. 5)."""
    out = []
    for N in (16, 32):
        s, g, fy, ff = _exact_problem(N)
        r = s.solve(g[s.primary], fy, ff)
        err = 0.0
        for c in (1, 2, 3):
            X = s.grid.node_xyz(c, s.grid.all_idx())
            m = s.S[c] & s.grid.unknown_mask(c)
            err = max(err, np.abs(r["u"][c - 1] - _fields.traction_free_W(X, 0.5)[..., c - 1])[m].max())
        out.append((r["iters"], np.abs(r["phi"] - g[s.primary]).max(), err))
    (i16, p16, e16), (i32, p32, e32) = out
    assert i16 <= 25 and i32 <= 25
    assert e16 / e32 > 3.5
    assert p16 / p32 > 3.5


def test_gmres_matches_dense_solve():
    """GMRES to 1e-12 equals a dense LU solve of the assembled BIE matrix."""
    s = kfbim.Setup(ki.sphere(), ki.grid(12))
    n = s.n
    A = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        A[:, j] = s.apply(e)
    b = np.random.default_rng(1).standard_normal(n)
    x_d = np.linalg.solve(A, b)
    x_g, it, _ = kfbim.gmres(s.apply, b, tol=1e-12)
    assert np.abs(x_g - x_d).max() < 1e-9 * np.abs(x_d).max()
    assert np.abs(np.linalg.eigvals(A)).min() > 0.05


def test_gmres_on_random_matrix():
    rng = np.random.default_rng(5)
    A = np.eye(40) + 0.3 * rng.standard_normal((40, 40)) / np.sqrt(40)
    b = rng.standard_normal(40)
    x, it, hist = kfbim.gmres(lambda v: A @ v, b, tol=1e-13)
    assert np.abs(A @ x - b).max() < 1e-11
    assert hist[-1] < 1e-13


def test_navier_constant_density_and_convergence():
    """Navier (Lame, mu = 1, lambda = 2): constant densities are reproduced
    exactly; the manufactured displacement exp(x+y+z) sin(i+xy) converges at
    second order with bounded GMRES counts."""
    errs, its = [], []
    for N in (16, 32):
        s = kfbim.Setup(ki.sphere(), ki.grid(N), mu=ki.LAME_MU, lam=ki.LAME_LAMBDA)
        phi = _const_density(s)
        assert np.abs(s.apply(phi) - phi).max() < 1e-12
        rows = np.arange(s.cp.n)
        g = ki.lame_displacement(s.cp.xyz)[rows, s.cp.comp - 1][s.primary]
        fy = ki.lame_forcing(s.cp.xyz)
        ff = [ki.lame_forcing(s.grid.node_xyz(c, s.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
        r = s.solve(g, fy, ff)
        e = 0.0
        for c in (1, 2, 3):
            X = s.grid.node_xyz(c, s.grid.all_idx())
            m = s.S[c] & s.grid.unknown_mask(c)
            ue = ki.lame_displacement(X)[..., c - 1]
            e = max(e, np.abs(r["u"][c - 1] - ue)[m].max() / np.abs(ue[m]).max())
        errs.append(e)
        its.append(r["iters"])
    assert errs[0] / errs[1] > 3.5
    assert max(its) <= 25


def _stokes_velocity_error(geom, N):
    """Max velocity error of the manufactured Stokes pair over the Omega face
    nodes, relative to the largest exact value there."""
    s = kfbim.Setup(geom, ki.grid(N))
    x = s.cp.xyz
    g = ki.stokes_velocity(x)[np.arange(s.cp.n), s.cp.comp - 1][s.primary]
    ff = [ki.stokes_forcing(s.grid.node_xyz(c, s.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    r = s.solve(g, ki.stokes_forcing(x), ff)
    err = scale = 0.0
    for c in (1, 2, 3):
        m = s.S[c]
        ue = ki.stokes_velocity(s.grid.node_xyz(c, s.grid.all_idx()))[..., c - 1]
        err = max(err, np.abs((r["u"][c - 1] - ue)[m]).max())
        scale = max(scale, np.abs(ue[m]).max())
    return s, err / scale


def test_grazing_segments_are_resolved(monkeypatch):
    """R = 0.5 about (0.01, -0.02, 0) at N = 32 grazes two combined face/cell
    segments (both faces outside, the cell centre inside).  Their two roots
    each, with the divergence and gradient corrections of their half-segment,
    make it as accurate as R = 0.45 about the same centre (no grazing); with
    the corrections of those roots dropped (a mistake planted in the oracle)
    the error grows several times, so the pin sees them."""
    s, e_graze = _stokes_velocity_error(ki.sphere(0.5, (0.01, -0.02, 0.0)), 32)
    assert int(np.sum(s.cp.graze > 0)) == 4
    _, e_plain = _stokes_velocity_error(ki.sphere(0.45, (0.01, -0.02, 0.0)), 32)
    assert e_graze < 1.5 * e_plain
    orig = kfbim.correct.corrections

    def dropped(grid, cp, S, J, mu):
        J = J.copy()
        J[cp.graze > 0] = 0.0
        return orig(grid, cp, S, J, mu)

    monkeypatch.setattr(kfbim.correct, "corrections", dropped)
    _, e_dropped = _stokes_velocity_error(ki.sphere(0.5, (0.01, -0.02, 0.0)), 32)
    assert e_dropped > 4 * e_graze
