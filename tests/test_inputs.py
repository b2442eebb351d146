"""The seeded input generators behind the parity, convergence and benchmark
runs (kfbim_inputs), pinned to the mathematics: the manufactured Stokes pair
(divergence-free, forcing = -mu Lap u + grad p) and the Lame pair (jets and
forcing -mu Lap u - (lambda + mu) grad div u, Eq. Navier) against sympy's
symbolic derivatives, and the harmonic boundary-data fields (divergence-free
and harmonic, i.e. exact Stokes solutions with constant pressure and f = 0)
by finite differences, which are exact up to rounding and a small truncation
term for these polynomial fields."""
import numpy as np
import pytest

import kfbim_inputs as ki

sp = pytest.importorskip("sympy")
x, y, z = sp.symbols("x y z")
V = (x, y, z)
P = np.random.default_rng(7).uniform(-1.0, 1.0, (60, 3))
ARGS = (P[:, 0], P[:, 1], P[:, 2])


def ev(expr):
    return np.broadcast_to(sp.lambdify(V, expr, "numpy")(*ARGS), (len(P),)).astype(float)


def close(a, b, tol):
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= tol * max(np.abs(np.asarray(b)).max(), 1.0)


@pytest.mark.parametrize("mu", [1.0, 2.5])
def test_stokes_pair(mu):
    U = [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z), sp.Integer(0)]
    p = sp.sin(x + y + z)
    assert sp.simplify(sum(sp.diff(U[i], V[i]) for i in range(3))) == 0
    f = [-mu * sum(sp.diff(U[i], v, 2) for v in V) + sp.diff(p, V[i]) for i in range(3)]
    assert close(ki.stokes_velocity(P), np.stack([ev(e) for e in U], -1), 1e-14)
    assert close(ki.stokes_pressure(P), ev(p), 1e-14)
    assert close(ki.stokes_forcing(P, mu), np.stack([ev(e) for e in f], -1), 1e-13)


def test_lame_pair():
    mu, lam = ki.LAME_MU, ki.LAME_LAMBDA
    U = [sp.exp(x + y + z) * sp.sin(i + x * y) for i in (1, 2, 3)]
    u, G, H = ki.lame_jets(P)
    for i in range(3):
        assert close(u[:, i], ev(U[i]), 1e-14)
        for j in range(3):
            assert close(G[:, i, j], ev(sp.diff(U[i], V[j])), 1e-13)
            for k in range(3):
                assert close(H[:, i, j, k], ev(sp.diff(U[i], V[j], V[k])), 1e-13)
    div = sum(sp.diff(U[i], V[i]) for i in range(3))
    f = [-mu * sum(sp.diff(U[i], v, 2) for v in V) - (lam + mu) * sp.diff(div, V[i]) for i in range(3)]
    assert close(ki.lame_forcing(P), np.stack([ev(e) for e in f], -1), 1e-13)
    assert close(ki.lame_pressure(P), -(lam + mu) * ev(div), 1e-13)


def _derivatives(field, X, h):
    """Jacobian J[..., c, j] = d_j u^(c) and Laplacian of each component by
    fourth-order central differences."""
    n = X.shape[0]
    Jac = np.zeros((n, 3, 3))
    lap = np.zeros((n, 3))
    u0 = field(X)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        up1, um1, up2, um2 = field(X + e), field(X - e), field(X + 2 * e), field(X - 2 * e)
        Jac[:, :, j] = (8 * (up1 - um1) - (up2 - um2)) / (12 * h)
        lap += (-up2 + 16 * up1 - 30 * u0 + 16 * um1 - um2) / (12 * h * h)
    return u0, Jac, lap


@pytest.mark.parametrize("seed,degree", [(0, 6), (5, 3), (100, 6)])
def test_harmonic_curl_field_is_an_exact_stokes_solution(seed, degree):
    field = ki.harmonic_curl_field(seed, degree=degree)
    X = P[:20] * 0.6
    u0, Jac, lap = _derivatives(field, X, 5e-3)
    scale = np.abs(u0).max()
    assert scale > 0.1
    # div u = 0 and Lap u = 0: with p constant and f = 0 these are the Stokes equations
    assert np.abs(np.trace(Jac, axis1=1, axis2=2)).max() <= 1e-7 * np.abs(Jac).max()
    assert np.abs(lap).max() <= 1e-8 * np.abs(Jac).max()
    # the curl is not trivially zero, and the generator is seeded
    assert np.abs(Jac - np.transpose(Jac, (0, 2, 1))).max() > 1e-3 * np.abs(Jac).max()
    assert np.array_equal(field(X), ki.harmonic_curl_field(seed, degree=degree)(X))
    assert not np.allclose(field(X), ki.harmonic_curl_field(seed + 1, degree=degree)(X))


def test_harmonic_curl_field_has_zero_flux_through_the_sphere():
    """Solvability of interior Stokes Dirichlet data: the flux of u through a
    closed surface vanishes (sphere r = 0.5, Gauss-Legendre x trapezoid rule,
    exact for the field's polynomial degree)."""
    field = ki.harmonic_curl_field(3)
    t, w = np.polynomial.legendre.leggauss(24)
    ph = np.linspace(0, 2 * np.pi, 48, endpoint=False)
    T, PH = np.meshgrid(t, ph, indexing="ij")
    n = np.stack([np.sqrt(1 - T**2) * np.cos(PH), np.sqrt(1 - T**2) * np.sin(PH), T], -1)
    flux = np.sum(w[:, None] * np.sum(field(0.5 * n) * n, -1)) * (2 * np.pi / 48) * 0.25
    total = np.sum(w[:, None] * np.abs(np.sum(field(0.5 * n) * n, -1))) * (2 * np.pi / 48) * 0.25
    assert abs(flux) <= 1e-12 * total
