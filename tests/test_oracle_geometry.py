"""Pins of the oracle's level sets, frames and curvature (Alg. 1 step 1)
against finite differences and the sphere's closed form."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import geometry

GEOMS = [ki.sphere(0.5, (0.1, -0.05, 0.02)), ki.star(),
         ki.ellipsoid((0.6, 0.45, 0.35), ki.seeded_rotation(3))]


def _points(rng, n=40):
    x = rng.uniform(-0.7, 0.7, (n, 3))
    s = np.hypot(x[:, 0], x[:, 1])
    return x[s > 0.05]


@pytest.mark.parametrize("geom", GEOMS + [ki.torus(), ki.peanut(), ki.callback_sphere(0.4, (0.1, 0, 0))],
                         ids=lambda g: g["kind"])
def test_gradient_hessian_finite_differences(geom):
    rng = np.random.default_rng(11)
    X = _points(rng)
    F, G, H = geometry.level_set(geom, X)
    eps = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        Fp, Gp, _ = geometry.level_set(geom, X + e)
        Fm, Gm, _ = geometry.level_set(geom, X - e)
        assert np.allclose((Fp - Fm) / (2 * eps), G[:, k], rtol=1e-6, atol=1e-7)
        assert np.allclose((Gp - Gm) / (2 * eps), H[:, :, k], rtol=1e-5, atol=1e-6)
    assert np.allclose(H, np.swapaxes(H, 1, 2), atol=1e-12)


def test_sphere_curvature_closed_form():
    R = 0.37
    geom = ki.sphere(R, (0.0, 0.0, 0.0))
    rng = np.random.default_rng(2)
    d = rng.standard_normal((20, 3))
    X = R * d / np.linalg.norm(d, axis=1)[:, None]
    n, T, K = geometry.frames(geom, X)
    assert np.allclose(n, X / R)
    assert np.allclose(K, np.eye(2)[None] / R)
    assert np.allclose(np.einsum("nai,nbi->nab", T, T), np.eye(2)[None])
    assert np.allclose(np.einsum("nai,ni->na", T, n), 0.0)


def _surface_point_along_normal(geom, y, n, s, t, T):
    """Point of Gamma on the line y + s tau_1 + t tau_2 + z n (bisection in z)."""
    base = y + s * T[0] + t * T[1]
    lo, hi = -0.2, 0.2
    flo = geometry.level_value(geom, (base + lo * n)[None])[0]
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        fm = geometry.level_value(geom, (base + mid * n)[None])[0]
        if (fm <= 0) == (flo <= 0):
            lo, flo = mid, fm
        else:
            hi = mid
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: g["kind"])
def test_monge_height_matches_curvature(geom):
    """The surface is the graph z = -1/2 sigma^T K sigma + O(|sigma|^3) over the
    tangent plane, which fixes the sign convention of K used by jump eq. (i)."""
    rng = np.random.default_rng(5)
    for _ in range(4):
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        # project a ray from the centre onto the surface
        c = np.asarray(geom["center"])
        lo, hi = 0.0, 1.0
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if geometry.level_value(geom, (c + mid * d)[None])[0] <= 0:
                lo = mid
            else:
                hi = mid
        y = c + lo * d
        if np.hypot(*(y - c)[:2]) < 0.1:
            continue
        n, T, K = (a[0] for a in geometry.frames(geom, y[None]))
        for eps in (1e-3,):
            for (s, t) in [(eps, 0.0), (0.0, eps), (eps, eps), (eps, -0.5 * eps)]:
                z = _surface_point_along_normal(geom, y, n, s, t, T)
                sig = np.array([s, t])
                pred = -0.5 * sig @ K @ sig
                assert abs(z - pred) < 50 * eps ** 3 + 1e-13, (z, pred)


@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: g["kind"])
def test_normal_derivative_along_surface(geom):
    """d n / d s_a = sum_b K_ab tau_b (used by jump eq. (iv))."""
    rng = np.random.default_rng(9)
    c = np.asarray(geom["center"])
    d = rng.standard_normal(3)
    d /= np.linalg.norm(d)
    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if geometry.level_value(geom, (c + mid * d)[None])[0] <= 0:
            lo = mid
        else:
            hi = mid
    y = c + lo * d
    n, T, K = (a[0] for a in geometry.frames(geom, y[None]))
    eps = 1e-5
    for a in range(2):
        pts = []
        for sgn in (1.0, -1.0):
            z = _surface_point_along_normal(geom, y, n, sgn * eps * (a == 0), sgn * eps * (a == 1), T)
            p = y + sgn * eps * T[a] + z * n
            pts.append(geometry.frames(geom, p[None])[0][0])
        dn = (pts[0] - pts[1]) / (2 * eps)
        assert np.allclose(dn, K[a] @ T, atol=1e-5)


def test_torus_curvature_closed_form():
    """Principal curvatures of the torus (c - s)^2 + z^2 = a^2 at tube angle t:
    1/a around the tube and cos t / (c + a cos t) around the axis (negative on
    the inner side, where the surface is saddle-shaped)."""
    g = ki.torus(0.35, 0.7)
    t, f = np.meshgrid(np.linspace(0, 2 * np.pi, 9)[:-1], np.linspace(0, 2 * np.pi, 7)[:-1])
    t, f = t.ravel(), f.ravel()
    r = 0.7 + 0.35 * np.cos(t)
    X = np.stack([r * np.cos(f), r * np.sin(f), 0.35 * np.sin(t)], -1)
    assert np.abs(geometry.level_value(g, X)).max() < 1e-14
    n, _, K = geometry.frames(g, X)
    want_n = np.stack([np.cos(t) * np.cos(f), np.cos(t) * np.sin(f), np.sin(t)], -1)
    assert np.abs(n - want_n).max() < 1e-14
    got = np.sort(np.linalg.eigvalsh(K), axis=-1)
    want = np.sort(np.stack([np.full_like(t, 1 / 0.35), np.cos(t) / r], -1), axis=-1)
    assert np.abs(got - want).max() < 1e-12
