"""Pins of the oracle's jump conditions (Sec. 4.3, derived from IUS-1..4) and
surface fits, against exact jets of analytic fields that satisfy the interface
conditions."""
import itertools

import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import geometry, grid as gridmod, jumps

MU = 1.3


def test_second_order_system_full_rank():
    rng = np.random.default_rng(1)
    for _ in range(5):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        n = Q[:, 0][None]
        T = np.stack([Q[:, 1], Q[:, 2]])[None]
        K = rng.standard_normal((1, 2, 2))
        K = K + np.swapaxes(K, 1, 2)
        L = jumps.second_order_system(n, T, K, MU)[0]
        assert np.linalg.matrix_rank(L) == 21
        assert np.linalg.cond(L) < 1e3


# ---- traction-free polynomial pairs (w, pi) on a sphere of radius R at 0 ----
R = 0.45


def _monos(d):
    return [e for e in itertools.product(range(d + 1), repeat=3) if sum(e) <= d]


MW, MP = _monos(3), _monos(2)


def _mono_vals(ms, x, der=(0, 0, 0)):
    cols = []
    for e in ms:
        f = 1.0
        ee = list(e)
        for k in range(3):
            for _ in range(der[k]):
                f *= ee[k]
                ee[k] -= 1
        if f == 0 or min(ee) < 0:
            cols.append(np.zeros(len(x)))
        else:
            cols.append(f * x[:, 0] ** ee[0] * x[:, 1] ** ee[1] * x[:, 2] ** ee[2])
    return np.stack(cols, -1)


def traction_free_family():
    """Null space of {div w = 0 in R^3, (-pi I + mu(grad w + grad w^T)) n = 0 on
    |x| = R} over cubic w and quadratic pi (exact polynomial identities,
    imposed at enough sample points)."""
    rng = np.random.default_rng(0)
    nw, npi = len(MW), len(MP)
    X = rng.standard_normal((120, 3))
    rows = [np.concatenate([_mono_vals(MW, X, tuple(int(k == c) for k in range(3)))
                            for c in range(3)] + [np.zeros((len(X), npi))], axis=1)]
    S = rng.standard_normal((200, 3))
    S = R * S / np.linalg.norm(S, axis=1)[:, None]
    n = S / R
    for i in range(3):
        T = np.zeros((len(S), 3 * nw + npi))
        T[:, 3 * nw:] = -_mono_vals(MP, S) * n[:, i:i + 1]
        for k in range(3):
            T[:, i * nw:(i + 1) * nw] += MU * _mono_vals(MW, S, tuple(int(m == k) for m in range(3))) * n[:, k:k + 1]
            T[:, k * nw:(k + 1) * nw] += MU * _mono_vals(MW, S, tuple(int(m == i) for m in range(3))) * n[:, k:k + 1]
        rows.append(T)
    M = np.vstack(rows)
    _, s, vt = np.linalg.svd(M)
    null = vt[np.sum(s > 1e-10 * s[0]):]
    return null


def jets(coef, x):
    """Value, gradient, Hessian of w and pi, and -mu Lap w + grad pi at x."""
    nw = len(MW)
    w = np.zeros((len(x), 3))
    gw = np.zeros((len(x), 3, 3))
    hw = np.zeros((len(x), 3, 3, 3))
    for c in range(3):
        cc = coef[c * nw:(c + 1) * nw]
        w[:, c] = _mono_vals(MW, x) @ cc
        for j in range(3):
            gw[:, c, j] = _mono_vals(MW, x, tuple(int(k == j) for k in range(3))) @ cc
            for l in range(3):
                d = [0, 0, 0]
                d[j] += 1
                d[l] += 1
                hw[:, c, j, l] = _mono_vals(MW, x, tuple(d)) @ cc
    cp_ = coef[3 * nw:]
    pi = _mono_vals(MP, x) @ cp_
    gpi = np.stack([_mono_vals(MP, x, tuple(int(k == j) for k in range(3))) @ cp_ for j in range(3)], -1)
    f = -MU * np.einsum("ncjj->nc", hw) + gpi
    return w, gw, hw, pi, gpi, f


def test_traction_free_family_nontrivial():
    null = traction_free_family()
    assert null.shape[0] >= 8        # rigid motions, R^2 - r^2 and more


@pytest.mark.parametrize("member", [0, 3, 6, 9])
def test_jump_relations_exact_on_traction_free_pairs(member):
    """With exact surface derivatives of phi = w|Gamma and [f~] = -mu Lap w +
    grad pi, the first-order formulas and the 21x21 system return exactly
    the jets of (w, pi): u+ = w, p+ = pi inside, u- = 0, p- = 0 outside."""
    null = traction_free_family()
    rng = np.random.default_rng(member)
    coef = rng.standard_normal(null.shape[0]) @ null
    d = rng.standard_normal((30, 3))
    y = R * d / np.linalg.norm(d, axis=1)[:, None]
    geom = ki.sphere(R)
    n, T, K = geometry.frames(geom, y)
    w, gw, hw, pi, gpi, f = jets(coef, y)
    # exact surface derivatives of phi^(c) = w_c on the sphere (Monge coordinates)
    d1 = np.einsum("ncj,naj->nca", gw, T)
    gn = np.einsum("ncj,nj->nc", gw, n)
    d2 = np.zeros((len(y), 3, 3))
    for m, (a, b) in enumerate([(0, 0), (0, 1), (1, 1)]):
        d2[:, :, m] = np.einsum("ncjl,nj,nl->nc", hw, T[:, a], T[:, b]) - K[:, a, b][:, None] * gn
    A, q = jumps.first_order(n, T, d1, MU)
    assert np.abs(A - gw).max() < 1e-10 * max(1.0, np.abs(gw).max())
    assert np.abs(q - pi).max() < 1e-10 * max(1.0, np.abs(pi).max())
    L = jumps.second_order_system(n, T, K, MU)
    rhs = jumps.second_order_rhs(n, T, K, A, q, d2, f, MU)
    x = np.linalg.solve(L, rhs[..., None])[..., 0]
    for c in range(3):
        for m, (k, l) in enumerate(jumps.SYM):
            assert np.abs(x[:, 6 * c + m] - hw[:, c, k, l]).max() < 1e-9 * max(1.0, np.abs(hw).max())
    assert np.abs(x[:, 18:] - gpi).max() < 1e-9 * max(1.0, np.abs(gpi).max())


def test_fit_exact_for_tangent_plane_quadratics():
    """The weighted quadratic fit reproduces a quadratic in the (s, t)
    coordinates of the point's tangent plane exactly."""
    g = gridmod.Grid(24, -1.0, 1.0)
    geom = ki.star()
    cp, _ = gridmod.control_points(g, geom)
    fr = geometry.frames(geom, cp.xyz)
    prim = jumps.primary_points(cp, fr)
    nb = jumps.neighbour_lists(cp, prim)
    coef = np.array([0.3, -1.1, 0.7, 2.0, -0.4, 0.9])
    for y in range(0, cp.n, 211):
        s = (cp.xyz - cp.xyz[y]) @ fr[1][y, 0]
        t = (cp.xyz - cp.xyz[y]) @ fr[1][y, 1]
        phi = coef[0] + coef[1] * s + coef[2] * t + coef[3] * s * s + coef[4] * s * t + coef[5] * t * t
        der = jumps.surface_derivatives(cp, fr, nb, phi, g.h)[y]
        want = np.array([coef[0], coef[1], coef[2], 2 * coef[3], coef[4], 2 * coef[5]])
        for cc in range(3):
            assert np.allclose(der[cc], want, rtol=1e-8, atol=1e-8)


def test_primary_points_cover_each_direction_once():
    """Every point is primary for the line family most normal to Gamma there."""
    g = gridmod.Grid(24, -1.0, 1.0)
    cp, _ = gridmod.control_points(g, ki.sphere())
    fr = geometry.frames(ki.sphere(), cp.xyz)
    prim = jumps.primary_points(cp, fr)
    n = fr[0]
    for m in range(cp.n):
        assert prim[m] == (np.argmax(np.abs(n[m])) == cp.axis[m]) or \
            abs(abs(n[m, cp.axis[m]]) - np.abs(n[m]).max()) < 1e-12
    assert 0.3 < prim.mean() < 0.8


# ---- Navier (Lame): traction-free polynomial displacements on the sphere ----
LAM = 2.0


def navier_traction_free_family():
    """Null space of {(lambda div w I + mu (grad w + grad w^T)) n = 0 on |x| = R}
    over cubic displacements w (the auxiliary p = -(lambda + mu) div w)."""
    rng = np.random.default_rng(1)
    nw = len(MW)
    S = rng.standard_normal((240, 3))
    S = R * S / np.linalg.norm(S, axis=1)[:, None]
    n = S / R
    rows = []
    for i in range(3):
        T = np.zeros((len(S), 3 * nw))
        for c in range(3):     # lambda div w n_i
            T[:, c * nw:(c + 1) * nw] += LAM * _mono_vals(MW, S, tuple(int(k == c) for k in range(3))) * n[:, i:i + 1]
        for k in range(3):
            T[:, i * nw:(i + 1) * nw] += MU * _mono_vals(MW, S, tuple(int(m == k) for m in range(3))) * n[:, k:k + 1]
            T[:, k * nw:(k + 1) * nw] += MU * _mono_vals(MW, S, tuple(int(m == i) for m in range(3))) * n[:, k:k + 1]
        rows.append(T)
    M = np.vstack(rows)
    _, s, vt = np.linalg.svd(M)
    return vt[np.sum(s > 1e-10 * s[0]):]


@pytest.mark.parametrize("member", [0, 5])
def test_navier_jump_relations_exact_on_traction_free_pairs(member):
    null = navier_traction_free_family()
    assert null.shape[0] >= 6
    rng = np.random.default_rng(member)
    coefw = rng.standard_normal(null.shape[0]) @ null
    coef = np.concatenate([coefw, np.zeros(len(MP))])
    d = rng.standard_normal((25, 3))
    y = R * d / np.linalg.norm(d, axis=1)[:, None]
    n, T, K = geometry.frames(ki.sphere(R), y)
    w, gw, hw, _, _, _ = jets(coef, y)
    pi = -(LAM + MU) * np.einsum("ncc->n", gw)
    gpi = -(LAM + MU) * np.einsum("ncjc->nj", hw)
    f = -MU * np.einsum("ncjj->nc", hw) + gpi
    d1 = np.einsum("ncj,naj->nca", gw, T)
    gn = np.einsum("ncj,nj->nc", gw, n)
    d2 = np.zeros((len(y), 3, 3))
    for m, (a, b) in enumerate([(0, 0), (0, 1), (1, 1)]):
        d2[:, :, m] = np.einsum("ncjl,nj,nl->nc", hw, T[:, a], T[:, b]) - K[:, a, b][:, None] * gn
    A, q = jumps.first_order(n, T, d1, MU, LAM)
    assert np.abs(A - gw).max() < 1e-10 * max(1.0, np.abs(gw).max())
    assert np.abs(q - pi).max() < 1e-10 * max(1.0, np.abs(pi).max())
    L = jumps.second_order_system(n, T, K, MU, LAM)
    rhs = jumps.second_order_rhs(n, T, K, A, q, d2, f, MU, LAM)
    x = np.linalg.solve(L, rhs[..., None])[..., 0]
    for c in range(3):
        for m, (k, l) in enumerate(jumps.SYM):
            assert np.abs(x[:, 6 * c + m] - hw[:, c, k, l]).max() < 1e-9 * max(1.0, np.abs(hw).max())
    assert np.abs(x[:, 18:] - gpi).max() < 1e-9 * max(1.0, np.abs(gpi).max())


def test_navier_second_order_system_full_rank():
    rng = np.random.default_rng(2)
    for _ in range(4):
        Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        K = rng.standard_normal((1, 2, 2))
        K = K + np.swapaxes(K, 1, 2)
        L = jumps.second_order_system(Q[:, 0][None], np.stack([Q[:, 1], Q[:, 2]])[None], K, MU, LAM)[0]
        assert np.linalg.matrix_rank(L) == 21
