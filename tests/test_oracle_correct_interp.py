"""Pins of the oracle's RHS corrections (Sec. 4.3 items 1-4) and trace
interpolation (Sec. 4.4) with exact analytic jumps."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import correct, grid as gridmod, interp, mac
from tests import _fields


def _setup(N, geom):
    g = gridmod.Grid(N, -1.0, 1.0)
    cp, S = gridmod.control_points(g, geom)
    return g, cp, S


def _exact_jumps(cp):
    """Jumps of (u+, p+) = manufactured Stokes pair, (u-, p-) = 0."""
    x = cp.xyz
    rows = np.arange(cp.n)
    c = cp.comp - 1
    G, H = _fields.stokes_jets(x)
    J = np.zeros((cp.n, 12))
    J[:, 0] = ki.stokes_velocity(x)[rows, c]
    J[:, 1:4] = G[rows, c]
    J[:, 4:10] = H[rows, c]
    J[:, 10] = ki.stokes_pressure(x)
    J[:, 11] = np.cos(x.sum(-1))
    return J


def _piecewise(g, S):
    ue = []
    for c in (1, 2, 3):
        X = g.node_xyz(c, g.all_idx())
        ue.append(mac.zero_walls(np.where(S[c], ki.stokes_velocity(X)[..., c - 1], 0.0), c))
    X0 = g.node_xyz(0, g.all_idx())
    pe = np.where(S[0], ki.stokes_pressure(X0), 0.0)
    return ue, pe


def _residuals(N):
    g, cp, S = _setup(N, ki.sphere())
    J = _exact_jumps(cp)
    Cf, Cg = correct.corrections(g, cp, S, J, 1.0)
    f = []
    for c in (1, 2, 3):
        X = g.node_xyz(c, g.all_idx())
        ft = np.where(S[c], ki.stokes_forcing(X)[..., c - 1], 0.0)
        f.append(mac.zero_walls(ft + Cf[c - 1], c))
    ue, pe = _piecewise(g, S)
    Gp = mac.grad(pe, g.h)
    rmom = max(np.abs(mac.zero_walls(-mac.lap(ue[c], c + 1, g.h) + Gp[c] - f[c], c + 1)).max()
               for c in range(3))
    rdiv = np.abs(mac.div(ue, g.h) - Cg).max()
    u, p, _ = mac.interface_solve(f, Cg, 1.0, g.h)
    err = max(np.abs(u[c] - ue[c]).max() for c in range(3))
    return rmom, rdiv, err, (g, cp, S, u, J)


def test_corrected_truncation_and_solution_orders():
    """With exact jumps the corrected residual of the exact piecewise solution
    is O(h) at irregular nodes (item corrections are 'at least first order')
    and the discrete solution converges at second order (Sec. 4.3)."""
    r16, d16, e16, _ = _residuals(16)
    r32, d32, e32, _ = _residuals(32)
    assert r32 < 0.65 * r16                 # first order or better
    assert d32 < 0.65 * d16
    assert e16 / e32 > 3.5                  # second order
    # an uncorrected scheme is O(1/h^2)-wrong at irregular nodes
    g, cp, S = _setup(16, ki.sphere())
    ue, pe = _piecewise(g, S)
    X = g.node_xyz(1, g.all_idx())
    raw = np.abs(-mac.lap(ue[0], 1, g.h) + mac.grad(pe, g.h)[0]
                 - mac.zero_walls(np.where(S[1], ki.stokes_forcing(X)[..., 0], 0.0), 1)).max()
    assert raw > 20 * r16


def test_item4_sign_reading():
    """The continuity correction follows the generic rule (-(1/h) J for a cell
    in Omega whose face neighbour is outside).  With the printed '+' the
    divergence residual of the exact solution does not decrease."""
    g, cp, S = _setup(32, ki.sphere())
    J = _exact_jumps(cp)
    _, Cg = correct.corrections(g, cp, S, J, 1.0)
    ue, _ = _piecewise(g, S)
    D = mac.div(ue, g.h)
    good = np.abs(D - Cg).max()
    flipped = np.abs(D + Cg).max()
    assert good < 0.05 * flipped


def test_trace_exact_for_quadratics_with_consistent_jumps():
    """u+ = P (quadratic) inside, u- = P - Q outside (Q quadratic): with the
    jumps of Q the ten-node interpolation returns P(x) exactly."""
    g, cp, S = _setup(20, ki.star())
    rng = np.random.default_rng(4)
    P = rng.standard_normal((3, 10))
    Q = rng.standard_normal((3, 10))

    def quad(C, x):
        X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
        basis = np.stack([np.ones_like(X), X, Y, Z, 0.5 * X * X, 0.5 * Y * Y, 0.5 * Z * Z, Y * Z, X * Z, X * Y], -1)
        return basis @ C.T

    fields = []
    for c in (1, 2, 3):
        X = g.node_xyz(c, g.all_idx())
        fields.append(np.where(S[c], quad(P, X)[..., c - 1], quad(P - Q, X)[..., c - 1]))
    x = cp.xyz
    rows = np.arange(cp.n)
    c = cp.comp - 1
    J = np.zeros((cp.n, 12))
    Qc = Q[c]
    J[:, 0] = quad(Q, x)[rows, c]
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    J[:, 1] = Qc[:, 1] + Qc[:, 4] * X + Qc[:, 9] * Y + Qc[:, 8] * Z
    J[:, 2] = Qc[:, 2] + Qc[:, 5] * Y + Qc[:, 9] * X + Qc[:, 7] * Z
    J[:, 3] = Qc[:, 3] + Qc[:, 6] * Z + Qc[:, 8] * X + Qc[:, 7] * Y
    J[:, 4:10] = Qc[:, 4:10]
    tr = interp.trace(g, cp, S, fields, J)
    assert np.abs(tr - quad(P, x)[rows, c]).max() < 1e-11


def test_trace_second_order_on_solved_field():
    _, _, _, (g16, cp16, S16, u16, J16) = _residuals(16)
    _, _, _, (g32, cp32, S32, u32, J32) = _residuals(32)
    e16 = np.abs(interp.trace(g16, cp16, S16, u16, J16) - J16[:, 0]).max()
    e32 = np.abs(interp.trace(g32, cp32, S32, u32, J32) - J32[:, 0]).max()
    assert e16 / e32 > 3.0
