"""Pins of the oracle's pressure trace (interp.pressure_trace): a smooth
pressure with no jump is interpolated to second order; a pressure whose
exterior values are shifted by a constant jump c (with [p] = c in J) gives
exactly the trace of the unshifted field; and a linear field is reproduced
exactly (trilinear interpolation is exact on it)."""
import numpy as np

import kfbim_inputs as ki
from oracle import grid as gridmod, interp


def _setup(N):
    g = gridmod.Grid(N, -1.0, 1.0)
    cp, S = gridmod.control_points(g, ki.sphere())
    X = g.node_xyz(0, g.all_idx())
    return g, cp, S, X


def field(x):
    return np.sin(x[..., 0] + 2 * x[..., 1]) * np.cos(x[..., 2]) + x[..., 0] ** 2


def test_linear_field_exact_and_jump_shift_exact():
    g, cp, S, X = _setup(32)
    lin = 1.0 + 2.0 * X[..., 0] - 0.5 * X[..., 1] + 3.0 * X[..., 2]
    J = np.zeros((cp.n, 12))
    got = interp.pressure_trace(g, cp, S, lin, J)
    want = 1.0 + 2.0 * cp.xyz[:, 0] - 0.5 * cp.xyz[:, 1] + 3.0 * cp.xyz[:, 2]
    assert np.abs(got - want).max() < 1e-13
    c = 0.7
    shifted = np.where(S[0], lin, lin - c)            # p^- = p^+ - c outside Omega
    J[:, 10] = c
    assert np.abs(interp.pressure_trace(g, cp, S, shifted, J) - got).max() < 1e-13


def test_smooth_field_second_order():
    errs = []
    for N in (32, 64):
        g, cp, S, X = _setup(N)
        got = interp.pressure_trace(g, cp, S, field(X), np.zeros((cp.n, 12)))
        errs.append(np.abs(got - field(cp.xyz)).max())
    assert errs[0] / errs[1] > 3.5, errs
