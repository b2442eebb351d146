"""Closed-form fields used by the oracle pins (test helpers, no method code)."""
import numpy as np

import kfbim_inputs as ki


def stokes_jets(x):
    """Gradient (n,3,3) and Hessian entries (n,3,6; order 11,22,33,23,13,12)
    of the manufactured velocity of kfbim_inputs."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    sx, cx, sy, cy, sz, cz = np.sin(X), np.cos(X), np.sin(Y), np.cos(Y), np.sin(Z), np.cos(Z)
    n = x.shape[0]
    G = np.zeros((n, 3, 3))
    H = np.zeros((n, 3, 6))
    G[:, 0] = np.stack([cx * cy * cz, -sx * sy * cz, -sx * cy * sz], -1)
    H[:, 0] = np.stack([-sx * cy * cz, -sx * cy * cz, -sx * cy * cz, sx * sy * sz, -cx * cy * sz, -cx * sy * cz], -1)
    G[:, 1] = np.stack([sx * sy * cz, -cx * cy * cz, cx * sy * sz], -1)
    H[:, 1] = np.stack([cx * sy * cz, cx * sy * cz, cx * sy * cz, cx * cy * sz, -sx * sy * sz, sx * cy * cz], -1)
    return G, H


def traction_free_W(x, R):
    """W = ((3R^2 - r^2) / (2R^2)) (-xz, yz, x^2 - y^2): divergence-free and
    traction-free (pressure 0) on the sphere |x| = R."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    g = (3 * R * R - (X * X + Y * Y + Z * Z)) / (2 * R * R)
    return np.stack([-X * Z * g, Y * Z * g, (X * X - Y * Y) * g], -1)


def traction_free_W_forcing(x, R, mu):
    """-mu Lap W = 7 mu (-xz, yz, x^2 - y^2) / R^2."""
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 7.0 * mu * np.stack([-X * Z, Y * Z, X * X - Y * Y], -1) / R ** 2


def component_values(field, cp):
    rows = np.arange(cp.n)
    return field(cp.xyz)[rows, cp.comp - 1]
