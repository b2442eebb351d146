"""Analytic level sets F (Omega = {F <= 0}), or a caller-supplied one (kind
"callback": F and its derivatives as Python functions of a point), gradients
and Hessians, and the
local frame at surface points (Alg. 1 step 1: "compute tangential and normal
unit directions").  The outward normal is n = grad F / |grad F| (Sec. 2).

Curvature tensor in the tangent frame: K_ab = tau_a^T (Hess F) tau_b / |grad F|.
With this sign, a sphere of radius R has K = I / R and the surface near y is
the graph y + s tau_1 + t tau_2 - 1/2 (s,t) K (s,t)^T n + O(3).
"""
import numpy as np


# Sphere |x - c| = R, the domain of Examples 5.1 and 5.4; Omega = {F < 0} (Sec. 2).
def _sphere(geom, X):
    c = np.asarray(geom["center"])
    d = X - c
    r = np.sqrt(np.sum(d * d, axis=-1))
    F = r - geom["radius"]
    e = d / r[..., None]
    G = e
    H = (np.eye(3) - e[..., :, None] * e[..., None, :]) / r[..., None, None]
    return F, G, H


# Ellipsoid in a rotated body frame, the domain of Examples 5.2 and 5.5 (Sec. 2 for F).
def _ellipsoid(geom, X):
    c = np.asarray(geom["center"])
    Q = np.asarray(geom["rotation"]).reshape(3, 3)
    a = np.asarray(geom["axes"])
    xi = (X - c) @ Q            # local coordinates xi = Q^T (x - c)
    F = np.sum((xi / a) ** 2, axis=-1) - 1.0
    D = np.diag(2.0 / a ** 2)
    G = (xi * (2.0 / a ** 2)) @ Q.T
    Hm = Q @ D @ Q.T
    H = np.broadcast_to(Hm, X.shape[:-1] + (3, 3)).copy()
    return F, G, H


# Star-shaped surface of the benchmark configuration (not one of the paper's examples); F as in Sec. 2.
def _star(geom, X):
    """F = rho - R(theta, phi), theta = polar angle from +z, phi = azimuth.

    Gradient and Hessian by the chain rule through the spherical coordinates;
    grad rho = e_rho, grad theta = e_theta / rho, grad phi = e_phi / (rho sin theta).
    """
    c = np.asarray(geom["center"])
    r0, eps, m, n = geom["r0"], geom["eps"], geom["m"], geom["n"]
    d = X - c
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    s = np.sqrt(x * x + y * y)
    rho = np.sqrt(x * x + y * y + z * z)
    th = np.arctan2(s, z)
    ph = np.arctan2(y, x)
    st, ct = np.sin(th), np.cos(th)
    sp, cp = np.sin(ph), np.cos(ph)
    sm, cm = np.sin(m * th), np.cos(m * th)
    sn, cn = np.sin(n * ph), np.cos(n * ph)
    R = r0 + eps * sm * cn
    Rt = eps * m * cm * cn
    Rp = -eps * n * sm * sn
    Rtt = -eps * m * m * sm * cn
    Rtp = -eps * m * n * cm * sn
    Rpp = -eps * n * n * sm * cn
    F = rho - R

    er = np.stack([st * cp, st * sp, ct], axis=-1)
    et = np.stack([ct * cp, ct * sp, -st], axis=-1)
    ep = np.stack([-sp, cp, np.zeros_like(sp)], axis=-1)
    gth = et / rho[..., None]
    gph = ep / (rho * st)[..., None]
    G = er - Rt[..., None] * gth - Rp[..., None] * gph

    def outer(a, b):
        return a[..., :, None] * b[..., None, :]

    I = np.eye(3)
    H_rho = (I - outer(er, er)) / rho[..., None, None]
    H_th = (-outer(er, et) - outer(et, er) + (ct / st)[..., None, None] * outer(ep, ep)) \
        / (rho * rho)[..., None, None]
    w = st[..., None] * er + ct[..., None] * et
    H_ph = -(outer(w, ep) + outer(ep, w)) / (rho * rho * st * st)[..., None, None]
    H = (H_rho - Rt[..., None, None] * H_th - Rp[..., None, None] * H_ph
         - Rtt[..., None, None] * outer(gth, gth)
         - Rtp[..., None, None] * (outer(gth, gph) + outer(gph, gth))
         - Rpp[..., None, None] * outer(gph, gph))
    return F, G, H


def _torus(geom, X):
    """F = (c - s)^2 + z^2 - a^2 with s the distance from the z axis
    (Example 5.3's domain is F < 0); derivatives written out in x, y, z."""
    cen = np.asarray(geom["center"])
    a, c = geom["a"], geom["c"]
    d = X - cen
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    s = np.sqrt(x * x + y * y)
    F = (c - s) ** 2 + z * z - a * a
    G = np.stack([-2.0 * (c - s) * x / s, -2.0 * (c - s) * y / s, 2.0 * z], axis=-1)
    H = np.zeros(X.shape[:-1] + (3, 3))
    H[..., 0, 0] = 2.0 * x * x / (s * s) - 2.0 * (c - s) * y * y / s ** 3
    H[..., 1, 1] = 2.0 * y * y / (s * s) - 2.0 * (c - s) * x * x / s ** 3
    H[..., 0, 1] = H[..., 1, 0] = 2.0 * x * y / (s * s) + 2.0 * (c - s) * x * y / s ** 3
    H[..., 2, 2] = 2.0
    return F, G, H


# Sec. 2 with a caller-supplied level set: F, gradient and Hessian point by point.
def _callback(geom, X):
    """Evaluate geom["F"](x) and geom["derivs"](x) -> (gradient, Hessian) at
    every point of X (..., 3), one point at a time."""
    pts = X.reshape(-1, 3)
    F = np.empty(len(pts))
    G = np.empty((len(pts), 3))
    H = np.empty((len(pts), 3, 3))
    for k, x in enumerate(pts):
        F[k] = geom["F"](tuple(x))
        g, h = geom["derivs"](tuple(x))
        G[k] = g
        H[k] = np.asarray(h).reshape(3, 3)
    return F.reshape(X.shape[:-1]), G.reshape(X.shape), H.reshape(X.shape + (3,))


_KINDS = {"sphere": _sphere, "ellipsoid": _ellipsoid, "star": _star, "torus": _torus,
          "callback": _callback}


# Sec. 2: Gamma is the zero set of F and Omega = {F < 0}; Alg. 1 step 1.
def level_set(geom, X):
    """Return (F, grad F, Hess F) at points X of shape (..., 3)."""
    X = np.asarray(X, dtype=np.float64)
    return _KINDS[geom["kind"]](geom, X)


# Sec. 2: the value of F alone.
def level_value(geom, X):
    if geom["kind"] == "callback":
        X = np.asarray(X, dtype=np.float64)
        return np.array([geom["F"](tuple(x)) for x in X.reshape(-1, 3)]).reshape(X.shape[:-1])
    return level_set(geom, X)[0]


# Alg. 1 step 1 (tangential and normal unit directions); the curvature
# enters the second-order jumps of Sec. 4.3.
def frames(geom, X):
    """Outward normal n, tangents tau_1, tau_2 and curvature tensor K (2x2)
    at surface points X (..., 3).

    tau_1 is the normalised projection of the coordinate axis least aligned
    with n (first index on ties); tau_2 = n x tau_1.  Every result of the
    method is independent of this choice up to rounding (the jump relations
    and the tangent-plane fit are covariant under rotations of the frame).
    """
    _, G, H = level_set(geom, X)
    g = np.linalg.norm(G, axis=-1)
    n = G / g[..., None]
    m = np.argmin(np.abs(n), axis=-1)
    e = np.eye(3)[m]
    t1 = e - np.sum(e * n, axis=-1)[..., None] * n
    t1 = t1 / np.linalg.norm(t1, axis=-1)[..., None]
    t2 = np.cross(n, t1)
    T = np.stack([t1, t2], axis=-2)                      # (..., 2, 3)
    K = np.einsum("...ai,...ij,...bj->...ab", T, H, T) / g[..., None, None]
    return n, T, K
