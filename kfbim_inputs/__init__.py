"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module holds no arithmetic of the method itself: only geometry
descriptors (plain parameters of analytic surfaces, or, for the CALLBACK kind,
a level set and its derivatives as functions of a point), closed-form
manufactured Stokes and Lame fields used as boundary data and forcing, the
paper's example fields, seeded divergence-free harmonic fields and seeded
random densities.  Each consumer evaluates control points, jumps and
everything else with its own code.

Workloads (all in the bounding box [-1, 1]^3, viscosity 1):
  * sphere: radius 0.5 centred at the origin, N = 32 (plain FP64 case);
  * star:   r(theta, phi) = 0.5 + 0.1 sin(3 theta) cos(4 phi) (theta = polar
            angle, phi = azimuth), N = 64 and N = 128 (headline case);
  * ellipsoid: semi-axes (0.6, 0.45, 0.35) under a seeded rotation (Navier).
Boundary data come from the divergence-free manufactured field
u = (sin x cos y cos z, -cos x sin y cos z, 0), p = sin(x + y + z).
"""
import math

import numpy as np

BOX = (-1.0, 1.0)


def sphere(radius=0.5, center=(0.0, 0.0, 0.0)):
    return {"kind": "sphere", "center": [float(c) for c in center], "radius": float(radius)}


def star(r0=0.5, eps=0.1, m=3, n=4, center=(0.0, 0.0, 0.0)):
    """Star surface r(theta, phi) = r0 + eps sin(m theta) cos(n phi)."""
    return {"kind": "star", "center": [float(c) for c in center], "r0": float(r0),
            "eps": float(eps), "m": int(m), "n": int(n)}


def callback_sphere(radius=0.5, center=(0.0, 0.0, 0.0)):
    """The sphere as a caller-supplied level set (CALLBACK geometry):
    F = |x - c| - R with the arithmetic, in the same order, of the built-in
    sphere, so that both give identical setups."""
    cx, cy, cz = (float(v) for v in center)
    R = float(radius)

    def F(x):
        d0, d1, d2 = x[0] - cx, x[1] - cy, x[2] - cz
        return math.sqrt(d0 * d0 + d1 * d1 + d2 * d2) - R

    def derivs(x):
        d = (x[0] - cx, x[1] - cy, x[2] - cz)
        r = math.sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2])
        e = [di / r for di in d]
        return e, [[((i == j) - e[i] * e[j]) / r for j in range(3)] for i in range(3)]

    return {"kind": "callback", "F": F, "derivs": derivs}


def peanut(a=0.3, b=0.38, center=(0.03, -0.02, 0.05)):
    """A non-convex CALLBACK geometry: the Cassini surface of revolution about
    the x axis, F = P Q - b^4 with P = |x - c - a e_x|^2 and
    Q = |x - c + a e_x|^2 (one component with a waist for a < b < a sqrt 2).
    grad F = Q grad P + P grad Q, Hess F = grad P grad Q^T + grad Q grad P^T
    + 2 (P + Q) I."""
    cx, cy, cz = (float(v) for v in center)
    a, b4 = float(a), float(b) ** 4

    def parts(x):
        X, Y, Z = x[0] - cx, x[1] - cy, x[2] - cz
        rho2 = Y * Y + Z * Z
        P = (X - a) ** 2 + rho2
        Q = (X + a) ** 2 + rho2
        return P, Q, (2 * (X - a), 2 * Y, 2 * Z), (2 * (X + a), 2 * Y, 2 * Z)

    def F(x):
        P, Q, _, _ = parts(x)
        return P * Q - b4

    def derivs(x):
        P, Q, gP, gQ = parts(x)
        g = [Q * gP[i] + P * gQ[i] for i in range(3)]
        H = [[gP[i] * gQ[j] + gQ[i] * gP[j] + (2 * (P + Q) if i == j else 0.0) for j in range(3)]
             for i in range(3)]
        return g, H

    return {"kind": "callback", "F": F, "derivs": derivs}


def torus(a=0.35, c=0.7, center=(0.0, 0.0, 0.0)):
    """Torus (c - sqrt(x^2 + y^2))^2 + z^2 = a^2 about the z axis."""
    return {"kind": "torus", "center": [float(v) for v in center], "a": float(a), "c": float(c)}


def seeded_rotation(seed):
    """Rotation from the QR factorisation of a seeded Gaussian 3x3 matrix,
    columns sign-fixed by diag(R) > 0 and det = +1."""
    rng = np.random.default_rng(seed)
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))[None, :]
    if np.linalg.det(q) < 0:
        q[:, 2] = -q[:, 2]
    return q


def ellipsoid(axes=(0.6, 0.45, 0.35), rotation=None, center=(0.0, 0.0, 0.0)):
    rot = np.eye(3) if rotation is None else np.asarray(rotation, dtype=np.float64)
    return {"kind": "ellipsoid", "center": [float(c) for c in center],
            "axes": [float(a) for a in axes], "rotation": rot.reshape(-1).tolist()}


def grid(N, lo=BOX[0], hi=BOX[1]):
    return {"N": int(N), "lo": float(lo), "hi": float(hi)}


# ---------------------------------------------------------------- workloads
WORKLOADS = {
    "sphere32": (sphere(), grid(32)),
    "star64": (star(), grid(64)),
    "star128": (star(), grid(128)),
    # Navier (Lame mu = 1, lambda = 2) on the rotated ellipsoid; data: lame_*
    "ell128_navier": (ellipsoid((0.6, 0.45, 0.35), seeded_rotation(3)), grid(128)),
}
NAVIER_WORKLOADS = {"ell128_navier"}


# ------------------------------------------------- manufactured Stokes field
def stokes_velocity(x):
    """u = (sin x cos y cos z, -cos x sin y cos z, 0); x has shape (..., 3)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u1 = np.sin(X) * np.cos(Y) * np.cos(Z)
    u2 = -np.cos(X) * np.sin(Y) * np.cos(Z)
    u3 = np.zeros_like(X)
    return np.stack([u1, u2, u3], axis=-1)


def stokes_pressure(x):
    x = np.asarray(x, dtype=np.float64)
    return np.sin(x[..., 0] + x[..., 1] + x[..., 2])


def stokes_forcing(x, mu=1.0):
    """f = -mu Lap u + grad p for the manufactured pair above."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    c = np.cos(X + Y + Z)
    f1 = 3.0 * mu * np.sin(X) * np.cos(Y) * np.cos(Z) + c
    f2 = -3.0 * mu * np.cos(X) * np.sin(Y) * np.cos(Z) + c
    f3 = c
    return np.stack([f1, f2, f3], axis=-1)


# --------------------------------------------------------- seeded densities
def random_density(n, seed):
    """Seeded N(0,1) values, one per control point (for linear-map parity)."""
    return np.random.default_rng(seed).standard_normal(n)


def smooth_field(seed, degree=3):
    """Seeded smooth vector field x -> (3,) as a sum of low-frequency
    trigonometric modes with N(0,1)/(1+l)^2 amplitudes (l = mode order)."""
    rng = np.random.default_rng(seed)
    modes = []
    for comp in range(3):
        for l in range(degree + 1):
            for _ in range(3):
                k = rng.standard_normal(3)
                k = k / np.linalg.norm(k) * (l + 0.5)
                amp = rng.standard_normal() / (1.0 + l) ** 2
                ph = rng.uniform(0, 2 * np.pi)
                modes.append((comp, k, amp, ph))

    def field(x):
        x = np.asarray(x, dtype=np.float64)
        out = np.zeros(x.shape[:-1] + (3,))
        for comp, k, amp, ph in modes:
            out[..., comp] += amp * np.cos(x @ k + ph)
        return out

    return field


def harmonic_curl_field(seed, degree=6, scale=0.5):
    """Seeded divergence-free boundary-data field u = curl A, A^(c) a random
    solid-harmonic expansion of degree <= `degree` in x / scale.  Degree l
    contributes 2l + 1 terms Re (v . x/scale)^l with isotropic null vectors
    v = e1 + i e2 (e1, e2 orthonormal, seeded), each with an N(0,1)/(1+l)^2
    coefficient; such powers span the degree-l solid harmonics.  The curl
    makes the net flux through any closed surface zero, the solvability
    condition of interior Stokes Dirichlet data.  Returns x -> (..., 3)."""
    rng = np.random.default_rng(seed)
    terms = []                                   # (component, l, v, coefficient)
    for comp in range(3):
        for l in range(1, degree + 1):           # l = 0 is constant: no curl
            for _ in range(2 * l + 1):
                q, _r = np.linalg.qr(rng.standard_normal((3, 3)))
                v = q[:, 0] + 1j * q[:, 1]
                terms.append((comp, l, v, rng.standard_normal() / (1.0 + l) ** 2))

    def field(x):
        x = np.asarray(x, dtype=np.float64) / scale
        dA = np.zeros(x.shape[:-1] + (3, 3))      # dA[..., c, j] = d_j A^(c) (per unit x/scale)
        for comp, l, v, a in terms:
            w = (x @ v) ** (l - 1)
            dA[..., comp, :] += a * l * np.real(w[..., None] * v)
        out = np.empty(x.shape[:-1] + (3,))
        out[..., 0] = dA[..., 2, 1] - dA[..., 1, 2]
        out[..., 1] = dA[..., 0, 2] - dA[..., 2, 0]
        out[..., 2] = dA[..., 1, 0] - dA[..., 0, 1]
        return out / scale

    return field


# ------------------------------ paper Example 5.1 (sphere r = 1, box +-1.2)
def example51_velocity(x):
    """Example 5.1's velocity with u^(2)'s y^2(1 - y^2) read as y^2(2 - y^2):
    the printed field has div u = -2y; this reading is divergence-free."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u1 = X**2 * (2 - X**2) + 4 * X * Y * (X**2 + Y**2 - 1) + Z**2 * (3 * Z**2 - 6 * X**2 - 2)
    u2 = X**2 * (3 * X**2 - 6 * Y**2 - 1) + Y**2 * (2 - Y**2)
    u3 = 4 * Z * X * (Z**2 + X**2 - 1)
    return np.stack([u1, u2, u3], axis=-1)


def example51_pressure(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return 8 * Y * (3 * X**2 - Y**2) + 8 * X * (3 * Z**2 - X**2)


def example51_forcing(x, mu=1.0):
    """-mu Lap u + grad p for the field above (expanded by hand from the
    polynomials): Lap u = (24z^2 - 24x^2 + 48xy, 24x^2 - 24y^2 + 2, 48xz) and
    grad p = (24z^2 - 24x^2 + 48xy, 24x^2 - 24y^2, 48xz)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    lap = np.stack([24 * Z**2 - 24 * X**2 + 48 * X * Y, 24 * X**2 - 24 * Y**2 + 2, 48 * X * Z], -1)
    gp = np.stack([24 * Z**2 - 24 * X**2 + 48 * X * Y, 24 * X**2 - 24 * Y**2, 48 * X * Z], -1)
    return -mu * lap + gp


# ---------------- paper Example 5.2 (ellipsoid x^2 + y^2/0.64 + z^2/0.36 = 1)
def example52_geometry():
    return ellipsoid(axes=(1.0, 0.8, 0.6))


def example52_velocity(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u1 = 2 * X**3 * Y / 3 - Z**2 * X**2 + np.exp(Z) + np.sin(np.pi * Z)
    u2 = -X**2 * Y**2 + np.cos(np.pi * X)
    u3 = 2 * Z**3 * X / 3 + np.exp(X) + np.sin(np.pi * X)
    return np.stack([u1, u2, u3], axis=-1)


def example52_pressure(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return (X - 1) ** 3 * (Y - 1) ** 3 * (Z - 1) ** 3


def example52_forcing(x, mu=1.0):
    """-mu Lap u + grad p, with
    Lap u = (4xy - 2x^2 - 2z^2 + e^z - pi^2 sin(pi z), -2x^2 - 2y^2 - pi^2 cos(pi x),
             4xz + e^x - pi^2 sin(pi x))."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    pi2 = np.pi ** 2
    lap = np.stack([4 * X * Y - 2 * X**2 - 2 * Z**2 + np.exp(Z) - pi2 * np.sin(np.pi * Z),
                    -2 * X**2 - 2 * Y**2 - pi2 * np.cos(np.pi * X),
                    4 * X * Z + np.exp(X) - pi2 * np.sin(np.pi * X)], -1)
    a, b, c = X - 1, Y - 1, Z - 1
    gp = np.stack([3 * a**2 * b**3 * c**3, 3 * a**3 * b**2 * c**3, 3 * a**3 * b**3 * c**2], -1)
    return -mu * lap + gp


# ------------------------------- paper Example 5.3 (torus a = 0.35, c = 0.7)
def example53_geometry():
    return torus(0.35, 0.7)


def example53_velocity(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    u1 = (-4 * X * Y * (1 - X**2 - Y**2) - X**2 * (X**2 + 6 * Z**2 - 2) + Z**2 * (3 * Z**2 - 2)
          + np.exp(np.cos(Y)) + np.exp(np.sin(Z)))
    u2 = X**2 * (3 * X**2 - 6 * Y**2 - 2) - Y**2 * (Y**2 - 2) + np.exp(np.sin(X))
    u3 = -4 * (1 - X**2 - Z**2) * X * Z + np.exp(np.cos(X))
    return np.stack([u1, u2, u3], axis=-1)


def example53_pressure(x):
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    return np.exp(1 - Y**2 - Z**3) * np.sin(X**2 + 1)


def example53_forcing(x, mu=1.0):
    """-mu Lap u + grad p; the exponential terms of Lap u come from
    (e^{cos t})'' = e^{cos t} (sin^2 t - cos t), (e^{sin t})'' = e^{sin t} (cos^2 t - sin t)."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]

    def ecos2(t):
        return np.exp(np.cos(t)) * (np.sin(t) ** 2 - np.cos(t))

    def esin2(t):
        return np.exp(np.sin(t)) * (np.cos(t) ** 2 - np.sin(t))

    lap = np.stack([-24 * X**2 + 48 * X * Y + 24 * Z**2 + ecos2(Y) + esin2(Z),
                    24 * X**2 - 24 * Y**2 + esin2(X),
                    48 * X * Z + ecos2(X)], -1)
    E = np.exp(1 - Y**2 - Z**3)
    gp = np.stack([2 * X * E * np.cos(X**2 + 1), -2 * Y * E * np.sin(X**2 + 1),
                   -3 * Z**2 * E * np.sin(X**2 + 1)], -1)
    return -mu * lap + gp


# ------------------------- paper Examples 5.4-5.6 (Navier, Lame data E, nu)
class _Jet:
    """Value, gradient (..., 3) and Hessian (..., 3, 3) of a scalar field, with
    the sum, product and chain rules: enough to differentiate the examples'
    fields exactly."""

    def __init__(self, v, g, H):
        self.v, self.g, self.H = v, g, H

    @staticmethod
    def coord(X, k):
        g = np.zeros(X.shape)
        g[..., k] = 1.0
        return _Jet(X[..., k].copy(), g, np.zeros(X.shape + (3,)))

    @staticmethod
    def const(X, c):
        return _Jet(np.full(X.shape[:-1], float(c)), np.zeros(X.shape), np.zeros(X.shape + (3,)))

    def __add__(self, o):
        return _Jet(self.v + o.v, self.g + o.g, self.H + o.H)

    def __mul__(self, o):
        if not isinstance(o, _Jet):
            return _Jet(self.v * o, self.g * o, self.H * o)
        outer = self.g[..., :, None] * o.g[..., None, :]
        return _Jet(self.v * o.v, self.g * o.v[..., None] + o.g * self.v[..., None],
                    self.H * o.v[..., None, None] + o.H * self.v[..., None, None] + outer
                    + np.swapaxes(outer, -1, -2))

    def apply(self, f, f1, f2):
        """Chain rule for t -> f(t) with derivatives f1, f2."""
        a, b = f1(self.v), f2(self.v)
        return _Jet(f(self.v), self.g * a[..., None],
                    self.H * a[..., None, None] + b[..., None, None] * self.g[..., :, None] * self.g[..., None, :])


def _sin(j):
    return j.apply(np.sin, np.cos, lambda t: -np.sin(t))


def _cos(j):
    return j.apply(np.cos, lambda t: -np.sin(t), lambda t: -np.cos(t))


def _exp(j):
    return j.apply(np.exp, np.exp, np.exp)


def lame_from_young(E, nu):
    """(mu, lambda) from Young's modulus and Poisson's ratio."""
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def _navier_jets(key, X):
    X = np.asarray(X, dtype=np.float64)
    x, y, z = (_Jet.coord(X, k) for k in range(3))
    r2 = x * x + y * y + z * z
    if key == "5.4":
        S = _sin(r2 * (2.0 * np.pi))
        return [S * _cos(y * 2.0) * _cos(z), S * _cos(x) * _cos(x + z), S * _cos(x * np.pi) * _cos(y)]
    if key == "5.5":
        base = r2 + _Jet.const(X, -4.0) + _cos(x) * _cos(y) * _cos(z)
        return [base, base + x * y, base + y * z]
    # 5.6
    one = _Jet.const(X, 1.0)
    return [_exp(one + y * y * -1.0 + z * z * -1.0) * _sin(x * x * 3.0 + _Jet.const(X, 2.0)),
            _sin(one + r2 * -1.0), x * x * 3.0 + y * y * 2.0 + z * z]


NAVIER_EXAMPLES = {
    # key: (geometry, E, nu)
    "5.4": (lambda: sphere(1.0), 1000.0, 0.1),
    "5.5": (lambda: ellipsoid(axes=(1.0, 0.8, 0.6)), 4000.0, 0.05),
    "5.6": (lambda: torus(0.35, 0.7), 2000.0, 0.4),
}


def navier_example_displacement(key, X):
    return np.stack([j.v for j in _navier_jets(key, X)], axis=-1)


def navier_example_forcing(key, X):
    """f = -mu Lap u - (lambda + mu) grad(div u) with (mu, lambda) of the example."""
    _, E, nu = NAVIER_EXAMPLES[key]
    mu, lam = lame_from_young(E, nu)
    J = _navier_jets(key, X)
    lap = np.stack([np.trace(j.H, axis1=-2, axis2=-1) for j in J], axis=-1)
    graddiv = sum(J[i].H[..., :, i] for i in range(3))
    return -mu * lap - (lam + mu) * graddiv


# ------------------------------------ manufactured Lame displacement (Navier)
LAME_MU, LAME_LAMBDA = 1.0, 2.0


def lame_jets(x):
    """u_i = exp(x + y + z) sin(i + x y), i = 1..3: values (n,3), gradients
    (n,3,3) and Hessians (n,3,3,3) by the product rule."""
    x = np.asarray(x, dtype=np.float64)
    X, Y, Z = x[..., 0], x[..., 1], x[..., 2]
    E = np.exp(X + Y + Z)
    u = np.zeros(x.shape[:-1] + (3,))
    G = np.zeros(x.shape[:-1] + (3, 3))
    H = np.zeros(x.shape[:-1] + (3, 3, 3))
    for i in range(3):
        S = np.sin(i + 1 + X * Y)
        C = np.cos(i + 1 + X * Y)
        u[..., i] = E * S
        G[..., i, 0] = E * (S + Y * C)
        G[..., i, 1] = E * (S + X * C)
        G[..., i, 2] = E * S
        H[..., i, 0, 0] = E * (S + 2 * Y * C - Y * Y * S)
        H[..., i, 1, 1] = E * (S + 2 * X * C - X * X * S)
        H[..., i, 2, 2] = E * S
        H[..., i, 0, 1] = H[..., i, 1, 0] = E * (S + X * C + Y * C + C - X * Y * S)
        H[..., i, 0, 2] = H[..., i, 2, 0] = E * (S + Y * C)
        H[..., i, 1, 2] = H[..., i, 2, 1] = E * (S + X * C)
    return u, G, H


def lame_displacement(x):
    return lame_jets(x)[0]


def lame_forcing(x, mu=LAME_MU, lam=LAME_LAMBDA):
    """f = -mu Lap u - (lambda + mu) grad(div u) (Eq. Navier)."""
    _, _, H = lame_jets(x)
    lap = np.einsum("...ijj->...i", H)
    graddiv = np.einsum("...iij->...j", H)
    return -mu * lap - (lam + mu) * graddiv


def lame_pressure(x, mu=LAME_MU, lam=LAME_LAMBDA):
    """The auxiliary unknown p = -(lambda + mu) div u of the unified form."""
    _, G, _ = lame_jets(x)
    return -(lam + mu) * np.einsum("...ii->...", G)
