"""Jumps of the solution and its derivatives at the control points, from the
interface conditions IUS-1..IUS-4 (Sec. 4.1 remark; Sec. 4.3 states that they
follow from these equations but omits the derivation, which is restated here).

Notation at a surface point y with outward normal n, tangents tau_1, tau_2 and
curvature K (geometry.py):  A = [grad u] (A_cj = [d_j u^(c)]), q = [p],
H^(c) = [Hess u^(c)], s = [grad p], d_a phi = derivative of the density along
tau_a, d_ab phi = second derivative in the tangent-plane (Monge) coordinates.

First order (10 equations, 10 unknowns):
  A tau_a = d_a phi  (a = 1, 2)      tangential derivatives of [u] = phi (IUS-3)
  tr A = 0                            [div u] = 0 (IUS-2)
  (-q I + mu (A + A^T)) n = 0         [sigma n] = 0 (IUS-4)
  =>  A = sum_a d_a phi tau_a^T + (A n) n^T,
      A n = -D n - sum_a (n . d_a phi) tau_a,  D = sum_a tau_a . d_a phi,
      q = -2 mu D.
Second order (21 equations for the 18 entries of H^(1..3) and the 3 of s):
  (i)   tau_a^T H^(c) tau_b = d_ab phi^(c) + K_ab (A n)_c      (9; surface
        second derivative of [u^(c)] = phi^(c) along the curved surface)
  (ii)  sum_c H^(c)_{c j} = 0                                  (3; grad [div u] = 0)
  (iii) -mu tr H^(c) + s_c = [f~_c]                            (3; IUS-1)
  (iv)  tau_a . grad([sigma]) n + [sigma] d_a n = 0,  d_a n = sum_b K_ab tau_b
                                                               (6; d/ds_a of IUS-4)

Navier (Lame) variant (Sec. 2 Eq. Navier, unified form I-E of the Sec. 4.1
remark): p = -(lambda + mu) div u, div u + c p = 0 with c = 1/(lambda + mu), and
the interface traction is the elastic one, sigma = lambda (div u) I +
mu (grad u + grad u^T) = -kappa p I + mu (grad u + grad u^T), kappa = lambda c
(reading: the traction of the Navier double layer, Sec. 3, is used in IUS-4).
First order: A n = -(lambda / (lambda + 2 mu)) D n - sum_a (n . d_a phi) tau_a,
q = -(lambda + mu) tr A.  Second order: (ii) gains + c s_j, (iv) uses kappa s
and [sigma] = -kappa q I + mu (A + A^T).  Stokes is c = 0, kappa = 1.

Surface derivatives of each density component (the paper defers this step to
earlier work; our reading, parity unpinned): a weighted least-squares
quadratic in the tangent-plane coordinates (s, t) = ((z - y).tau_1,
(z - y).tau_2) over the points z of X_c' whose segment midpoints lie within
3h of y's (integer test on half-spacing keys), weights exp(-|z - y|^2 / h^2).
"""
import numpy as np
from scipy.spatial import cKDTree

from . import geometry, grid as gridmod

FIT_R2 = 36          # squared radius in (h/2)^2 units: 3h
FIT_SIGMA2 = 1.0     # Gaussian weight exp(-|z - y|^2 / (FIT_SIGMA2 h^2))
MIN_NEIGHBOURS = 12


# Sec. 4.3: the density's surface derivatives need neighbouring control points (our fit, parity unpinned).
def neighbour_lists(cp, primary):
    """For each point y and component c' the indices of the primary points of
    X_c' within the fit radius (exact integer test on fine keys)."""
    kint = gridmod.fine_keys(cp)
    keys = kint.astype(np.float64)
    out = []
    for cc in (1, 2, 3):
        cand = np.nonzero((cp.comp == cc) & primary)[0]
        tree = cKDTree(keys[cand])
        lists = tree.query_ball_point(keys, r=np.sqrt(FIT_R2) + 0.5)
        res = []
        for y, lst in enumerate(lists):
            lst = cand[np.array(sorted(lst), dtype=np.int64)]
            d2 = np.sum((kint[lst] - kint[y]) ** 2, axis=1)
            res.append(lst[d2 <= FIT_R2])
        out.append(res)
    return out


# Sec. 4.3: surface derivatives of the density by a least-squares fit (our reading, parity unpinned).
def surface_derivatives(cp, frames, nbrs, phi, h):
    """Fitted (value, d_1, d_2, d_11, d_12, d_22) of each phi^(c') at every
    point: array (n, 3, 6).  phi holds values at all points; only the
    neighbours listed in nbrs (primary points) enter the fit."""
    n_pts = cp.n
    n, T, K = frames
    out = np.zeros((n_pts, 3, 6))
    for cc in range(3):
        lists = nbrs[cc]
        m = max(len(l) for l in lists)
        idx = np.zeros((n_pts, m), dtype=np.int64)
        w = np.zeros((n_pts, m))
        for y, l in enumerate(lists):
            if len(l) < MIN_NEIGHBOURS:
                raise ValueError("too few neighbours for the surface fit")
            idx[y, :len(l)] = l
            w[y, :len(l)] = 1.0
        d = (cp.xyz[idx] - cp.xyz[:, None, :]) / h                 # (n, m, 3)
        s = np.einsum("nmk,nk->nm", d, T[:, 0, :])
        t = np.einsum("nmk,nk->nm", d, T[:, 1, :])
        w = w * np.exp(-np.sum(d * d, axis=-1) / FIT_SIGMA2)
        V = np.stack([np.ones_like(s), s, t, s * s, s * t, t * t], axis=-1)   # (n, m, 6)
        A = np.einsum("nmi,nm,nmj->nij", V, w, V)
        b = np.einsum("nmi,nm,nm->ni", V, w, phi[idx])
        a = np.linalg.solve(A, b[..., None])[..., 0]
        out[:, cc, 0] = a[:, 0]
        out[:, cc, 1] = a[:, 1] / h
        out[:, cc, 2] = a[:, 2] / h
        out[:, cc, 3] = 2.0 * a[:, 3] / h ** 2
        out[:, cc, 4] = a[:, 4] / h ** 2
        out[:, cc, 5] = 2.0 * a[:, 5] / h ** 2
    return out


SYM = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]   # H entry order 11,22,33,23,13,12


# Index helper for the Hessian unknowns of Sec. 4.3.
def _hidx(k, l):
    return SYM.index((min(k, l), max(k, l)))


# Sec. 4.1 remark, IUS-2..IUS-4: the first-order jumps.
def first_order(n, T, dphi, mu, lam=None):
    """A (n,3,3) and q (n,) from the tangential derivatives dphi (n,3,2).
    lam = None: Stokes; else the Navier (Lame) relations."""
    dphi_t = np.swapaxes(dphi, 1, 2)                             # (n, 2, 3): d_a phi
    D = np.einsum("nai,nai->n", T, dphi_t)
    nd = np.einsum("ni,nai->na", n, dphi_t)
    Ann = -D if lam is None else -D * lam / (lam + 2.0 * mu)
    An = Ann[:, None] * n - np.einsum("na,nai->ni", nd, T)
    A = np.einsum("nai,naj->nij", dphi_t, T) + An[:, :, None] * n[:, None, :]
    q = -2.0 * mu * D if lam is None else -(lam + mu) * (Ann + D)
    return A, q


# Sec. 4.3: second-order jumps from IUS-1..IUS-4 and their surface derivatives.
def second_order_system(n, T, K, mu, lam=None):
    """Matrix L (n, 21, 21) of equations (i)-(iv) acting on
    x = (H^(1) (6), H^(2) (6), H^(3) (6), s (3)); lam = None for Stokes."""
    c = 0.0 if lam is None else 1.0 / (lam + mu)
    kap = 1.0 if lam is None else lam / (lam + mu)
    npt = len(n)
    L = np.zeros((npt, 21, 21))
    row = 0
    for cc in range(3):                                  # (i)
        for (a, b) in [(0, 0), (0, 1), (1, 1)]:
            for k in range(3):
                for l in range(3):
                    L[:, row, 6 * cc + _hidx(k, l)] += T[:, a, k] * T[:, b, l]
            row += 1
    for j in range(3):                                   # (ii)
        for cc in range(3):
            L[:, row, 6 * cc + _hidx(cc, j)] += 1.0
        L[:, row, 18 + j] += c
        row += 1
    for cc in range(3):                                  # (iii)
        for k in range(3):
            L[:, row, 6 * cc + _hidx(k, k)] += -mu
        L[:, row, 18 + cc] += 1.0
        row += 1
    for a in range(2):                                   # (iv)
        for i in range(3):
            for j in range(3):
                L[:, row, 18 + j] += -kap * T[:, a, j] * n[:, i]
                for k in range(3):
                    L[:, row, 6 * i + _hidx(k, j)] += mu * T[:, a, j] * n[:, k]
                    L[:, row, 6 * k + _hidx(i, j)] += mu * T[:, a, j] * n[:, k]
            row += 1
    return L


# Sec. 4.3: right-hand side of the second-order jump system.
def second_order_rhs(n, T, K, A, q, d2phi, fy, mu, lam=None):
    """Right-hand side (n, 21) of (i)-(iv); d2phi (n, 3, 3) = (d_11, d_12, d_22)
    per component, fy (n, 3) = [f~] at the point; lam = None for Stokes."""
    kap = 1.0 if lam is None else lam / (lam + mu)
    npt = len(n)
    rhs = np.zeros((npt, 21))
    An = np.einsum("nij,nj->ni", A, n)
    row = 0
    for c in range(3):
        for m, (a, b) in enumerate([(0, 0), (0, 1), (1, 1)]):
            rhs[:, row] = d2phi[:, c, m] + K[:, a, b] * An[:, c]
            row += 1
    row += 3                                             # (ii): zero
    for c in range(3):
        rhs[:, row] = fy[:, c]
        row += 1
    sig = -kap * q[:, None, None] * np.eye(3) + mu * (A + np.swapaxes(A, 1, 2))
    dn = np.einsum("nab,nbk->nak", K, T)                 # d_a n
    for a in range(2):
        v = np.einsum("nik,nk->ni", sig, dn[:, a, :])
        for i in range(3):
            rhs[:, row] = -v[:, i]
            row += 1
    return rhs


def primary_points(cp, frames):
    """Primary/secondary classification (Sec. 3; our reading of the deferred
    definition): a point on an a-line is primary when the line is the most
    normal of the three directions there, |n_a| >= max_b |n_b| (with a 1e-12
    tolerance, so near-ties are primary in both families).  Only primary
    points carry density unknowns and BIE equations; the density at a
    secondary point is the fitted value from nearby primary points."""
    n = frames[0]
    na = np.abs(n[np.arange(cp.n), cp.axis])
    # the two roots of a grazing segment lie where their line is nearly tangent
    # to Gamma: always secondary
    return (na >= np.max(np.abs(n), axis=1) - 1e-12) & (cp.graze == 0)


# Sec. 4.3: per-point data of the jump evaluation.
class JumpData:
    """Per-point geometry and neighbour lists used by the jump evaluation."""

    def __init__(self, grid, geom, cp):
        self.h = grid.h
        self.cp = cp
        self.frames = geometry.frames(geom, cp.xyz)
        self.primary = primary_points(cp, self.frames)
        self.nbrs = neighbour_lists(cp, self.primary)


def jumps(jd, phi_p, fy, mu, lam=None):
    """Jump values at every control point y in X_c on an a-line:
    column 0 [u^(c)], 1-3 [grad u^(c)], 4-9 [Hess u^(c)] (order 11,22,33,23,13,12),
    10 [p], 11 [d_a p].  phi_p: density at the primary points (canonical
    order); fy (n, 3) = f at all points (zero for the double layer, Prop. DBI;
    f itself for the volume integral, Prop. FBI)."""
    cp = jd.cp
    n, T, K = jd.frames
    mu = float(mu)
    phi = np.zeros(cp.n)
    phi[jd.primary] = phi_p
    der = surface_derivatives(cp, jd.frames, jd.nbrs, phi, jd.h)   # (n, 3, 6)
    rows = np.arange(cp.n)
    phi = np.where(jd.primary, phi, der[rows, cp.comp - 1, 0])
    A, q = first_order(n, T, der[:, :, 1:3], mu, lam)
    L = second_order_system(n, T, K, mu, lam)
    rhs = second_order_rhs(n, T, K, A, q, der[:, :, 3:6], fy, mu, lam)
    x = np.linalg.solve(L, rhs[..., None])[..., 0]
    out = np.zeros((cp.n, 12))
    rows = np.arange(cp.n)
    c = cp.comp - 1
    out[:, 0] = phi
    out[:, 1:4] = A[rows, c, :]
    for m in range(6):
        out[:, 4 + m] = x[rows, 6 * c + m]
    out[:, 10] = q
    out[:, 11] = x[rows, 18 + cp.axis]
    return out
