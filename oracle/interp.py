"""Quadratic interpolation of the jump-corrected trace u^+ at control points
(Sec. 4.4, Eqs. Interpolation+/-; the unknowns are the value and first and
second derivatives of u^+ at x, ten in all).

Ten-node stencil (reading of the nearest-node choice of Sec. 4.4 and its figure): for a
control point of X_c on an a-line, with lower node P0 and fraction theta, the
base node b is P0 if theta < 1/2 else P0 + e_a; the stencil is
    b, b +- e_1, b +- e_2, b +- e_3, b + s_1 e_1 + s_2 e_2, b + s_1 e_1 + s_3 e_3,
    b + s_2 e_2 + s_3 e_3
with s_a pointing from b towards x along the line and s = +1 across it.  This
set is unisolvent for quadratics at any position of x (the axial nodes fix the
value, gradient and pure second derivatives, the three diagonal ones the mixed
derivatives), so no conditioning fallback is needed.

For nodes z_i in Omega^c the jump Taylor polynomial J_i is added (Sec. 4.4):
    v_i + J_i = P(z_i - x), P the quadratic Taylor polynomial of u^+ at x.
"""
import numpy as np


# Sec. 4.4: the ten interpolation nodes of a control point.
def stencil(cp):
    """Node indices (n, 10, 3) of each point's stencil on its own grid."""
    n = cp.n
    rows = np.arange(n)
    base = cp.idx.copy()
    up = cp.theta >= 0.5
    base[rows[up], cp.axis[up]] += 1
    sgn = np.ones((n, 3), dtype=np.int64)
    sgn[rows[up], cp.axis[up]] = -1
    E = np.eye(3, dtype=np.int64)
    offs = [np.zeros((n, 3), dtype=np.int64)]
    for a in range(3):
        offs.append(np.broadcast_to(E[a], (n, 3)))
        offs.append(-np.broadcast_to(E[a], (n, 3)))
    for (a, b) in [(0, 1), (0, 2), (1, 2)]:
        offs.append(sgn[:, a:a + 1] * E[a] + sgn[:, b:b + 1] * E[b])
    return base[:, None, :] + np.stack(offs, axis=1)


# Sec. 4.4: the quadratic Taylor basis of Eqs. Interpolation+/-.
def _taylor_rows(d):
    """Rows (1, x, y, z, x^2/2, y^2/2, z^2/2, yz, xz, xy) of offsets d (..., 3)."""
    x, y, z = d[..., 0], d[..., 1], d[..., 2]
    return np.stack([np.ones_like(x), x, y, z, 0.5 * x * x, 0.5 * y * y, 0.5 * z * z,
                     y * z, x * z, x * y], axis=-1)


# Sec. 4.4, Eqs. Interpolation+/-: the jump-corrected quadratic interpolation of u^+.
def trace(grid, cp, S, fields, J):
    """u^+ at every control point: solve the 10x10 Taylor system per point.
    fields: the three face fields; J (n, 12) jump values (jumps.py layout)."""
    st = stencil(cp)
    n = cp.n
    N = grid.N
    if np.any(st < 0) or np.any(st >= N):
        raise ValueError("interpolation stencil leaves the grid")
    vals = np.zeros((n, 10))
    outside = np.zeros((n, 10), dtype=bool)
    zxyz = np.zeros((n, 10, 3))
    for c in (1, 2, 3):
        sel = cp.comp == c
        s = st[sel]
        if np.any(s[..., c - 1] < 1):
            raise ValueError("interpolation stencil touches the wall face")
        vals[sel] = fields[c - 1][s[..., 2], s[..., 1], s[..., 0]]
        outside[sel] = ~S[c][s[..., 2], s[..., 1], s[..., 0]]
        zxyz[sel] = grid.node_xyz(c, s)
    d = zxyz - cp.xyz[:, None, :]
    V = _taylor_rows(d)                                   # (n, 10, 10)
    # jump Taylor polynomial J_i = [u] + d.[grad u] + 1/2 d^T [Hess u] d
    Hj = J[:, 4:10]
    coef = np.concatenate([J[:, 0:1], J[:, 1:4],
                           Hj[:, 0:3], Hj[:, 3:4], Hj[:, 4:5], Hj[:, 5:6]], axis=1)
    Ji = np.einsum("nmk,nk->nm", V, coef)
    rhs = vals + np.where(outside, Ji, 0.0)
    a = np.linalg.solve(V, rhs[..., None])[..., 0]
    return a[:, 0]


def pressure_trace(grid, cp, S, p, J):
    """p^+ at every control point by linear interpolation (Sec. 4.4, last
    paragraph: the stress needs no derivative of p, so a linear rule
    suffices).  Reading: trilinear interpolation over the eight cell centres
    around x; a cell in Omega^c contributes p + [p](x) (the jump [p] =
    p^+ - p^- at the point itself, slot 10 of J), its Omega-side extension to
    zeroth order.  p: cell field (N, N, N) in [k, j, i]; returns (n,)."""
    N, h, lo = grid.N, grid.h, grid.lo
    s = (cp.xyz - lo) / h - 0.5                       # cell-centre coordinates
    i0 = np.clip(np.floor(s).astype(np.int64), 0, N - 2)
    t = s - i0
    out = np.zeros(cp.n)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                ii, jj, kk = i0[:, 0] + di, i0[:, 1] + dj, i0[:, 2] + dk
                w = ((t[:, 0] if di else 1 - t[:, 0]) * (t[:, 1] if dj else 1 - t[:, 1])
                     * (t[:, 2] if dk else 1 - t[:, 2]))
                v = p[kk, jj, ii] + np.where(S[0][kk, jj, ii], 0.0, J[:, 10])
                out += w * v
    return out
