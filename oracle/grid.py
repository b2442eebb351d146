"""Staggered MAC grids, sides and interface/grid-line intersections
(Sec. 4.2 grid sets T_h^0..T_h^3; Alg. 1 step 1; Sec. 3 control points).

Index conventions (0-based, arrays indexed [k, j, i] = [z, y, x]):
  grid 0 (cells, p):      node (i,j,k) at lo + (i+1/2, j+1/2, k+1/2) h
  grid c in 1..3 (u^(c)): the coordinate along axis c-1 is lo + idx h (face
                          index 0..N-1; face 0 is the box wall, u = 0 there,
                          face N is the opposite wall), the others are centred.
Unknowns of u^(c): face index 1..N-1 along axis c-1, 0..N-1 across.  This is
the reading of the paper's index set I^(1) (which lists i = 0): face 0 lies on
dB where u = 0 (IUS-5), so it carries no unknown.

A node is on the Omega side (+) when F <= 0 (Omega = {F < 0}; nodes exactly
on Gamma are counted as Omega, the paper is silent on the tie).

Control points (Sec. 3, reading of the deferred classification): X_c is the
set of intersections of Gamma with the grid lines, in all three directions,
of u^(c)'s own grid, restricted to segments between two unknown nodes.  Each
point carries the density component phi^(c).  Canonical order: component c,
then line axis a, then the line (outer = higher axis index), then position
along the line.
"""
import numpy as np

from . import geometry


# Sec. 4.2: the cell grid T_h^0 and the staggered face grids T_h^1..T_h^3 of the box B.
class Grid:
    def __init__(self, N, lo, hi):
        self.N = int(N)
        self.lo = float(lo)
        self.hi = float(hi)
        self.h = (self.hi - self.lo) / self.N

    # Sec. 4.2: node offsets of the grid sets.
    def offsets(self, c):
        """Per-axis offset (in units of h) of grid c's nodes from lo."""
        off = np.array([0.5, 0.5, 0.5])
        if c > 0:
            off[c - 1] = 0.0
        return off

    # Sec. 4.2: node coordinates of the grid sets.
    def node_xyz(self, c, idx):
        """Coordinates of grid-c nodes; idx (..., 3) integer (i, j, k)."""
        return self.lo + (np.asarray(idx, dtype=np.float64) + self.offsets(c)) * self.h

    # Sec. 4.2: the index set of a grid.
    def all_idx(self):
        """(N, N, N, 3) array of (i, j, k) in [k, j, i] layout."""
        N = self.N
        k, j, i = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
        return np.stack([i, j, k], axis=-1)

    # Sec. 4.2: the unknowns of u^(c) (wall faces excluded, IUS-5).
    def unknown_mask(self, c):
        """True where grid c carries an unknown ([k, j, i] layout)."""
        m = np.ones((self.N,) * 3, dtype=bool)
        if c > 0:
            sl = [slice(None)] * 3
            sl[2 - (c - 1)] = 0
            m[tuple(sl)] = False
        return m


# Alg. 1 step 1: the side of Gamma of every node of a grid.
def sides(grid, geom, c):
    """Boolean [k, j, i] array: True where the grid-c node is in Omega."""
    X = grid.node_xyz(c, grid.all_idx())
    return geometry.level_value(geom, X) <= 0.0


# Sec. 3: control points are the intersections of Gamma with the grid lines.
class ControlPoints:
    """Intersections of Gamma with the grid lines of u^(1), u^(2), u^(3)."""

    def __init__(self, comp, axis, idx, theta, xyz, graze=None):
        self.comp = comp      # (n,) component c in 1..3
        self.axis = axis      # (n,) line axis a in 0..2
        self.idx = idx        # (n, 3) lower node (i, j, k) of the segment, grid c
        self.theta = theta    # (n,) fraction in [0, 1) from the lower node
        self.xyz = xyz        # (n, 3)
        self.n = len(comp)
        # (n,) 0, or 1 / 2 for the root below / above the cell centre of a
        # grazing face segment (both face nodes on one side, the cell centre
        # between them on the other)
        self.graze = np.zeros(self.n, dtype=np.int8) if graze is None else graze

    # Sec. 3: numbering of the control-point sets X_1, X_2, X_3.
    def offsets(self):
        """Start offsets of X_1, X_2, X_3 in the concatenated numbering."""
        return np.array([np.sum(self.comp < c) for c in (1, 2, 3, 4)])


# Alg. 1 step 1: intersection of Gamma with one grid-line segment.
def _bisect(geom, x0, dirv, h, side0, t0=0.0, t1=1.0):
    """Root of F on the segment x0 + t h dirv, t in [t0, t1] (default the whole
    segment), by 64 bisection steps; side0 is the side (F <= 0) of the t0 end."""
    lo = np.full(len(x0), float(t0))
    hi = np.full(len(x0), float(t1))
    for _ in range(64):
        mid = 0.5 * (lo + hi)
        s = geometry.level_value(geom, x0 + (mid * h)[:, None] * dirv) <= 0.0
        same = s == side0
        lo = np.where(same, mid, lo)
        hi = np.where(same, hi, mid)
    return lo


# Sec. 3 and Alg. 1 step 1: all control points, in canonical order.
def control_points(grid, geom):
    """All control points in canonical order, plus per-grid side arrays."""
    N, h = grid.N, grid.h
    S = {c: sides(grid, geom, c) for c in range(4)}
    comps, axes, idxs, thetas, grazes = [], [], [], [], []
    for c in (1, 2, 3):
        Sc = S[c]
        unk = grid.unknown_mask(c)
        for a in range(3):
            ax = 2 - a                       # numpy axis of coordinate a
            sl0 = [slice(None)] * 3
            sl1 = [slice(None)] * 3
            sl0[ax] = slice(0, N - 1)
            sl1[ax] = slice(1, N)
            both = unk[tuple(sl0)] & unk[tuple(sl1)]
            cross = (Sc[tuple(sl0)] != Sc[tuple(sl1)]) & both
            kk, jj, ii = np.nonzero(cross)
            idx = np.stack([ii, jj, kk], axis=-1)
            dirv = np.zeros(3)
            dirv[a] = 1.0
            side0 = Sc[idx[:, 2], idx[:, 1], idx[:, 0]]
            t = _bisect(geom, grid.node_xyz(c, idx), dirv, h, side0)
            g = np.zeros(len(idx), dtype=np.int8)
            if c == a + 1:
                # grazing face segments of the combined u^(c)/cell line: the
                # cell centre between two same-side faces lies on the other
                # side, so Gamma crosses once below and once above it
                Cs = S[0][tuple(sl0)]
                graze = (Sc[tuple(sl0)] == Sc[tuple(sl1)]) & (Cs != Sc[tuple(sl0)]) & both
                kk, jj, ii = np.nonzero(graze)
                gidx = np.stack([ii, jj, kk], axis=-1)
                gs0 = Sc[gidx[:, 2], gidx[:, 1], gidx[:, 0]]
                gx0 = grid.node_xyz(c, gidx)
                tl = _bisect(geom, gx0, dirv, h, gs0, 0.0, 0.5)
                tr = _bisect(geom, gx0, dirv, h, ~gs0, 0.5, 1.0)
                idx = np.concatenate([idx, gidx, gidx])
                t = np.concatenate([t, tl, tr])
                g = np.concatenate([g, np.full(len(gidx), 1, np.int8), np.full(len(gidx), 2, np.int8)])
            other = [b for b in range(3) if b != a]      # increasing axis order
            # canonical order: outer = higher other axis, inner = lower, then
            # along a (the two roots of a grazing segment in increasing t)
            order = np.lexsort((t, idx[:, a], idx[:, other[0]], idx[:, other[1]]))
            comps.append(np.full(len(idx), c))
            axes.append(np.full(len(idx), a))
            idxs.append(idx[order])
            thetas.append(t[order])
            grazes.append(g[order])
    comp = np.concatenate(comps)
    axis = np.concatenate(axes)
    idx = np.concatenate(idxs).astype(np.int64)
    theta = np.concatenate(thetas)
    graze = np.concatenate(grazes)
    off = np.full((len(comp), 3), 0.5)
    off[np.arange(len(comp)), comp - 1] = 0.0
    xyz = grid.lo + (idx + off) * h
    xyz[np.arange(len(comp)), axis] += theta * h
    return ControlPoints(comp, axis, idx, theta, xyz, graze), S


# Ordering helper for the control points of Sec. 3 (no arithmetic of the method).
def fine_keys(cp):
    """Integer position of each point's segment midpoint in units of h/2."""
    key = 2 * cp.idx + 1
    key[np.arange(cp.n), cp.comp - 1] -= 1
    key[np.arange(cp.n), cp.axis] += 1
    return key


# Reading of the resolution the method assumes: the fit neighbourhood of
# Sec. 4.3 inside the box.
def check_geometry(grid, geom, cp, S):
    """Reject geometries the discretisation does not resolve (KFBIM_E_GEOMETRY):
    Gamma within 3h of the box wall.  A combined u^(a)/cell line that changes
    side twice within one face segment (a grazing segment) is resolved by its
    two roots (control_points), so it is no longer an error."""
    for c in range(4):
        Sc = S[c]
        band = np.zeros_like(Sc)
        band[:3], band[-3:] = True, True
        band[:, :3], band[:, -3:] = True, True
        band[:, :, :3], band[:, :, -3:] = True, True
        if np.any(Sc & band):
            raise ValueError("interface closer than 3h to the box wall")
    return True
