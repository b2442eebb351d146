"""KFBI driver (Alg. 1): the interface solve of step 2, the BIE matvec, the
GMRES iteration of step 3 and the final interior fields.

  apply(phi)  = u^+ on Gamma of the interface problem with [u] = phi,
                f~ = 0 (Prop. DBI: u^+ = 1/2 phi - M_v phi)
  volume(f)   = u^+ of the interface problem with [u] = 0 and f~ (Prop. FBI)
  solve(g, f) : GMRES for 1/2 phi - M_v phi = g - G_v f from phi = 0, then
                one unified interface solve (IUS) for (u_h, p_h).
"""
import numpy as np

from . import grid as gridmod, jumps as jumpmod, correct, interp, mac


class Setup:
    """lam = None: Stokes (Eq. SP, unified IUS); lam = Lame lambda: Navier
    (Eq. Navier, unified I-E with c = 1/(lambda + mu))."""

    def __init__(self, geom, grid_desc, mu=1.0, cg_tol=1e-14, lam=None):
        self.geom = geom
        self.grid = gridmod.Grid(grid_desc["N"], grid_desc["lo"], grid_desc["hi"])
        self.mu = float(mu)
        self.lam = None if lam is None else float(lam)
        self.cpen = None if lam is None else 1.0 / (self.lam + self.mu)
        self.cg_tol = cg_tol
        self.cp, self.S = gridmod.control_points(self.grid, geom)
        gridmod.check_geometry(self.grid, geom, self.cp, self.S)
        self.jd = jumpmod.JumpData(self.grid, geom, self.cp)
        self.cg_iters = []

    # Sec. 3: one density unknown per primary control point.
    @property
    def n(self):
        """Number of density unknowns (primary control points)."""
        return int(np.sum(self.jd.primary))

    # Sec. 3: the primary control points.
    @property
    def primary(self):
        return self.jd.primary

    def masked_forcing(self, f_faces):
        """f~ on the face grids: f in Omega, 0 in Omega^c (Prop. FBI)."""
        return [np.where(self.S[c], f_faces[c - 1], 0.0) for c in (1, 2, 3)]

    def interface(self, phi, fy, f_faces):
        """Unified interface solve (IUS-1..5) on the grid: returns (u, p, J)."""
        J = jumpmod.jumps(self.jd, phi, fy, self.mu, self.lam)
        Cf, Cg = correct.corrections(self.grid, self.cp, self.S, J, self.mu)
        if f_faces is None:
            f = Cf
        else:
            ft = self.masked_forcing(f_faces)
            f = [ft[c] + Cf[c] for c in range(3)]
        f = [mac.zero_walls(f[c - 1], c) for c in (1, 2, 3)]
        u, p, it = mac.interface_solve(f, Cg, self.mu, self.grid.h, tol=self.cg_tol, cpen=self.cpen)
        self.cg_iters.append(it)
        return u, p, J

    # Sec. 4.4: u^+ at the primary control points.
    def trace(self, u, J):
        """u^+ at the primary control points from face fields u and jumps J."""
        return interp.trace(self.grid, self.cp, self.S, u, J)[self.primary]

    # Prop. DBI and Eq. BIE-S: the GMRES matvec.
    def apply(self, phi):
        """(1/2 I - M_v) phi at the primary control points."""
        u, _, J = self.interface(phi, np.zeros((self.cp.n, 3)), None)
        return self.trace(u, J)

    # Prop. FBI: the volume integral on Gamma.
    def volume_trace(self, fy, f_faces):
        """(G_v f) on Gamma at the primary control points."""
        u, _, J = self.interface(np.zeros(self.n), fy, f_faces)
        return interp.trace(self.grid, self.cp, self.S, u, J)[self.primary]

    def solve(self, g, fy=None, f_faces=None, tol=1e-10, maxit=200):
        """Alg. 1 step 3 + final fields.  g: boundary data at the primary
        points; fy: f at all control points.  Returns dict(phi, u, p, iters, res)."""
        if fy is None:
            fy = np.zeros((self.cp.n, 3))
        rhs = np.array(g, dtype=np.float64)
        if f_faces is not None:
            rhs = rhs - self.volume_trace(fy, f_faces)
        phi, its, hist = gmres(self.apply, rhs, tol=tol, maxit=maxit)
        u, p, _ = self.interface(phi, fy, f_faces)
        return {"phi": phi, "u": u, "p": p, "iters": its, "res": hist}


def gmres(apply, b, tol=1e-10, maxit=200):
    """Unrestarted GMRES from x = 0 with classical Gram-Schmidt applied twice
    and the small least-squares problem solved by lstsq; stops when
    ||b - A x|| / ||b|| < tol (Sec. 5: relative l2 residual)."""
    n = len(b)
    beta = np.linalg.norm(b)
    if beta == 0.0:
        return np.zeros(n), 0, [0.0]
    V = np.zeros((maxit + 1, n))
    Hm = np.zeros((maxit + 1, maxit))
    V[0] = b / beta
    hist = [1.0]
    y = np.zeros(0)
    k = 0
    for k in range(1, maxit + 1):
        w = apply(V[k - 1])
        h1 = V[:k] @ w
        w = w - V[:k].T @ h1
        h2 = V[:k] @ w
        w = w - V[:k].T @ h2
        Hm[:k, k - 1] = h1 + h2
        Hm[k, k - 1] = np.linalg.norm(w)
        e1 = np.zeros(k + 1)
        e1[0] = beta
        y = np.linalg.lstsq(Hm[:k + 1, :k], e1, rcond=None)[0]
        res = np.linalg.norm(e1 - Hm[:k + 1, :k] @ y) / beta
        hist.append(res)
        if res < tol or Hm[k, k - 1] == 0.0:
            break
        V[k] = w / Hm[k, k - 1]
    x = V[:k].T @ y
    return x, k, hist
