"""Right-hand-side corrections of the modified MAC scheme (Sec. 4.3, items 1-4,
Eq. MAC with f = f~ + C{mu Lap u} + C{p_x}, g = sum C{u_x}).

One rule reproduces items 1-3 and the pressure part of item 4: for an equation
at node P whose stencil coefficient on a neighbour Q across Gamma is a_PQ,
    C_P += a_PQ * chi_Q * J(Q),   chi_Q = +1 if Q in Omega, -1 otherwise,
    J(Q) = [v] + xi [v_a] + xi^2/2 [v_aa] (pressure: [p] + xi [p_a]),
    xi = x_Q - r along the line, r the intersection on segment PQ.
E.g. item 1 (P in Omega, a = -mu/h^2, chi = -1) gives +mu/h^2 (...) as printed.
Reading of item 4's continuity term: the same rule gives -(1/h)(...) for a
cell in Omega whose face neighbour is outside; the paper prints '+'.  The
rule is what makes the corrected divergence consistent with the Taylor
expansion behind the scheme, so it is taken here.

Targets: rows of f^(c) at grid-c nodes (Laplacian and pressure-gradient
corrections) and rows of g at cells (continuity corrections).
"""
import numpy as np


# Sec. 4.3 items 1-4: the side sign chi_Q of a correction.
def _chi(side):
    return np.where(side, 1.0, -1.0)


# Sec. 4.3 items 1-4: the corrected right-hand sides of Eq. MAC.
def corrections(grid, cp, S, J, mu):
    """Return (Cf (3 face fields), Cg (cell field)) from jump values J (n, 12)."""
    N, h = grid.N, grid.h
    Cf = [np.zeros((N, N, N)) for _ in range(3)]
    Cg = np.zeros((N, N, N))
    rows = np.arange(cp.n)
    c = cp.comp
    a = cp.axis
    P0 = cp.idx
    P1 = cp.idx.copy()
    P1[rows, a] += 1
    th = cp.theta
    J0 = J[:, 0]
    Ja = J[rows, 1 + a]
    Jaa = J[rows, 4 + a]           # H entries 11, 22, 33 are columns 4, 5, 6

    def Ju(xi):
        return J0 + xi * Ja + 0.5 * xi * xi * Jaa

    def Jp(xi):
        return J[:, 10] + xi * J[:, 11]

    def side(cc, P):
        out = np.zeros(len(P), dtype=bool)
        for g in (1, 2, 3):
            sel = cc == g
            out[sel] = S[g][P[sel, 2], P[sel, 1], P[sel, 0]]
        return out

    s0 = side(c, P0)
    s1 = side(c, P1)
    # item 1-3: Laplacian, coefficient -mu/h^2 on each across-neighbour; the
    # faces of a grazing segment are on one side (no Laplacian correction)
    lap_a = -mu / (h * h)
    v0 = lap_a * _chi(s1) * Ju((1.0 - th) * h)      # row P0, neighbour P1
    v1 = lap_a * _chi(s0) * Ju(-th * h)             # row P1, neighbour P0
    for m in np.nonzero(cp.graze == 0)[0]:
        cf = Cf[c[m] - 1]
        i, j, k = P0[m]
        cf[k, j, i] += v0[m]
        i, j, k = P1[m]
        cf[k, j, i] += v1[m]
    # item 4: lines shared by u^(a) and the cells (c == a + 1)
    u_left = Ju(-th * h)                              # J at P0 (xi = x_P0 - r)
    u_right = Ju((1.0 - th) * h)                      # J at P1 (xi = x_P1 - r)
    p_mid = Jp(0.5 * h - th * h)                      # J_p at the cell centre C
    for m in np.nonzero(c == a + 1)[0]:
        i, j, k = P0[m]
        sC = bool(S[0][k, j, i])                     # cell C between P0 and P1
        # crossing between P0 and C, or between C and P1 (a grazing segment
        # has one of each: its two roots)
        below = cp.graze[m] == 1 if cp.graze[m] else sC == bool(s1[m])
        if below:                                    # crossing between P0 and C
            Cg[k, j, i] += (-1.0 / h) * _chi(s0[m]) * u_left[m]
            Cf[c[m] - 1][k, j, i] += (1.0 / h) * _chi(sC) * p_mid[m]
        else:                                        # crossing between C and P1
            Cg[k, j, i] += (1.0 / h) * _chi(s1[m]) * u_right[m]
            i1, j1, k1 = P1[m]
            Cf[c[m] - 1][k1, j1, i1] += (-1.0 / h) * _chi(sC) * p_mid[m]
    return Cf, Cg
