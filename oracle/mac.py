"""MAC operators, the FFT (DST) Poisson solver and the Schur-complement CG of
Sec. 4.2 (Eqs. MAC, linearS, linearS1 and items i-iii).

Fields use the padded N^3 layout of grid.py.  Face index 0 of u^(c) along its
normal axis is the wall value, held at 0.

Operators (delta^+, delta^- and Delta_h of Sec. 4.2):
  G p   (cells -> faces):  (G p)^(c) at face i = (p_i - p_{i-1}) / h, faces 1..N-1
  D u   (faces -> cells):  (D u) at cell m = sum_c (u_{m+1} - u_m) / h, with the
                           wall faces 0 and N equal to 0;  D = -G^T.
  Lap u (faces -> faces):  7-point Delta_h; along the normal axis the wall
                           faces are 0; along the tangential axes the ghost
                           value beyond the wall is -u of the first interior
                           node (zero wall value, IUS-5 on the ghost layers of
                           T_h^1..T_h^3).
Reading of the box conditions: with these ghost rules Delta_h on u^(c) is
diagonalised by DST-I along axis c (length N-1) and DST-II along the other
two axes, which is what makes the FFT Poisson solver of item ii) applicable.
"""
import numpy as np
import scipy.fft as sfft


# Array axis of a grid axis (layout helper for Sec. 4.2).
def _ax(a):
    return 2 - a


# Sec. 4.2 and IUS-5: u = 0 on the wall faces.
def zero_walls(u, c):
    sl = [slice(None)] * 3
    sl[_ax(c - 1)] = 0
    u = u.copy()
    u[tuple(sl)] = 0.0
    return u


# Sec. 4.2, Eq. MAC: the difference operator delta^- on p (G).
def grad(p, h):
    """G p: three face fields; face 0 (wall) left at 0."""
    out = []
    for c in (1, 2, 3):
        ax = _ax(c - 1)
        g = np.zeros_like(p)
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        dst = [slice(None)] * 3
        hi[ax] = slice(1, None)
        lo[ax] = slice(0, -1)
        dst[ax] = slice(1, None)
        g[tuple(dst)] = (p[tuple(hi)] - p[tuple(lo)]) / h
        out.append(g)
    return out


# Sec. 4.2, Eq. MAC: the difference operator delta^+ on u (D = -G^T).
def div(u, h):
    """D u at cells: sum_c (u^(c)_{m+1} - u^(c)_m) / h with wall faces 0."""
    N = u[0].shape[0]
    out = np.zeros((N, N, N))
    for c in (1, 2, 3):
        ax = _ax(c - 1)
        uc = zero_walls(u[c - 1], c)
        pad = [(0, 0)] * 3
        pad[ax] = (0, 1)                       # face N = wall
        ue = np.pad(uc, pad)
        hi = [slice(None)] * 3
        lo = [slice(None)] * 3
        hi[ax] = slice(1, None)
        lo[ax] = slice(0, -1)
        out += (ue[tuple(hi)] - ue[tuple(lo)]) / h
    return out


# Sec. 4.2, Eq. MAC: Delta_h with the ghost layers of T_h^1..T_h^3.
def lap(uc, c, h):
    """Delta_h u^(c) on the unknown nodes (wall face entries returned as 0)."""
    u = zero_walls(uc, c)
    out = np.zeros_like(u)
    for a in range(3):
        ax = _ax(a)
        if a == c - 1:
            pad = [(0, 0)] * 3
            pad[ax] = (0, 1)
            ue = np.pad(u, pad)                # face N = 0; face 0 already 0
            ue = np.concatenate([np.take(ue, [0], axis=ax) * 0.0, ue], axis=ax)
        else:
            first = np.take(u, [0], axis=ax)
            last = np.take(u, [u.shape[ax] - 1], axis=ax)
            ue = np.concatenate([-first, u, -last], axis=ax)
        n = u.shape[ax]
        out += (np.take(ue, np.arange(2, n + 2), axis=ax) - 2.0 * u
                + np.take(ue, np.arange(0, n), axis=ax)) / (h * h)
    return zero_walls(out, c)


# Sec. 4.2 item iii: the eigenvalues of the FFT (DST) solver.
def _eig1(n_modes, N, first):
    m = np.arange(first, first + n_modes)
    return 4.0 * np.sin(np.pi * m / (2.0 * N)) ** 2


def poisson(rc, c, h):
    """Solve -Delta_h u^(c) = r^(c) (the FFT Poisson solver of Sec. 4.2 item
    ii) with scipy's DST: type I along axis c-1 on faces 1..N-1, type II
    along the other axes; eigenvalues (4/h^2) sum sin^2(pi m / 2N)."""
    N = rc.shape[0]
    axc = _ax(c - 1)
    sl = [slice(None)] * 3
    sl[axc] = slice(1, None)
    r = rc[tuple(sl)]
    types = [2, 2, 2]
    types[axc] = 1
    R = r
    for ax in range(3):
        R = sfft.dst(R, type=types[ax], axis=ax)
    lam = np.zeros(R.shape)
    for ax in range(3):
        n = R.shape[ax]
        e = _eig1(n, N, 1)
        shape = [1, 1, 1]
        shape[ax] = n
        lam = lam + e.reshape(shape)
    R = R / (lam / (h * h))
    for ax in range(3):
        R = sfft.idst(R, type=types[ax], axis=ax)
    out = np.zeros_like(rc)
    out[tuple(sl)] = R
    return out


def schur_apply(d, mu, h, alpha, cpen=None):
    """(1/mu) G^T (-Delta_h)^{-1} G d + (1/alpha) gamma gamma^T d, gamma = 1.

    Reading of the sign in item ii): the '+' printed with the rank-one term
    gives an SPD operator for CG; both signs give the same velocity and the
    same mean-free pressure.  G^T = -D.
    Navier (cpen = c = 1/(lambda + mu), continuity row div u + c p = g):
    (1/mu) G^T (-Delta_h)^{-1} G d + c d, no rank-one term."""
    g = grad(d, h)
    w = [poisson(g[c - 1], c, h) for c in (1, 2, 3)]
    if cpen is not None:
        return -div(w, h) / mu + cpen * d
    return -div(w, h) / mu + np.sum(d) / alpha


def schur_rhs(f, g, mu, h):
    """b = g + (1/mu) G^T (-Delta_h)^{-1} f   (item ii, with D = -G^T)."""
    w = [poisson(f[c - 1], c, h) for c in (1, 2, 3)]
    return g - div(w, h) / mu


# Sec. 4.2 items i-iii: CG on the Schur complement.
def cg(apply, b, tol=1e-14, maxit=2000):
    """Unpreconditioned conjugate gradients from x = 0 (the paper uses no
    preconditioner).  Stops at ||r|| <= tol ||b||."""
    x = np.zeros_like(b)
    r = b.copy()
    d = r.copy()
    rr = float(np.sum(r * r))
    bn = np.sqrt(float(np.sum(b * b)))
    it = 0
    if bn == 0.0:
        return x, 0
    while it < maxit and np.sqrt(rr) > tol * bn:
        q = apply(d)
        dq = float(np.sum(d * q))
        alpha = rr / dq
        x = x + alpha * d
        r = r - alpha * q
        rr_new = float(np.sum(r * r))
        d = r + (rr_new / rr) * d
        rr = rr_new
        it += 1
    return x, it


# Sec. 4.2, Eqs. linearS and linearS1: the MAC system through its Schur complement.
def interface_solve(f, g, mu, h, tol=1e-14, cpen=None):
    """Solve the (corrected) MAC system [-mu Lap, G; D, 0][u; p] = [f; g]
    through the augmented system with lambda_h (gamma = 1, alpha = mu N^3):
    Schur CG for p (item ii), then u = (1/mu)(-Delta_h)^{-1}(f - G p)
    (item iii).  Navier (cpen = c): [-mu Lap, G; D, c I], Schur operator
    S + c I.  Returns (u (3 face fields), p, CG iterations)."""
    N = g.shape[0]
    alpha = mu * N ** 3
    b = schur_rhs(f, g, mu, h)
    p, it = cg(lambda d: schur_apply(d, mu, h, alpha, cpen), b, tol=tol)
    Gp = grad(p, h)
    u = [poisson(f[c - 1] - Gp[c - 1], c, h) / mu for c in (1, 2, 3)]
    return u, p, it
