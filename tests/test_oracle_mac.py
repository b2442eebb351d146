"""Pins of the oracle's MAC operators, DST Poisson solver and Schur CG
(Sec. 4.2) against closed forms and dense linear algebra."""
import numpy as np
import pytest

from oracle import mac


@pytest.mark.parametrize("N", [8, 12])
@pytest.mark.parametrize("c", [1, 2, 3])
def test_poisson_inverts_stencil(c, N):
    # N = 12: a size that is not a power of two (like the 96^3 grid), so the
    # oracle's transforms are pinned there too
    h = 0.25
    r = mac.zero_walls(np.random.default_rng(c).standard_normal((N, N, N)), c)
    u = mac.poisson(r, c, h)
    assert np.abs(-mac.lap(u, c, h) - r).max() < 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("N", [8, 12])
@pytest.mark.parametrize("c", [1, 2, 3])
def test_dst_modes_are_eigenvectors(c, N):
    """Delta_h applied to sin(pi a i/N) (normal axis) x sin(pi b (j+1/2)/N) x
    sin(pi d (k+1/2)/N) returns -(4/h^2)(sum sin^2(pi m/2N)) times the mode."""
    h = 0.3
    rng = np.random.default_rng(7)
    for _ in range(5):
        modes = [int(rng.integers(1, N)) if ax == c - 1 else int(rng.integers(1, N + 1))
                 for ax in range(3)]
        idx = np.arange(N)
        vecs = []
        for ax in range(3):
            if ax == c - 1:
                vecs.append(np.sin(np.pi * modes[ax] * idx / N))
            else:
                vecs.append(np.sin(np.pi * modes[ax] * (idx + 0.5) / N))
        u = vecs[2][:, None, None] * vecs[1][None, :, None] * vecs[0][None, None, :]
        lam = -4.0 / h ** 2 * sum(np.sin(np.pi * m / (2 * N)) ** 2 for m in modes)
        Lu = mac.lap(u, c, h)
        u = mac.zero_walls(u, c)
        assert np.abs(Lu - lam * u).max() < 1e-11 * abs(lam)


def _dense(op, nin, shape_in):
    cols = []
    for j in range(nin):
        e = np.zeros(nin)
        e[j] = 1.0
        cols.append(op(e.reshape(shape_in)))
    return np.array(cols).T


def test_div_is_minus_grad_transpose():
    N, h = 4, 0.5
    n = N ** 3
    G = _dense(lambda p: np.concatenate([g.ravel() for g in mac.grad(p, h)]), n, (N, N, N))
    D = _dense(lambda u: mac.div([u[0], u[1], u[2]], h).ravel(), 3 * n, (3, N, N, N))
    keep = np.concatenate([mac.zero_walls(np.ones((N, N, N)), c).astype(bool).ravel()
                           for c in (1, 2, 3)])
    assert np.array_equal(D[:, keep], -G[keep, :].T)
    assert np.all(G[~keep, :] == 0)


def test_schur_symmetric_positive():
    N, h, mu = 4, 0.5, 1.7
    alpha = mu * N ** 3
    S = _dense(lambda d: mac.schur_apply(d, mu, h, alpha).ravel(), N ** 3, (N, N, N))
    assert np.abs(S - S.T).max() < 1e-12 * np.abs(S).max()
    ev = np.linalg.eigvalsh(0.5 * (S + S.T))
    assert ev.min() > 1e-6
    # constant mode: eigenvalue N^3/alpha = 1/mu (reading of the rank-one sign)
    one = np.ones(N ** 3)
    assert np.allclose(S @ one, one / mu)


def test_augmented_system_dense_lu():
    """The augmented system [-mu Lap, G, 0; D, 0, -gamma; 0, -gamma^T, alpha]
    (Eq. linearS1), solved densely, gives the same velocity and mean-free
    pressure as the oracle's Schur CG + velocity recovery."""
    N, h, mu = 5, 0.4, 1.3
    rng = np.random.default_rng(3)
    f = [mac.zero_walls(rng.standard_normal((N, N, N)), c) for c in (1, 2, 3)]
    g = rng.standard_normal((N, N, N))
    masks = [mac.zero_walls(np.ones((N, N, N)), c).astype(bool).ravel() for c in (1, 2, 3)]
    nu = [int(m.sum()) for m in masks]
    n = N ** 3
    nU = sum(nu)

    def unpack_u(x):
        out, o = [], 0
        for c in range(3):
            full = np.zeros(n)
            full[masks[c]] = x[o:o + nu[c]]
            out.append(full.reshape(N, N, N))
            o += nu[c]
        return out

    def op(x):
        u = unpack_u(x[:nU])
        p = x[nU:nU + n].reshape(N, N, N)
        lam = x[-1]
        Gp = mac.grad(p, h)
        r1 = np.concatenate([(-mu * mac.lap(u[c], c + 1, h) + Gp[c]).ravel()[masks[c]]
                             for c in range(3)])
        r2 = (mac.div(u, h) - lam).ravel()
        r3 = -np.sum(p) + mu * n * lam
        return np.concatenate([r1, r2, [r3]])

    M = _dense(op, nU + n + 1, (nU + n + 1,))
    rhs = np.concatenate([np.concatenate([f[c].ravel()[masks[c]] for c in range(3)]),
                          g.ravel(), [0.0]])
    x = np.linalg.solve(M, rhs)
    u_d = unpack_u(x[:nU])
    p_d = x[nU:nU + n].reshape(N, N, N)
    u, p, _ = mac.interface_solve(f, g, mu, h, tol=1e-15)
    for c in range(3):
        assert np.abs(u[c] - u_d[c]).max() < 1e-10 * np.abs(u_d[c]).max()
    dp = (p - p.mean()) - (p_d - p_d.mean())
    assert np.abs(dp).max() < 1e-10 * np.abs(p_d).max()
