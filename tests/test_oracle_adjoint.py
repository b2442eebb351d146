"""Pins of the oracle adjoint (oracle/adjoint.py): the dense maps reproduce the
oracle's matvec, and the gradient of a velocity loss with respect to the
boundary data matches central differences of the oracle's own GMRES forward
solve.  The loss is quadratic in g, so central differences carry no
truncation error; the step is large against the solve tolerance."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import adjoint, kfbim as okfbim


@pytest.fixture(scope="module")
def sphere16():
    o = okfbim.Setup(ki.sphere(), ki.grid(16))
    A, U = adjoint.dense_maps(o)
    return o, A, U


def _loss_parts(o):
    N = o.grid.N
    mask = np.concatenate([o.S[c].ravel() for c in (1, 2, 3)]).astype(float)
    field = ki.harmonic_curl_field(5, degree=3)
    tgt = []
    for c in (1, 2, 3):
        xyz = o.grid.node_xyz(c, o.grid.all_idx())
        tgt.append(0.8 * field(xyz)[..., c - 1].ravel())
    rows = np.arange(o.cp.n)
    g0 = field(o.cp.xyz)[rows, o.cp.comp - 1][o.primary]
    assert mask.size == 3 * N ** 3
    return mask, np.concatenate(tgt), g0


def test_dense_maps_reproduce_the_matvec(sphere16):
    o, A, U = sphere16
    x = np.random.default_rng(1).standard_normal(o.n)
    ax = o.apply(x)
    assert np.abs(A @ x - ax).max() <= 1e-11 * np.abs(ax).max()
    u, _, _ = o.interface(x, np.zeros((o.cp.n, 3)), None)
    uf = np.concatenate([u[c].ravel() for c in range(3)])
    assert np.abs(U @ x - uf).max() <= 1e-11 * np.abs(uf).max()


def test_gradient_matches_central_differences(sphere16):
    o, A, U = sphere16
    mask, tgt, g0 = _loss_parts(o)

    def loss(g):
        res = o.solve(g, tol=1e-13)
        uf = np.concatenate([res["u"][c].ravel() for c in range(3)])
        r = mask * (uf - tgt)
        return 0.5 * float(r @ r)

    u0 = U @ np.linalg.solve(A, g0)
    grad = adjoint.gradient_g(A, U, mask * (u0 - tgt))
    rng = np.random.default_rng(2)
    for _ in range(2):
        d = rng.standard_normal(o.n)
        eps = 1e-2 * np.linalg.norm(g0) / np.linalg.norm(d)
        fd = (loss(g0 + eps * d) - loss(g0 - eps * d)) / (2 * eps)
        ad = float(grad @ d)
        assert abs(fd - ad) <= 1e-6 * np.linalg.norm(grad) * np.linalg.norm(d), (fd, ad)
