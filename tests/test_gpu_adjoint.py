"""Adjoint on the GPU: the transposed matvec against the forward matvec (inner
product identity), the gradient of a velocity loss against the oracle's
brute-force adjoint on 16^3, against central differences along 32 random
directions on the sphere at 32^3 and the star at 128^3 (through the
torch.autograd binding), and MIXED against FP64 at 128^3.  The loss is quadratic in g, so central differences carry no
truncation error; the step is large against the GMRES tolerance."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import adjoint as oadjoint, kfbim as okfbim

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import FP64, MIXED, Solver, build, solve_velocity  # noqa: E402

build()


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def boundary_data(s, seed=5, degree=3):
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    return ki.harmonic_curl_field(seed, degree=degree)(xyz)[rows, comp - 1][prim]


def loss_parts(s, seed=5):
    """Omega mask on the face grids and a target velocity (0.8 x the exact
    field of the boundary data)."""
    N, lo, h = s.N, s.lo, s.h
    idx = np.arange(N)
    field = ki.harmonic_curl_field(seed, degree=3)
    mask, tgt = [], []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")
        tgt.append(0.8 * field(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
        mask.append(s.sides(c).ravel().astype(float))
    return cuda(np.concatenate(mask)), cuda(np.concatenate(tgt))


@pytest.mark.parametrize("key,geom,N,prec", [("sphere32", ki.sphere(), 32, FP64),
                                             ("star64", ki.star(), 64, FP64),
                                             ("star64_mixed", ki.star(), 64, MIXED)])
def test_inner_product_identity(key, geom, N, prec):
    s = Solver(geom, ki.grid(N), precision=prec)
    rng = np.random.default_rng(3)
    x = cuda(rng.standard_normal(s.n_primary))
    y = cuda(rng.standard_normal(s.n_primary))
    ax = torch.zeros_like(x)
    aty = torch.zeros_like(y)
    s.apply(x, ax)
    s.apply_adjoint(y, aty)
    a = float(ax @ y)
    b = float(x @ aty)
    scale = float(ax.norm() * y.norm())
    assert abs(a - b) <= (1e-10 if prec == FP64 else 1e-9) * scale, (a, b)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_gradient_matches_oracle_adjoint_sphere16(prec):
    o = okfbim.Setup(ki.sphere(), ki.grid(16))
    A, U = oadjoint.dense_maps(o)
    s = Solver(ki.sphere(), ki.grid(16), precision=prec)
    mask, tgt = loss_parts(s)
    g0 = boundary_data(s)
    phi = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    u = torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda")
    p = torch.zeros(16 ** 3, dtype=torch.float64, device="cuda")
    s.solve(cuda(g0), phi, None, None, u, p)
    ubar = mask * (u - tgt)
    gbar = torch.zeros_like(phi)
    s.solve_adjoint(ubar, gbar)
    want = oadjoint.gradient_g(A, U, ubar.cpu().numpy())
    got = gbar.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()


@pytest.mark.parametrize("key,geom,N,prec,tol", [("sphere32", ki.sphere(), 32, FP64, 1e-12),
                                                 ("star128_mixed", ki.star(), 128, MIXED, 1e-11)])
def test_gradient_matches_central_differences_32_directions(key, geom, N, prec, tol):
    """Central differences of the loss along 32 seeded directions against the
    adjoint gradient (C5: 32 random directions).  At 128^3 the MIXED path is
    used (a FP64 solve there takes seconds, and 64 of them are needed) with
    GMRES to 1e-11, which keeps the solve linear to about 1e-10 relative."""
    s = Solver(geom, ki.grid(N), precision=prec, gmres_tol=tol)
    mask, tgt = loss_parts(s)
    g0 = cuda(boundary_data(s))

    def loss(g):
        u = solve_velocity(s, g)
        r = mask * (u - tgt)
        return 0.5 * (r * r).sum()

    g = g0.clone().requires_grad_(True)
    L = loss(g)
    L.backward()
    grad = g.grad.detach()
    rng = np.random.default_rng(4)
    fd, ad = [], []
    with torch.no_grad():
        for _ in range(32):
            d = cuda(rng.standard_normal(s.n_primary))
            eps = 1e-2 * float(g0.norm() / d.norm())
            fd.append(float(loss(g0 + eps * d) - loss(g0 - eps * d)) / (2 * eps))
            ad.append(float(grad @ d))
    fd, ad = np.array(fd), np.array(ad)
    assert np.abs(fd - ad).max() <= 1e-6 * np.abs(ad).max(), np.abs(fd - ad).max() / np.abs(ad).max()


def test_mixed_adjoint_matches_fp64_star128():
    geom, grid = ki.WORKLOADS["star128"]
    grads = []
    for prec in (FP64, MIXED):
        s = Solver(geom, grid, precision=prec)
        mask, tgt = loss_parts(s)
        g = cuda(boundary_data(s)).requires_grad_(True)
        u = solve_velocity(s, g)
        r = mask * (u - tgt)
        (0.5 * (r * r).sum()).backward()
        grads.append(g.grad.detach().cpu().numpy())
        assert s.last_stats["gmres_residual"] < 1e-10
    assert np.abs(grads[1] - grads[0]).max() <= 1e-7 * np.abs(grads[0]).max()
