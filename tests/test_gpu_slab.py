"""The three-kernel FP32 Schur CG iteration (z-pencil transforms after the
previous iteration's vector update, one CTA per xy plane, inverse z-pencil
transforms with the CG dot products) against the FP64 oracle and against the
one-axis staged passes it replaces.

* The FP32 Schur operator of the slab kernels (Sec. 4.2 item ii, the operator
  of Eq. linearS1 without its rank-one term) against the oracle's stencil form
  mu^-1 G^T (-Delta_h)^-1 G d: relative max-norm error <= 1e-5 (FP32
  transforms: about log2(N) roundings of 6e-8 per transform, 16 transforms).
* The MIXED matvec and interface solve with the slab CG against the same
  context kind with the staged passes (transforms STAGED): both are refined
  in FP64 to a relative residual of 1e-11, so they agree to 1e-10, and each
  matches the oracle to 1e-8 (the MIXED bar).
* Navier: the c p block of the Schur operator is added in the inverse z pass."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim as okfbim, mac

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import MIXED, KfbimError, Solver, build  # noqa: E402

build()

XF_AUTO, XF_STAGED = 0, 3


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def cuda(a, dtype=np.float64):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


@pytest.mark.parametrize("N", [32, 64, 128])
def test_schur_operator_f32_matches_oracle(N):
    s = Solver(ki.star(), ki.grid(N), precision=MIXED)
    d = np.random.default_rng(N).standard_normal((N, N, N))
    alpha = 1.0 * N ** 3
    want = mac.schur_apply(d, 1.0, s.h, alpha) - d.sum() / alpha
    q = torch.zeros(N ** 3, dtype=torch.float32, device="cuda")
    s.schur_apply_f32(cuda(d.ravel(), np.float32), q)
    assert rel(q.cpu().numpy().astype(np.float64).reshape(N, N, N), want) < 1e-5
    s.close()


def test_schur_operator_f32_navier_adds_c_d():
    N, lam = 32, 2.0
    s = Solver(ki.sphere(), ki.grid(N), precision=MIXED, lam=lam)
    d = np.random.default_rng(1).standard_normal((N, N, N))
    want = mac.schur_apply(d, 1.0, s.h, None, cpen=1.0 / (lam + 1.0))
    q = torch.zeros(N ** 3, dtype=torch.float32, device="cuda")
    s.schur_apply_f32(cuda(d.ravel(), np.float32), q)
    assert rel(q.cpu().numpy().astype(np.float64).reshape(N, N, N), want) < 1e-5
    s.close()


def test_schur_operator_f32_needs_the_slab_path():
    s = Solver(ki.sphere(), ki.grid(32), precision=MIXED, transforms=XF_STAGED)
    d = torch.zeros(32 ** 3, dtype=torch.float32, device="cuda")
    with pytest.raises(KfbimError) as e:
        s.schur_apply_f32(d, torch.zeros_like(d))
    assert e.value.code == -1
    s.close()


CASES = [("sphere32", ki.sphere(), 32), ("star64", ki.star(), 64), ("star128", ki.star(), 128)]


@pytest.mark.parametrize("key,geom,N", CASES, ids=[c[0] for c in CASES])
def test_slab_matvec_matches_staged_and_oracle(key, geom, N):
    o = okfbim.Setup(geom, ki.grid(N))
    phi = ki.random_density(o.n, seed=17)
    want = o.apply(phi)
    got = {}
    for xf in (XF_AUTO, XF_STAGED):
        s = Solver(geom, ki.grid(N), precision=MIXED, transforms=xf)
        out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
        s.apply(cuda(phi), out)
        got[xf] = out.cpu().numpy()
        s.close()
    assert rel(got[XF_AUTO], want) < 1e-8
    assert rel(got[XF_STAGED], want) < 1e-8
    assert rel(got[XF_AUTO], got[XF_STAGED]) < 1e-10


def test_slab_interface_solve_navier_matches_oracle():
    geom, N, lam = ki.WORKLOADS["ell128_navier"][0], 32, 2.0
    o = okfbim.Setup(geom, ki.grid(N), lam=lam)
    phi = ki.random_density(o.n, seed=5)
    want = o.apply(phi)
    s = Solver(geom, ki.grid(N), precision=MIXED, lam=lam)
    out = torch.zeros(s.n_primary, dtype=torch.float64, device="cuda")
    s.apply(cuda(phi), out)
    assert rel(out.cpu().numpy(), want) < 1e-8
    s.close()
