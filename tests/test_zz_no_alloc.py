"""The allocation-free Poisson entry point (kfbim_poisson_noalloc) against the
context-based kfbim_poisson, through the C ABI.  It exists for callers that
may not allocate device memory (a memory manager owns the device heap, or
cudaMalloc's implicit synchronisation is not allowed in their loop); its
scratch is a static device array shared by every call, so two consecutive
calls with different inputs must both match.  Collected last on purpose."""
import numpy as np
import pytest

import kfbim_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import Solver, build  # noqa: E402
from paper_2303_04992_gb300.binding import KfbimError, poisson_noalloc  # noqa: E402

build()


def _field(N, c, seed):
    r = np.random.default_rng(seed).standard_normal((N, N, N))
    sl = [slice(None)] * 3
    sl[2 - (c - 1)] = 0
    r[tuple(sl)] = 0.0
    return torch.from_numpy(r.ravel()).cuda()


@pytest.mark.parametrize("N", [32, 64])
def test_noalloc_poisson_matches_context_poisson_twice(N):
    s = Solver(ki.sphere(), ki.grid(N))
    for c in (1, 2, 3):
        for seed in (10 * c, 10 * c + 1):          # two calls in a row per component
            r = _field(N, c, seed)
            want = s.poisson(c, r, torch.zeros_like(r))
            got = poisson_noalloc(c, N, -1.0, 1.0, r, torch.full_like(r, np.nan))
            torch.cuda.synchronize()
            err = (got - want).abs().max().item() / want.abs().max().item()
            assert err < 1e-12, (N, c, seed, err)
    s.close()


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    r = torch.zeros(128 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(KfbimError) as e:
        poisson_noalloc(1, 128, -1.0, 1.0, r, torch.zeros_like(r))
    assert e.value.code == -1
