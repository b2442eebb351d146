"""Device memory through a caller's allocator (kfbim_setup_ex): with torch's
caching allocator the context's workspace shows up in
torch.cuda.memory_allocated, is handed back at kfbim_destroy, and the solver
computes bit for bit what it computes on cudaMalloc memory."""
import numpy as np
import pytest

import kfbim_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import MIXED, KfbimError, Solver, build  # noqa: E402

build()


def test_torch_allocator_holds_the_workspace():
    geom, grid, N = ki.star(), ki.grid(64), 64
    s0 = Solver(geom, grid, precision=MIXED)
    phi = torch.from_numpy(ki.random_density(s0.n_primary, seed=3)).cuda()
    out0 = torch.zeros_like(phi)
    out1 = torch.zeros_like(phi)
    torch.cuda.synchronize()
    base = torch.cuda.memory_allocated()
    s1 = Solver(geom, grid, precision=MIXED, allocator="torch")
    held = torch.cuda.memory_allocated() - base
    assert held > 20 * N ** 3 * 8          # FP64 and FP32 grid workspace, tables
    s0.apply(phi, out0)
    s1.apply(phi, out1)
    torch.cuda.synchronize()
    assert torch.equal(out0, out1)
    s1.close()
    assert torch.cuda.memory_allocated() == base
    s0.close()


def test_unknown_allocator_is_rejected():
    with pytest.raises(KfbimError) as e:
        Solver(ki.sphere(), ki.grid(16), allocator="pool")
    assert e.value.code == -1
