"""The binding's argument checks (no GPU): every device call refuses, before
calling the library, a tensor of the wrong dtype, a non-contiguous one, one
with fewer values than include/kfbim.h gives for the call, and a host tensor;
exactly sized arguments reach the library unchanged.  A tensor subclass that
reports itself as a CUDA tensor and a fake library that records its calls
stand in for the GPU."""
import ctypes

import numpy as np
import pytest

import kfbim_inputs as ki
from paper_2303_04992_gb300 import KfbimError, build
from paper_2303_04992_gb300.binding import Solver

torch = pytest.importorskip("torch")


class FakeCuda(torch.Tensor):
    @property
    def is_cuda(self):
        return True

    @property
    def device(self):
        return torch.device("cuda", 0)


class FakeLib:
    def __init__(self):
        self.calls = []

    def kfbim_last_error(self, ctx):
        return b"fake"

    def __getattr__(self, name):
        def call(*args):
            self.calls.append((name, args))
            return 0
        return call


N, NPT, NPRIM = 8, 10, 7
N3 = N ** 3


def fake_solver():
    s = Solver.__new__(Solver)
    s._lib, s._ctx, s._device = FakeLib(), ctypes.c_void_p(1), 0
    s.N, s.n_points, s.n_primary = N, NPT, NPRIM
    s.last_stats = None
    s._stream = lambda: None
    return s


def dev(n, dtype=torch.float64):
    return torch.zeros(n, dtype=dtype).as_subclass(FakeCuda)


# method, its device arguments in call order with their sizes, extra leading args
CASES = {
    "apply": ([NPRIM, NPRIM], ()),
    "solve": ([NPRIM, NPRIM, 3 * NPT, 3 * N3, 3 * N3, N3], ()),
    "apply_adjoint": ([NPRIM, NPRIM], ()),
    "solve_adjoint": ([3 * N3, NPRIM], ()),
    "jumps": ([NPRIM, 12 * NPT, 3 * NPT], ()),
    "interface": ([NPRIM, 3 * N3, N3, 3 * NPT, 3 * N3], ()),
    "pressure_trace": ([N3, 12 * NPT, NPT], ()),
    "trace": ([3 * N3, 12 * NPT, NPRIM], ()),
    "poisson": ([N3, N3], (1,)),
    "schur_apply": ([N3, N3], ()),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_exact_sizes_reach_the_library(name):
    sizes, lead = CASES[name]
    s = fake_solver()
    ts = [dev(n) for n in sizes]
    getattr(s, name)(*lead, *ts)
    assert len(s._lib.calls) == 1
    ptrs = {a.value for a in s._lib.calls[0][1] if isinstance(a, ctypes.c_void_p)}
    assert {t.data_ptr() for t in ts} <= ptrs


@pytest.mark.parametrize("name", sorted(CASES))
def test_short_wrong_dtype_strided_and_host_tensors_are_refused(name):
    sizes, lead = CASES[name]
    for k in range(len(sizes)):
        bad = [dev(sizes[k] - 1),                                  # one value short
               dev(sizes[k], torch.float32),                       # wrong dtype
               dev(2 * sizes[k])[::2],                             # not contiguous
               torch.zeros(sizes[k], dtype=torch.float64)]         # host tensor
        for b in bad:
            s = fake_solver()
            ts = [dev(n) for n in sizes]
            ts[k] = b
            with pytest.raises(KfbimError) as e:
                getattr(s, name)(*lead, *ts)
            assert e.value.code == -1
            assert s._lib.calls == []


def test_transform_f32_takes_float32():
    s = fake_solver()
    s.transform_f32(1, 0, dev(N3, torch.float32), dev(N3, torch.float32), 1)
    assert len(s._lib.calls) == 1
    with pytest.raises(KfbimError):
        s.transform_f32(1, 0, dev(N3), dev(N3), 1)


def test_solve_batch_sizes_scale_with_B():
    s = fake_solver()
    B = 3
    s.solve_batch(dev((B, NPRIM)).reshape(B, NPRIM), dev(B * NPRIM), dev(B * 3 * NPT), dev(B * 3 * N3),
                  dev(B * 3 * N3), dev(B * N3))
    assert s._lib.calls[0][0] == "kfbim_solve_batch" and s._lib.calls[0][1][1] == B
    with pytest.raises(KfbimError):
        s.solve_batch(dev((B, NPRIM)).reshape(B, NPRIM), dev(B * NPRIM - 1))
    assert len(s._lib.calls) == 1


def test_other_device_is_refused():
    s = fake_solver()
    s._device = 1
    with pytest.raises(KfbimError) as e:
        s.apply(dev(NPRIM), dev(NPRIM))
    assert "cuda:1" in str(e.value)


def test_solve_host_checks_numpy_buffers():
    s = fake_solver()
    s.solve_host(np.zeros(NPRIM), np.zeros(NPRIM), None, None, np.zeros(3 * N3), np.zeros(N3))
    assert s._lib.calls[0][0] == "kfbim_solve_host"
    for bad in (np.zeros(NPRIM - 1), np.zeros(NPRIM, np.float32), np.zeros(2 * NPRIM)[::2],
                torch.zeros(NPRIM, dtype=torch.float64)):
        with pytest.raises(KfbimError):
            s.solve_host(np.zeros(NPRIM), bad)
    assert len(s._lib.calls) == 1


def test_host_context_points_and_sides_still_work():
    build()
    s = Solver(ki.sphere(), ki.grid(16), device=False)
    xyz, comp, axis, prim = s.points()
    assert xyz.shape == (s.n_points, 3) and prim.sum() == s.n_primary
    assert s.sides(0).sum() > 0
