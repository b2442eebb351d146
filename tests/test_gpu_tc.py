"""Tensor-core (tcgen05, 3xTF32) transform passes at N = 128 against the FFT
passes: every transform type and axis, with and without the spectral weights
(the FFT passes are themselves pinned to the oracle through the solver parity
tests), then whole MIXED matvecs and solves run on tensor-core passes against
the FFT-pass solver and the FP64 solver, and the autotuner's record."""
import numpy as np
import pytest

import kfbim_inputs as ki

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2303_04992_gb300 import (FP64, MIXED, XF_AUTO, XF_FFT, XF_TENSOR, KfbimError,  # noqa: E402
                                    Solver, build)

build()

N = 128
# transform types (transforms.cuh): 1 DCT2F, 2 DCT2I, 3 DST2F, 4 DST2I, 5 DST1F, 6 DST1I
PLAIN = [(t, ax, 0, 0) for t in range(1, 7) for ax in range(3)]
WEIGHTED = ([(1, c, 1, c) for c in range(3)] + [(5, c, 2, c) for c in range(3)]
            + [(5, c, 3, c) for c in range(3)])


@pytest.fixture(scope="module")
def tc_solver():
    return Solver(ki.sphere(), ki.grid(N), precision=MIXED, transforms=XF_TENSOR)


@pytest.mark.parametrize("case", PLAIN + WEIGHTED, ids=lambda c: "t%d_ax%d_w%d_c%d" % c)
def test_tc_pass_matches_fft_pass(tc_solver, case):
    xform, axis, wmode, wc = case
    g = torch.Generator(device="cuda").manual_seed(1000 + 10 * xform + axis)
    x = torch.randn(N ** 3, generator=g, device="cuda", dtype=torch.float32)
    a = torch.empty_like(x)
    b = torch.empty_like(x)
    tc_solver.transform_f32(xform, axis, x, a, XF_FFT, wmode, wc)
    tc_solver.transform_f32(xform, axis, x, b, XF_TENSOR, wmode, wc)
    torch.cuda.synchronize()
    err = float((a - b).abs().max() / a.abs().max())
    assert err < 5e-6, err


def test_tc_pass_in_place_and_double_pass(tc_solver):
    g = torch.Generator(device="cuda").manual_seed(7)
    x = torch.randn(N ** 3, generator=g, device="cuda", dtype=torch.float32)
    y = x.clone()
    tc_solver.transform_f32(3, 2, y, y, XF_TENSOR)        # DST-II along z, in place
    tc_solver.transform_f32(4, 2, y, y, XF_TENSOR)        # and back
    torch.cuda.synchronize()
    assert float((y - x).abs().max() / x.abs().max()) < 5e-6


def test_tc_pass_rejected_off_128():
    s = Solver(ki.sphere(), ki.grid(64), precision=MIXED)
    x = torch.zeros(64 ** 3, device="cuda", dtype=torch.float32)
    with pytest.raises(KfbimError) as e:
        s.transform_f32(1, 0, x, x, XF_TENSOR)
    assert e.value.code == -1
    assert s.transforms_info()["plain"] == 0 and s.transforms_info()["fused"] == 0


def _manufactured(s):
    xyz, comp, _, prim = s.points()
    rows = np.arange(len(comp))
    g = ki.stokes_velocity(xyz)[rows, comp - 1][prim]
    fp = ki.stokes_forcing(xyz).T.copy()
    lo, h = s.lo, s.h
    idx = np.arange(N)
    fg = []
    for c in (1, 2, 3):
        off = [0.5, 0.5, 0.5]
        off[c - 1] = 0.0
        Z, Y, X = np.meshgrid(lo + (idx + off[2]) * h, lo + (idx + off[1]) * h,
                              lo + (idx + off[0]) * h, indexing="ij")
        fg.append(ki.stokes_forcing(np.stack([X, Y, Z], -1))[..., c - 1].ravel())
    return [torch.from_numpy(a).cuda() for a in (g, fp, np.concatenate(fg))]


@pytest.fixture(scope="module")
def star_pair():
    # relax = 0: every matvec refined to refine_tol, so that the GMRES
    # iteration count compares with the FP64 solve's (the relaxed form takes
    # a few more iterations by design; tests/test_gpu_star128_oracle.py)
    geom, grid = ki.WORKLOADS["star128"]
    return (Solver(geom, grid, precision=MIXED, transforms=XF_TENSOR, relax=0.0),
            Solver(geom, grid, precision=MIXED, transforms=XF_FFT, relax=0.0))


def test_tc_apply_matches_fft_apply(star_pair):
    s_tc, s_fft = star_pair
    phi = torch.from_numpy(np.random.default_rng(11).standard_normal(s_tc.n_primary)).cuda()
    a = torch.zeros_like(phi)
    b = torch.zeros_like(phi)
    s_tc.apply(phi, a)
    s_fft.apply(phi, b)
    torch.cuda.synchronize()
    assert float((a - b).abs().max() / b.abs().max()) < 1e-9


def test_tc_solve_matches_fp64(star_pair):
    s_tc, _ = star_pair
    geom, grid = ki.WORKLOADS["star128"]
    s64 = Solver(geom, grid, precision=FP64)
    g, fp, fg = _manufactured(s_tc)
    phi = torch.zeros(s_tc.n_primary, dtype=torch.float64, device="cuda")
    phi64 = torch.zeros_like(phi)
    s_tc.solve(g, phi, fp, fg)
    st = dict(s_tc.last_stats)
    s64.solve(g, phi64, fp, fg)
    torch.cuda.synchronize()
    assert float((phi - phi64).abs().max() / phi64.abs().max()) < 1e-8
    assert abs(st["gmres_iters"] - s64.last_stats["gmres_iters"]) <= 3
    # the coarser accumulation costs at most a third refinement sweep per interface solve
    assert st["refine_sweeps"] <= 3 * st["interface_solves"]


def test_autotuner_record():
    geom, grid = ki.WORKLOADS["star128"]
    s = Solver(geom, grid, precision=MIXED, transforms=XF_AUTO)
    info = s.transforms_info()
    ms = info["tune_ms"]
    assert all(m > 0 for m in ms)
    # a tensor-core stage must beat the FFT stage by the iteration factor 1.5
    assert info["plain"] == int(ms[1] * 1.5 < ms[0])
    assert info["fused"] == int(ms[3] * 1.5 < ms[2])
