"""The C-ABI library builds, loads and exports every symbol of include/kfbim.h
(no GPU needed); its host setup reproduces the oracle's control points."""
import os
import re

import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim as okfbim
from paper_2303_04992_gb300 import build
from paper_2303_04992_gb300.binding import SYMBOLS, KfbimError, Solver, load_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "kfbim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kfbim_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    build()
    lib = load_library()
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in SYMBOLS, n


def test_host_setup_matches_oracle_points():
    for geom, grid in [(ki.sphere(), ki.grid(32)), (ki.star(), ki.grid(32)),
                       (ki.ellipsoid((0.6, 0.45, 0.35), ki.seeded_rotation(3)), ki.grid(32)),
                       (ki.example53_geometry(), ki.grid(64, -1.2, 1.2))]:
        s = Solver(geom, grid, device=False)
        o = okfbim.Setup(geom, grid)
        xyz, comp, axis, prim = s.points()
        assert s.n_points == o.cp.n and s.n_primary == o.n
        assert np.array_equal(comp, o.cp.comp) and np.array_equal(axis, o.cp.axis)
        assert np.array_equal(prim, o.primary)
        assert np.abs(xyz - o.cp.xyz).max() < 1e-14
        for c in range(4):
            assert np.array_equal(s.sides(c), o.S[c])
        s.close()


def test_control_points_are_the_density_blocks():
    """kfbim_control_points(c) lists component c's density unknowns in the
    order of its block of g and phi; kfbim_jump_points lists every control
    point (where f is needed), in the order of fpts."""
    geom, grid = ki.star(), ki.grid(32)
    s = Solver(geom, grid, device=False)
    o = okfbim.Setup(geom, grid)
    xyz, comp, _, prim = s.points()
    nrm = s.normals()
    blocks = []
    for c in (1, 2, 3):
        cx, cn = s.control_points(c)
        sel = prim & (comp == c)
        assert np.array_equal(cx, xyz[sel]) and np.array_equal(cn, nrm[sel])
        assert np.abs(cx - o.cp.xyz[o.primary & (o.cp.comp == c)]).max() < 1e-14
        blocks.append(cx)
    # the blocks concatenated are the primary points in density order
    assert np.array_equal(np.concatenate(blocks), xyz[prim])
    assert np.array_equal(s.jump_points(), xyz)
    with pytest.raises(KfbimError) as e:
        s.control_points(0)
    assert e.value.code == -1
    s.close()


def test_host_setup_navier_matches_oracle_points():
    geom = ki.ellipsoid((0.6, 0.45, 0.35), ki.seeded_rotation(3))
    s = Solver(geom, ki.grid(32), device=False, lam=2.0)
    o = okfbim.Setup(geom, ki.grid(32), lam=2.0)
    _, comp, _, prim = s.points()
    assert np.array_equal(prim, o.primary) and np.array_equal(comp, o.cp.comp)
    with __import__("pytest").raises(KfbimError):
        Solver(geom, ki.grid(32), device=False, lam=-3.0)   # lambda + mu <= 0
    s.close()


def test_host_setup_rejects_bad_geometry():
    import pytest
    with pytest.raises(KfbimError) as e:
        Solver(ki.sphere(0.95), ki.grid(16), device=False)
    assert e.value.code == -2
    with pytest.raises(KfbimError) as e:
        Solver(ki.sphere(), ki.grid(24), device=False)      # not a power of two, not 96
    assert e.value.code == -1
    with pytest.raises(KfbimError) as e:
        Solver(ki.sphere(), ki.grid(80), device=False)
    assert e.value.code == -1


def test_host_setup_accepts_96():
    """N = 96, the one grid size that is not a power of two (its transforms
    have a 24-point stage); the host tables match the oracle's points."""
    from oracle import kfbim as okfbim
    s = Solver(ki.sphere(), ki.grid(96), device=False)
    o = okfbim.Setup(ki.sphere(), ki.grid(96))
    xyz, comp, axis, prim = s.points()
    assert s.N == 96 and s.n_primary == o.n
    assert np.array_equal(comp, o.cp.comp) and np.array_equal(prim, o.primary)
    assert np.abs(xyz - o.cp.xyz).max() < 1e-14
    s.close()


def test_host_only_context_refuses_device_calls():
    import pytest
    s = Solver(ki.sphere(), ki.grid(16), device=False)
    with pytest.raises(KfbimError) as e:
        s._check(s._lib.kfbim_apply(s._ctx, None, None, None))
    assert e.value.code == -1


def test_callback_sphere_reproduces_the_builtin_setup():
    """A caller-supplied level set with the built-in sphere's arithmetic gives
    the same control points, sides and tables, bit for bit."""
    a = Solver(ki.sphere(), ki.grid(32), device=False)
    b = Solver(ki.callback_sphere(), ki.grid(32), device=False)
    assert (a.n_points, a.n_primary) == (b.n_points, b.n_primary)
    assert a.table_sizes() == b.table_sizes()
    for x, y in zip(a.points(), b.points()):
        assert np.array_equal(x, y)
    for c in range(4):
        assert np.array_equal(a.sides(c), b.sides(c))


def test_callback_peanut_matches_oracle_points():
    """A non-convex shape that no built-in kind covers (a Cassini surface of
    revolution with a waist), through the CALLBACK kind, against the oracle
    evaluating the same level set."""
    geom = ki.peanut()
    s = Solver(geom, ki.grid(32), device=False)
    o = okfbim.Setup(geom, ki.grid(32))
    xyz, comp, axis, prim = s.points()
    assert s.n_points == o.cp.n and s.n_primary == o.n
    assert np.array_equal(comp, o.cp.comp) and np.array_equal(axis, o.cp.axis)
    assert np.array_equal(prim, o.primary)
    assert np.abs(xyz - o.cp.xyz).max() < 1e-14
    for c in range(4):
        assert np.array_equal(s.sides(c), o.S[c])


def test_callback_geometry_errors():
    import ctypes
    import pytest
    from paper_2303_04992_gb300.binding import Geometry, Grid, Options
    lib = load_library()
    o = Options()
    lib.kfbim_default_options(ctypes.byref(o))
    g = Geometry()
    g.kind = 4                                          # CALLBACK without functions
    ctx = ctypes.c_void_p()
    assert lib.kfbim_setup_host(ctypes.byref(g), ctypes.byref(Grid(32, -1.0, 1.0)), ctypes.byref(o),
                                ctypes.byref(ctx)) == -1
    assert not ctx.value
    flat = dict(ki.peanut())
    flat["derivs"] = lambda x: ([0.0, 0.0, 0.0], [[0.0] * 3] * 3)   # vanishing gradient
    with pytest.raises(KfbimError) as e:
        Solver(flat, ki.grid(32), device=False)
    assert e.value.code == -2


def test_normals_match_the_oracle_frames():
    from oracle import geometry
    for geom in (ki.star(), ki.peanut(), ki.sphere(0.45, (0.01, -0.02, 0.0))):
        s = Solver(geom, ki.grid(32), device=False)
        xyz = s.points()[0]
        got = s.normals()
        want = geometry.frames(geom, xyz)[0]
        assert np.abs(got - want).max() < 1e-13
        assert np.abs(np.linalg.norm(got, axis=1) - 1.0).max() < 1e-14
        if geom["kind"] == "sphere":
            d = xyz - np.array(geom["center"])
            assert np.abs(got - d / np.linalg.norm(d, axis=1)[:, None]).max() < 1e-13


def test_grazing_sphere_matches_oracle_points():
    """A sphere whose surface grazes grid lines (a chord shorter than h between
    two same-side faces, the cell centre between them on the other side): the
    two roots of each such segment are secondary control points, in the
    library's host setup exactly as in the oracle."""
    geom, grid = ki.sphere(0.5, (0.01, -0.02, 0.0)), ki.grid(32)
    s = Solver(geom, grid, device=False)
    o = okfbim.Setup(geom, grid)
    assert int(np.sum(o.cp.graze > 0)) == 4 and not np.any(o.primary[o.cp.graze > 0])
    xyz, comp, axis, prim = s.points()
    assert s.n_points == o.cp.n and s.n_primary == o.n
    assert np.array_equal(comp, o.cp.comp) and np.array_equal(axis, o.cp.axis)
    assert np.array_equal(prim, o.primary)
    assert np.abs(xyz - o.cp.xyz).max() < 1e-14
    for c in range(4):
        assert np.array_equal(s.sides(c), o.S[c])


def test_correction_rows_match_the_oracle():
    """The library's correction table touches exactly the right-hand-side
    rows the oracle's corrections touch (random jumps), for built-in, CALLBACK
    and grazing geometries."""
    from oracle import correct as ocorrect
    for geom in (ki.sphere(), ki.star(), ki.peanut(), ki.sphere(0.5, (0.01, -0.02, 0.0))):
        o = okfbim.Setup(geom, ki.grid(32))
        J = np.random.default_rng(1).standard_normal((o.cp.n, 12))
        Cf, Cg = ocorrect.corrections(o.grid, o.cp, o.S, J, 1.0)
        rows = sum(int(np.count_nonzero(f)) for f in Cf) + int(np.count_nonzero(Cg))
        s = Solver(geom, ki.grid(32), device=False)
        assert s.table_sizes()[1] == rows


def test_random_sphere_placements_set_up_like_the_oracle():
    """Generic placements (radius and centre drawn at random) all set up; many
    graze grid lines, which were rejected before grazing segments got their two
    roots.  Points, flags and sides agree with the oracle."""
    rng = np.random.default_rng(2024)
    grazing = 0
    for _ in range(8):
        geom = ki.sphere(rng.uniform(0.35, 0.55), tuple(rng.uniform(-0.05, 0.05, 3)))
        s = Solver(geom, ki.grid(32), device=False)
        o = okfbim.Setup(geom, ki.grid(32))
        grazing += int(np.any(o.cp.graze > 0))
        xyz, comp, axis, prim = s.points()
        assert s.n_points == o.cp.n and np.array_equal(prim, o.primary)
        assert np.array_equal(comp, o.cp.comp) and np.array_equal(axis, o.cp.axis)
        assert np.abs(xyz - o.cp.xyz).max() < 1e-14
        assert np.array_equal(s.sides(0), o.S[0])
    assert grazing >= 2


def test_callback_exception_is_raised_after_setup():
    import pytest
    geom = dict(ki.peanut())

    def bad(x):
        raise ZeroDivisionError("level set failed")

    geom["F"] = bad
    with pytest.raises(ZeroDivisionError):
        Solver(geom, ki.grid(16), device=False)


def _bad_setup_cases():
    good_geom, good_grid = ki.sphere(), ki.grid(32)
    return [
        ("N not a power of two", good_geom, ki.grid(48), {}),
        ("N below 16", good_geom, ki.grid(8), {}),
        ("N above 256", good_geom, ki.grid(512), {}),
        ("empty box", good_geom, {"N": 32, "lo": 1.0, "hi": 1.0}, {}),
        ("mu <= 0", good_geom, good_grid, {"mu": 0.0}),
        ("gmres_max 0", good_geom, good_grid, {"gmres_max": 0}),
        ("gmres_max 201", good_geom, good_grid, {"gmres_max": 201}),
        ("cg_max 0", good_geom, good_grid, {"cg_max": 0}),
        ("precision 7", good_geom, good_grid, {"precision": 7}),
        ("pde 5", good_geom, good_grid, {"pde": 5}),
        ("transforms 9", good_geom, good_grid, {"transforms": 9}),
        ("lambda + mu <= 0", good_geom, good_grid, {"lam": -2.0}),
        ("torus a >= c", ki.torus(0.5, 0.4), good_grid, {}),
    ]


@pytest.mark.parametrize("case", _bad_setup_cases(), ids=lambda c: c[0])
def test_setup_rejects_invalid_arguments(case):
    _, geom, grid, opts = case
    with pytest.raises(KfbimError) as e:
        Solver(geom, grid, device=False, **opts)
    assert e.value.code == -1
    # the library stays usable
    Solver(ki.sphere(), ki.grid(16), device=False).close()
