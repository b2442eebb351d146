"""Pins of the oracle's grids, sides and intersections (Sec. 4.2, Alg. 1 step 1)."""
import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import geometry, grid as gridmod


@pytest.mark.parametrize("geom", [ki.sphere(), ki.star()], ids=["sphere", "star"])
def test_points_on_surface_and_lines(geom):
    g = gridmod.Grid(24, -1.0, 1.0)
    cp, S = gridmod.control_points(g, geom)
    F = geometry.level_value(geom, cp.xyz)
    assert np.abs(F).max() < 1e-13
    assert np.all((cp.theta >= 0) & (cp.theta < 1))
    # coordinates across the line are those of grid c's nodes
    for m in range(0, cp.n, 97):
        c, a = cp.comp[m], cp.axis[m]
        node = g.node_xyz(c, cp.idx[m])
        for b in range(3):
            if b != a:
                assert cp.xyz[m, b] == node[b]
        assert node[a] <= cp.xyz[m, a] <= node[a] + g.h


def test_counts_match_brute_force():
    """Count of sign changes along every grid line by explicit loops."""
    geom = ki.sphere(0.43, (0.03, -0.02, 0.05))
    N = 12
    g = gridmod.Grid(N, -1.0, 1.0)
    cp, _ = gridmod.control_points(g, geom)
    for c in (1, 2, 3):
        for a in range(3):
            count = 0
            rng_idx = [range(1, N) if b == c - 1 else range(N) for b in range(3)]
            for i in rng_idx[0]:
                for j in rng_idx[1]:
                    for k in rng_idx[2]:
                        idx = [i, j, k]
                        nxt = list(idx)
                        nxt[a] += 1
                        if nxt[a] >= N:
                            continue
                        f0 = geometry.level_value(geom, g.node_xyz(c, np.array(idx))[None])[0]
                        f1 = geometry.level_value(geom, g.node_xyz(c, np.array(nxt))[None])[0]
                        count += (f0 <= 0) != (f1 <= 0)
            assert count == np.sum((cp.comp == c) & (cp.axis == a))


def test_canonical_order():
    g = gridmod.Grid(20, -1.0, 1.0)
    cp, _ = gridmod.control_points(g, ki.star())
    key = []
    for m in range(cp.n):
        a = cp.axis[m]
        other = [b for b in range(3) if b != a]
        key.append((cp.comp[m], a, cp.idx[m][other[1]], cp.idx[m][other[0]], cp.idx[m][a]))
    assert key == sorted(key)


def test_rejects_interface_near_wall():
    g = gridmod.Grid(16, -1.0, 1.0)
    geom = ki.sphere(0.95)
    cp, S = gridmod.control_points(g, geom)
    with pytest.raises(ValueError):
        gridmod.check_geometry(g, geom, cp, S)
