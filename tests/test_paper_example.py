"""Loose check against the paper's own table for Example 5.1 at N = 64
(golden values in tests/golden/paper_example51.json, cited there).  The
paper's control-point classification and fit are not specified, so only the
order of magnitude of the errors and the GMRES count are compared."""
import json
import os

import numpy as np
import pytest

import kfbim_inputs as ki
from oracle import kfbim

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_example51.json")))


@pytest.mark.slow
def test_example51_against_paper_table():
    geom = ki.sphere(GOLD["radius"])
    grid = ki.grid(GOLD["N"], *GOLD["box"])
    s = kfbim.Setup(geom, grid)
    rows = np.arange(s.cp.n)
    g = ki.example51_velocity(s.cp.xyz)[rows, s.cp.comp - 1][s.primary]
    fy = ki.example51_forcing(s.cp.xyz)
    ff = [ki.example51_forcing(s.grid.node_xyz(c, s.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    r = s.solve(g, fy, ff, tol=GOLD["gmres_tol"])
    errs = {}
    for c in (1, 2, 3):
        X = s.grid.node_xyz(c, s.grid.all_idx())
        ue = ki.example51_velocity(X)[..., c - 1]
        m = s.S[c] & s.grid.unknown_mask(c)
        errs["u%d" % c] = np.abs(r["u"][c - 1] - ue)[m].max() / np.abs(ue[m]).max()
    X0 = s.grid.node_xyz(0, s.grid.all_idx())
    pe = ki.example51_pressure(X0)
    m = s.S[0]
    d = (r["p"] - pe)[m]
    d -= d.mean()
    errs["p"] = np.abs(d).max() / np.abs(pe[m] - pe[m].mean()).max()
    assert 0.5 * GOLD["gmres_iterations"] <= r["iters"] <= 2.0 * GOLD["gmres_iterations"]
    for k, v in GOLD["max_error"].items():
        assert errs[k] < 4.0 * v, (k, errs[k], v)
