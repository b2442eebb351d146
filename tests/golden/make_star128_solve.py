"""Writes star128_solve.npz: the FP64 oracle's full solve (Alg. 1 step 3 and
the final interface solve) of the headline workload, for the GPU parity test
of the same solve at full size.

Workload: the star r(theta, phi) = 0.5 + 0.1 sin(3 theta) cos(4 phi) in
[-1, 1]^3, MAC grid 128^3, mu = 1; boundary data and forcing from the
manufactured field of kfbim_inputs (u = (sin x cos y cos z, -cos x sin y cos z,
0), p = sin(x + y + z)).  The inputs are analytic, so the file stores no
input: only the oracle's outputs.

GMRES runs to a relative residual of 1e-13 (not the workload's 1e-10) so that
the stored density is the discrete solution to about kappa(A) * 1e-13 and a
GPU solve can be compared with it at 1e-10 without the two GMRES stopping
points dominating the difference.

Stored: phi at every primary control point (the full density); per velocity
component and for the pressure, the values at 4096 seeded node indices and
the max-norm of the whole field; the GMRES iteration count and residual.
Only oracle/ and kfbim_inputs are called.  About 12 minutes on one core:
    python tests/golden/make_star128_solve.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import kfbim_inputs as ki  # noqa: E402
from oracle import kfbim as okfbim  # noqa: E402

SAMPLES = 4096
GMRES_TOL = 1e-13
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "star128_solve.npz")


def main():
    t0 = time.time()
    geom, grid = ki.WORKLOADS["star128"]
    o = okfbim.Setup(geom, grid)
    x = o.cp.xyz
    g = ki.stokes_velocity(x)[np.arange(o.cp.n), o.cp.comp - 1][o.primary]
    fy = ki.stokes_forcing(x)
    ff = [ki.stokes_forcing(o.grid.node_xyz(c, o.grid.all_idx()))[..., c - 1] for c in (1, 2, 3)]
    sol = o.solve(g, fy, ff, tol=GMRES_TOL, maxit=300)
    N = o.grid.N
    rng = np.random.default_rng(128)
    out = {"phi": sol["phi"], "gmres_iters": np.int64(sol["iters"]),
           "gmres_residual": np.float64(sol["res"][-1]), "gmres_tol": np.float64(GMRES_TOL),
           "N": np.int64(N)}
    for c in range(3):
        idx = rng.choice(N ** 3, SAMPLES, replace=False)
        out[f"u{c + 1}_idx"] = idx
        out[f"u{c + 1}_val"] = sol["u"][c].ravel()[idx]
        out[f"u{c + 1}_max"] = np.float64(np.abs(sol["u"][c]).max())
    idx = rng.choice(N ** 3, SAMPLES, replace=False)
    out["p_idx"] = idx
    out["p_val"] = sol["p"].ravel()[idx]
    out["p_max"] = np.float64(np.abs(sol["p"]).max())
    np.savez_compressed(OUT, **out)
    print(f"wrote {OUT}: {sol['iters']} GMRES iterations, residual {sol['res'][-1]:.3e}, "
          f"{time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
