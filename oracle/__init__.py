"""Plain FP64 CPU oracle of the kernel-free boundary integral (KFBI) method for
the 3D Stokes interior Dirichlet problem (arXiv 2303.04992).

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import it.  The CUDA
library never calls into it and shares no code with it.

The oracle restates the paper's steps in their order, with numpy/scipy
primitives (FFT-based DST, dense solves, a k-d tree for neighbour search) and
no fusion or reordering:

  geometry.py  level sets, normals, curvature             (Alg. 1 step 1)
  grid.py      staggered grids, sides, intersections       (Sec. 4.2, Alg. 1 step 1)
  mac.py       MAC operators, DST Poisson, Schur CG         (Sec. 4.2, Eq. linearS1)
  jumps.py     surface fits and jump conditions             (Sec. 4.3, Eqs. IUS-1..4)
  correct.py   right-hand-side corrections                  (Sec. 4.3 items 1-4)
  interp.py    ten-node quadratic trace interpolation       (Sec. 4.4)
  kfbim.py     interface solve, matvec, GMRES, final fields (Alg. 1 steps 2-3)
  adjoint.py   gradient of a velocity loss w.r.t. the boundary data, by the
               dense transpose of the forward maps (small grids)

Where the paper is silent, ambiguous or self-contradictory, each function
states the reading it relies on.
Parity status: every function is pinned by a `-m "not gpu"` test except the
control-point surface fit (the paper defers that design to earlier work), whose
choice of neighbourhood and weights is parity unpinned; it is covered only
through the end-to-end pins (constant density, rigid motion, convergence).
"""
