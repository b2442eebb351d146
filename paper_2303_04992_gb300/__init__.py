"""GB300 kernel-free boundary integral (KFBI) solver for the 3D Stokes interior
Dirichlet problem (arXiv 2303.04992).

The compute path is the CUDA library built from csrc/ (libkfbim.so, C ABI in
include/kfbim.h).  This package is the thin Python binding: `Solver` marshals
torch tensors (device memory, current stream) into the C calls.  Importing the
package loads nothing; the first `Solver(...)` loads the library and fails
loudly when it has not been built.
"""
from .binding import Solver, KfbimError, load_library, library_path  # noqa: F401
from .build import build  # noqa: F401
from .autograd import solve_velocity  # noqa: F401

FP64 = 0
MIXED = 1
FP32 = 2         # FP32 grid solve without FP64 refinement (matvec ~1e-6)
MIXED_TF32 = 3   # MIXED on tensor-core (3xTF32) transform passes, N = 128
XF_AUTO = 0      # slab CG; one-axis passes: timed choice per stage kind
XF_FFT = 1       # slab CG; four-step FFT one-axis passes
XF_TENSOR = 2    # tcgen05 transform-matrix GEMM passes (N = 128), CG included
XF_STAGED = 3    # one-axis FFT passes everywhere, CG included
