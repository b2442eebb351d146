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
XF_AUTO = 0      # FP32 axis passes: timed choice per stage kind
XF_FFT = 1       # four-step FFT passes
XF_TENSOR = 2    # tcgen05 transform-matrix GEMM passes (N = 128)
