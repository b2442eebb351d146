// The four-step transform pass kernels for N = 96 (pass2.h).
#include "pass2_impl.cuh"

KFBIM_PASS2_INSTANTIATE(96)
