// Host entry of the four-step transform pass of transforms2.cuh.  Each grid
// size's kernels are instantiated in a translation unit of their own
// (pass2_n32.cu ... pass2_n256.cu, and pass2_n96.cu) so that they compile in
// parallel.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "transforms2.cuh"

namespace kfbim {

// Jobs per launch of the batched form (3 per instance, 16 instances).
constexpr int kPass2BatchJobs = 48;

// Raises a kernel's dynamic shared-memory limit on the current device once.
cudaError_t raise_dynamic_smem(const void* kern, size_t bytes);

// One launch of k_axis_pass2 for grid N (32, 64, 96, 128 or 256) over njobs jobs
// (blockIdx.y = job), with the FP32 or FP64 tables of the context.
// Instantiated for (Tin, T, Tout) = (double, double, double), (double, float,
// float), (float, float, float) and MAXJ = 3, kPass2BatchJobs.
template <int N, typename Tin, typename T, typename Tout, int MAXJ>
cudaError_t pass2_launch(const PassJobs<Tin, Tout, MAXJ>& jobs, int njobs, const C2<T>* tw, const C2<T>* qN,
                         const T* s2, cudaStream_t s);

}  // namespace kfbim
