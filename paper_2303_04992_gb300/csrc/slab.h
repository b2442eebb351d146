// Host entry of the four-kernel FP32 Schur CG iteration of slab.cuh
// (Sec. 4.2, Eq. linearS1), compiled in its own translation unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kfbim {

struct CGScalars;
template <typename T>
struct C2;

// One CG run's buffers: x, r, d, q (N^3 floats each), z1 and z3 (two N^3
// float temporaries), the FP32 transform tables (full-circle twiddles
// exp(-2 pi i t / 2N), t < 2N; post-twiddles exp(-i pi k / 2N), k < N; the
// eigenvalue table 4 sin^2 of the DCT (N) and DST (N) modes), 1/mu, the
// device scalars and the reduction partials (>= 1216 doubles).
struct SlabCg {
  int N;
  float *x, *r, *d, *q, *z1, *z3;
  const C2<float>* tw;
  const C2<float>* qN;
  const float* s2;
  float inv_mu;
  CGScalars* s;
  double* partial;
};

// Largest number of CG runs one launch of the iteration's kernels serves.
constexpr int kSlabBatchMax = 64;

// The iteration for `nrun` independent CG runs on one grid at once
// (blockIdx.y = run; each run's arithmetic and reduction order are those of a
// single run): run k uses the buffers and scalars of runs[k], which hold the
// shared tables too (only runs[0]'s tables, N and inv_mu are read).
int slab_cg_iteration_batch(const SlabCg* runs, int nrun, cudaStream_t st);

// Grids the four-kernel iteration covers (N = 32, 64, 128: a whole plane of
// floats and its team exchange buffers fit in one CTA's shared memory).
bool slab_supported(int N);
// Raises the kernels' dynamic shared-memory limits on the current device.
cudaError_t slab_prepare(int N);
// Enqueues one CG iteration (a no-op on the device once s->done is set);
// returns the number of kernels launched.
int slab_cg_iteration(const SlabCg& a, cudaStream_t st);
// One kernel of the iteration (0 k_cg_zfwd, 1 k_cg_xy, 2 k_cg_zinv,
// 3 k_cg_upd), for per-kernel timing; returns the number launched (0 or 1).
int slab_launch(int which, const SlabCg& a, cudaStream_t st);
// Algorithmic bytes each kernel moves (FP32 values read and written):
// 5, 4, 4 and 6 N^3 floats.
constexpr int kSlabValues[4] = {5, 4, 4, 6};
// The first three kernels of an iteration only: with s->beta = 0 and
// s->done = 0 they leave d = r and q = S d (the three spectral terms plus
// s->cdiag d, without the rank-one term) and set s->sumd, s->dq, s->alpha.
int slab_schur_apply(const SlabCg& a, cudaStream_t st);

}  // namespace kfbim
