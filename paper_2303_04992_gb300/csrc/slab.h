// Host entry of the three-kernel FP32 Schur CG iteration of slab.cuh
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
// device scalars and the reduction partials (at least 4 (N / 32) N slots of
// eight bytes: k_cg_zinv stores four FP32 pairs per block).
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

// Grids the slab iteration covers (N = 32, 64, 128: a whole plane of
// floats and its team exchange buffers fit in one CTA's shared memory).
bool slab_supported(int N);
// Raises the kernels' dynamic shared-memory limits on the current device.
cudaError_t slab_prepare(int N);
// Enqueues one CG iteration (a no-op on the device once s->done is set);
// returns the number of kernels launched.  Each iteration leaves its own
// vector update (x += alpha d, r -= alpha q) pending for the next one, so
// a run that has stopped needs slab_cg_finish (or the batch form) before x
// is read.
int slab_cg_iteration(const SlabCg& a, cudaStream_t st);
// x += alpha d, the update still pending when the run stopped (whether by
// done or by an iteration cap); returns the number of kernels launched.
int slab_cg_finish(const SlabCg& a, cudaStream_t st);
int slab_cg_finish_batch(const SlabCg* runs, int nrun, cudaStream_t st);
// One kernel of the iteration (0 k_cg_zfwd, 1 k_cg_xy, 2 k_cg_zinv; 3 the
// finishing update), for per-kernel timing; returns the number launched.
int slab_launch(int which, const SlabCg& a, cudaStream_t st);
// Algorithmic bytes each kernel moves (FP32 values read and written, with
// an update pending): 9, 4, 5 and 3 N^3 floats.
constexpr int kSlabValues[4] = {9, 4, 5, 3};
// The three kernels of one iteration from a fresh run: with s->alpha = 0,
// s->beta = 0 and s->done = 0 they leave d = r and q = S d (the three
// spectral terms plus s->cdiag d plus s->rank1 sum(d)) and set s->sumd,
// s->dq, s->alpha.
int slab_schur_apply(const SlabCg& a, cudaStream_t st);

}  // namespace kfbim
