// Launchers of the three-kernel FP32 Schur CG iteration (slab.cuh).
#include <cuda_runtime.h>

#include "slab.cuh"
#include "slab.h"

namespace kfbim {

bool slab_supported(int N) { return N == 32 || N == 64 || N == 128; }

namespace {

constexpr int kFinBlocks = 608;   // 4 x 152 SMs

template <int N, int MAXB>
cudaError_t prepare_nb() {
  cudaError_t e = cudaFuncSetAttribute(slab::k_cg_xy<N, MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)slab::XySmem<N>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(slab::k_cg_zfwd<N, MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)slab::ZSmem<N>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(slab::k_cg_zinv<N, MAXB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)slab::ZSmem<N>::bytes);
  return e;
}

template <int N>
cudaError_t prepare_n() {
  cudaError_t e = prepare_nb<N, 1>();
  return e == cudaSuccess ? prepare_nb<N, kSlabBatchMax>() : e;
}

template <int MAXB>
slab::SlabArgs<MAXB> make_args(const SlabCg* runs, int nrun) {
  slab::SlabArgs<MAXB> a{};
  for (int k = 0; k < nrun; ++k) {
    a.x[k] = runs[k].x;
    a.r[k] = runs[k].r;
    a.d[k] = runs[k].d;
    a.q[k] = runs[k].q;
    a.z1[k] = runs[k].z1;
    a.z3[k] = runs[k].z3;
    a.s[k] = runs[k].s;
    a.partial[k] = runs[k].partial;
  }
  return a;
}

// Kernel `which` of the iteration: 0 k_cg_zfwd, 1 k_cg_xy, 2 k_cg_zinv; 3 is
// k_cg_fin, the update still pending when a run stops.
template <int N, int MAXB>
void launch_nb(int which, const slab::SlabArgs<MAXB>& args, const SlabCg& t, int nrun, cudaStream_t st) {
  using C = slab::Cfg<N>;
  const unsigned zblocks = (N / C::TILE) * N;
  switch (which) {
    case 0:
      slab::k_cg_zfwd<N, MAXB><<<dim3(zblocks, nrun), C::TILE_THREADS, slab::ZSmem<N>::bytes, st>>>(args, t.tw,
                                                                                                     t.qN);
      break;
    case 1:
      slab::k_cg_xy<N, MAXB><<<dim3(N, nrun), C::PLANE_THREADS, slab::XySmem<N>::bytes, st>>>(args, t.tw, t.qN,
                                                                                              t.s2, t.inv_mu);
      break;
    case 2:
      slab::k_cg_zinv<N, MAXB><<<dim3(zblocks, nrun), C::TILE_THREADS, slab::ZSmem<N>::bytes, st>>>(args, t.tw,
                                                                                                     t.qN);
      break;
    default: {
      const int64_t n4 = (int64_t)N * N * N / 4;
      const int64_t need = (n4 + slab::FIN_THREADS - 1) / slab::FIN_THREADS;
      const unsigned blocks = (unsigned)(need < kFinBlocks ? need : kFinBlocks);
      slab::k_cg_fin<MAXB><<<dim3(blocks, nrun), slab::FIN_THREADS, 0, st>>>(args, n4);
    }
  }
}

template <int N>
void launch_n(int which, const SlabCg& a, cudaStream_t st) {
  launch_nb<N, 1>(which, make_args<1>(&a, 1), a, 1, st);
}

template <int N>
void schur_n(const SlabCg& a, cudaStream_t st) {
  const slab::SlabArgs<1> args = make_args<1>(&a, 1);
  for (int k = 0; k < 3; ++k) launch_nb<N, 1>(k, args, a, 1, st);
}

template <int N>
void iteration_n(const SlabCg& a, cudaStream_t st) {
  const slab::SlabArgs<1> args = make_args<1>(&a, 1);
  for (int k = 0; k < 3; ++k) launch_nb<N, 1>(k, args, a, 1, st);
}

template <int N>
void iteration_batch_n(const SlabCg* runs, int nrun, cudaStream_t st) {
  const slab::SlabArgs<kSlabBatchMax> args = make_args<kSlabBatchMax>(runs, nrun);
  for (int k = 0; k < 3; ++k) launch_nb<N, kSlabBatchMax>(k, args, runs[0], nrun, st);
}

template <int N>
void finish_batch_n(const SlabCg* runs, int nrun, cudaStream_t st) {
  launch_nb<N, kSlabBatchMax>(3, make_args<kSlabBatchMax>(runs, nrun), runs[0], nrun, st);
}

}  // namespace

cudaError_t slab_prepare(int N) {
  switch (N) {
    case 128: return prepare_n<128>();
    case 64: return prepare_n<64>();
    case 32: return prepare_n<32>();
    default: return cudaErrorInvalidValue;
  }
}

int slab_cg_iteration(const SlabCg& a, cudaStream_t st) {
  switch (a.N) {
    case 128: iteration_n<128>(a, st); break;
    case 64: iteration_n<64>(a, st); break;
    case 32: iteration_n<32>(a, st); break;
    default: return 0;
  }
  return 3;
}

int slab_cg_iteration_batch(const SlabCg* runs, int nrun, cudaStream_t st) {
  if (nrun < 1 || nrun > kSlabBatchMax) return 0;
  switch (runs[0].N) {
    case 128: iteration_batch_n<128>(runs, nrun, st); break;
    case 64: iteration_batch_n<64>(runs, nrun, st); break;
    case 32: iteration_batch_n<32>(runs, nrun, st); break;
    default: return 0;
  }
  return 3;
}

int slab_cg_finish(const SlabCg& a, cudaStream_t st) { return slab_launch(3, a, st); }

int slab_cg_finish_batch(const SlabCg* runs, int nrun, cudaStream_t st) {
  if (nrun < 1 || nrun > kSlabBatchMax) return 0;
  switch (runs[0].N) {
    case 128: finish_batch_n<128>(runs, nrun, st); break;
    case 64: finish_batch_n<64>(runs, nrun, st); break;
    case 32: finish_batch_n<32>(runs, nrun, st); break;
    default: return 0;
  }
  return 1;
}

int slab_launch(int which, const SlabCg& a, cudaStream_t st) {
  if (which < 0 || which > 3) return 0;
  switch (a.N) {
    case 128: launch_n<128>(which, a, st); break;
    case 64: launch_n<64>(which, a, st); break;
    case 32: launch_n<32>(which, a, st); break;
    default: return 0;
  }
  return 1;
}

int slab_schur_apply(const SlabCg& a, cudaStream_t st) {
  switch (a.N) {
    case 128: schur_n<128>(a, st); break;
    case 64: schur_n<64>(a, st); break;
    case 32: schur_n<32>(a, st); break;
    default: return 0;
  }
  return 3;
}

}  // namespace kfbim
