// Launchers of the four-kernel FP32 Schur CG iteration (slab.cuh).
#include <cuda_runtime.h>

#include "slab.cuh"
#include "slab.h"

namespace kfbim {

bool slab_supported(int N) { return N == 32 || N == 64 || N == 128; }

namespace {

constexpr int kUpdBlocks = 1216;   // 8 x 152 SMs

template <int N>
cudaError_t prepare_n() {
  cudaError_t e = cudaFuncSetAttribute(slab::k_cg_xy<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)slab::XySmem<N>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(slab::k_cg_zfwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)slab::ZSmem<N>::bytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(slab::k_cg_zinv<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)slab::ZSmem<N>::bytes);
  return e;
}

// Kernel `which` of the iteration: 0 k_cg_zfwd, 1 k_cg_xy, 2 k_cg_zinv, 3 k_cg_upd.
template <int N>
void launch_n(int which, const SlabCg& a, cudaStream_t st) {
  using C = slab::Cfg<N>;
  const int zblocks = (N / C::TILE) * N;
  switch (which) {
    case 0:
      slab::k_cg_zfwd<N><<<zblocks, C::TILE_THREADS, slab::ZSmem<N>::bytes, st>>>(a.r, a.d, a.z1, a.z3, a.tw, a.qN,
                                                                                  a.s, a.partial);
      break;
    case 1:
      slab::k_cg_xy<N><<<N, C::PLANE_THREADS, slab::XySmem<N>::bytes, st>>>(a.z1, a.z3, a.tw, a.qN, a.s2,
                                                                            a.inv_mu, a.s);
      break;
    case 2:
      slab::k_cg_zinv<N><<<zblocks, C::TILE_THREADS, slab::ZSmem<N>::bytes, st>>>(a.z1, a.z3, a.d, a.q, a.tw,
                                                                                  a.qN, a.s, a.partial);
      break;
    default: {
      const int64_t n4 = (int64_t)N * N * N / 4;
      const int blocks = (int)((n4 + 255) / 256 < kUpdBlocks ? (n4 + 255) / 256 : kUpdBlocks);
      slab::k_cg_upd<<<blocks, 256, 0, st>>>(a.x, a.r, a.d, a.q, n4, a.s, a.partial);
    }
  }
}

template <int N>
void schur_n(const SlabCg& a, cudaStream_t st) {
  for (int k = 0; k < 3; ++k) launch_n<N>(k, a, st);
}

template <int N>
void iteration_n(const SlabCg& a, cudaStream_t st) {
  for (int k = 0; k < 4; ++k) launch_n<N>(k, a, st);
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
  return 4;
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
