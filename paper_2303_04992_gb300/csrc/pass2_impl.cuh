// Definition of pass2_launch (pass2.h), included by the per-grid-size
// translation units only.
#pragma once

#include "pass2.h"

namespace kfbim {

template <int N, typename Tin, typename T, typename Tout, int MAXJ>
cudaError_t pass2_launch(const PassJobs<Tin, Tout, MAXJ>& jobs, int njobs, const C2<T>* tw, const C2<T>* qN,
                         const T* s2, cudaStream_t s) {
  const size_t smem = Pass2Smem<T, N>::bytes;
  auto kern = k_axis_pass2<Tin, T, Tout, N, MAXJ>;
  const cudaError_t e = raise_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)(N * N / LPC2), (unsigned)njobs), PASS2_THREADS, smem, s>>>(jobs, tw, qN, s2);
  return cudaGetLastError();
}

}  // namespace kfbim

#define KFBIM_PASS2_INSTANTIATE_ONE(N, TIN, T, TOUT, MAXJ)                                                  \
  template cudaError_t kfbim::pass2_launch<N, TIN, T, TOUT, MAXJ>(                                          \
      const kfbim::PassJobs<TIN, TOUT, MAXJ>&, int, const kfbim::C2<T>*, const kfbim::C2<T>*, const T*, \
      cudaStream_t);
#define KFBIM_PASS2_INSTANTIATE(N)                                                   \
  KFBIM_PASS2_INSTANTIATE_ONE(N, double, double, double, 3)                          \
  KFBIM_PASS2_INSTANTIATE_ONE(N, double, double, double, kfbim::kPass2BatchJobs)     \
  KFBIM_PASS2_INSTANTIATE_ONE(N, double, float, float, 3)                            \
  KFBIM_PASS2_INSTANTIATE_ONE(N, double, float, float, kfbim::kPass2BatchJobs)       \
  KFBIM_PASS2_INSTANTIATE_ONE(N, float, float, float, 3)                             \
  KFBIM_PASS2_INSTANTIATE_ONE(N, float, float, float, kfbim::kPass2BatchJobs)
