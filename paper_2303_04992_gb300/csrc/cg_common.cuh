// Reductions and device scalars shared by the CG kernels of kernels.cuh and
// slab.cuh: block sums, the last-block grid reduction, the CG scalar block and
// the per-thread accumulators of the CG dot products (Sec. 4.2, Eq. linearS1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kfbim {

// Dot products of the Schur CG (Sec. 4.2) and of GMRES (Alg. 1 step 3).
template <typename Ta>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  v = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
  if (w == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __syncthreads();
  return v;
}

// Unpreconditioned CG on the Schur complement (Sec. 4.2, Eq. linearS1).
// Device scalars of one CG run on (S + 1 1^T rank1) x = b.  Every reduction
// is finished by the last block to arrive (fixed-order sum of the block
// partials), which also updates the scalars, so one CG iteration is the
// Schur apply plus three kernels and needs no host round trip.  Once
// rr <= stop the iteration is a no-op (done = 1): alpha = beta = 0 and the
// transform passes of S d return immediately.
struct CGScalars {
  double rr, bb, stop, dq, alpha, beta, sumd, rank1, cdiag;
  int done, iters;
  unsigned int ticket[3];
  int trips;   // iterations run by the device-side loop of a conditional graph
};

// Sum of the gridDim.x partials by the last block; returns true in that block.
__device__ __forceinline__ bool last_block_sum(double v, double* __restrict__ partial,
                                               unsigned int* ticket, double* sh, double* out) {
  __shared__ bool is_last;
  v = block_sum<double>(v, sh);
  if (threadIdx.x == 0) {
    partial[blockIdx.x] = v;
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s += ((volatile double*)partial)[b];
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) {
    *out = s;
    *ticket = 0u;
  }
  return true;
}

// Per-thread partial sums of the CG reductions.  FP64 vectors: plain FP64
// sums.  FP32 vectors (MIXED): compensated FP32 sums that carry the rounding
// error of every product and every addition, so the partial is exact to
// about 2^-48 relative, as good as an FP64 accumulation, without the FP64
// pipe (a small fraction of the FP32 rate on this GPU): each product a*b is
// split exactly into p + e by one FMA, each addition s + p into t + err by
// Knuth's TwoSum, and the errors are summed in a second FP32 word.  The
// intrinsics (_rn) keep the compiler from contracting the error-free steps
// into FMAs.  value() hands the pair to the FP64 block and grid sums.
template <typename T>
struct CgAcc;
template <>
struct CgAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { s += a * b; }
  __device__ __forceinline__ void add(double v) { s += v; }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct CgAcc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float p) {
    const float t = __fadd_rn(s, p);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    s = t;
    c = __fadd_rn(c, err);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    c = __fadd_rn(c, e);
  }
  // add another accumulator's pair (s2, c2): TwoSum of the leading words,
  // the error and the trailing words into c
  __device__ __forceinline__ void merge(float s2, float c2) {
    const float t = __fadd_rn(s, s2);
    const float bp = __fsub_rn(t, s);
    const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, err));
  }
  __device__ __forceinline__ double value() const { return double(s) + double(c); }
};

// Grid sums of K compensated FP32 accumulators without FP64 arithmetic
// (which runs at a small fraction of the FP32 rate on this GPU): warp
// butterflies and the block and grid steps merge (s, c) pairs; block b
// stores its K pairs at partial[K b + j]; the last block to finish merges
// them in block order.  Returns true in that block, whose thread 0 holds the
// K grid sums in out.  sh: K * 32 pairs of shared memory.
__device__ __forceinline__ void warp_merge(CgAcc<float>& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, a.s, o);
    const float c2 = __shfl_xor_sync(0xffffffffu, a.c, o);
    a.merge(s2, c2);
  }
}

template <int K>
__device__ __forceinline__ void block_merge(CgAcc<float> (&a)[K], float2* sh) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < K; ++j) warp_merge(a[j]);
  if (lane == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) sh[32 * j + w] = make_float2(a[j].s, a[j].c);
  }
  __syncthreads();
  if (w == 0) {
    const bool in = lane < (int)(blockDim.x >> 5);
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 p = in ? sh[32 * j + lane] : make_float2(0.f, 0.f);
      a[j].s = p.x;
      a[j].c = p.y;
      warp_merge(a[j]);
    }
  }
  __syncthreads();
}

template <int K>
__device__ __forceinline__ bool last_block_merge(CgAcc<float> (&a)[K], float2* __restrict__ partial,
                                                 unsigned int* ticket, float2* sh, double (&out)[K]) {
  __shared__ bool is_last;
  block_merge<K>(a, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) partial[K * blockIdx.x + j] = make_float2(a[j].s, a[j].c);
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  CgAcc<float> g[K];
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 p = __ldcg(partial + K * b + j);
      g[j].merge(p.x, p.y);
    }
  }
  block_merge<K>(g, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int j = 0; j < K; ++j) out[j] = g[j].value();
    *ticket = 0u;
  }
  return true;
}

}  // namespace kfbim
