// Transform pass as a dense GEMM on the 5th-generation tensor cores (tcgen05),
// N = 128, FP32 data: the "DST-GEMM" form of one axis pass of the FFT Poisson
// solver (Sec. 4.2 item ii) and of the spectral Schur operator.
//
// For a pass along `axis`, the field is a 128 x N^2 matrix X (rows: index n
// along the axis, columns: the N^2 lines), and the pass computes D = T X with T
// the 128 x 128 transform matrix (any of the six real transforms; the
// conventions are those of transforms.cuh), optionally followed by the
// pointwise spectral weight.  One tcgen05.mma (kind::tf32, M = 128, N = 64,
// K = 8) multiplies T (A operand, held in tensor memory for the whole kernel)
// by a 64-line tile of X (B operand, K-major, 128-byte swizzled shared memory).
// Precision: 3xTF32 -- T = T_hi + T_lo and X = X_hi + X_lo split into TF32
// parts, D = T_hi X_hi + T_hi X_lo + T_lo X_hi with FP32 accumulation in
// tensor memory, about FP32 accuracy.
//
// CTA: 256 threads, persistent over a contiguous range of tiles of the
// launch's (non-skipped) jobs, which all use the same transform.  Pipeline per
// tile: cp.async copies straight into the operand layout (a ring of three
// stages, two tiles ahead) -> in-place TF32 hi/lo split -> 48 MMAs issued by
// one thread into accumulator buffer it % 2 -> commit to mbarrier it % 2; the
// epilogue of the previous tile (tcgen05.ld, weight, coalesced store) and the
// copies of the tile after next overlap the MMAs.
// Every mbarrier wait is bounded (about one second of clock cycles); a
// timeout sets *err, the CTA stops waiting and issuing, and later launches
// return at once while *err is set (results are then invalid; the host
// reports the error).
#pragma once

#include "transforms2.cuh"

namespace kfbim {

constexpr int TC_N = 128;                          // transform length: GEMM M and K
constexpr int TC_COLS = 64;                        // lines per tile: GEMM N
constexpr int TC_THREADS = 256;
constexpr int TC_MAXJ = 48;
constexpr int TC_TILES_PER_JOB = TC_N * TC_N / TC_COLS;
constexpr int TC_B_BYTES = TC_COLS * TC_N * 4;     // one operand copy (hi or lo) of a tile
constexpr int TC_STAGES = 3;                       // cp.async ring depth
constexpr int TC_OUT_BYTES = TC_N * TC_COLS * 4;   // output staging
constexpr int TC_SMEM = 1024 + 2 * TC_STAGES * TC_B_BYTES + TC_OUT_BYTES + 256;
constexpr uint32_t TC_TMEM_COLS = 512;             // T_hi [0,128) T_lo [128,256) D0, D1 [256,384)
// tcgen05 instruction descriptor: D F32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_COLS >> 3) << 17) |
                              ((uint32_t)(TC_N >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, 128-byte swizzle, K-major: rows of 128 B,
// 8-row groups 1024 B apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(TC_IDESC), "r"(acc));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > 2000000000LL) return false;
  }
}

// 32 lanes x 32 consecutive columns of tensor memory -> 32 registers per thread.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 registers per thread -> 32 lanes x 32 consecutive columns of tensor memory.
__device__ __forceinline__ void tc_st32(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
      "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
      "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
      "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
      "r"(__float_as_uint(v[15])), "r"(__float_as_uint(v[16])), "r"(__float_as_uint(v[17])),
      "r"(__float_as_uint(v[18])), "r"(__float_as_uint(v[19])), "r"(__float_as_uint(v[20])),
      "r"(__float_as_uint(v[21])), "r"(__float_as_uint(v[22])), "r"(__float_as_uint(v[23])),
      "r"(__float_as_uint(v[24])), "r"(__float_as_uint(v[25])), "r"(__float_as_uint(v[26])),
      "r"(__float_as_uint(v[27])), "r"(__float_as_uint(v[28])), "r"(__float_as_uint(v[29])),
      "r"(__float_as_uint(v[30])), "r"(__float_as_uint(v[31]))
      : "memory");
}

// Global offset of column c (a line) of an N^3 field for a pass along axis,
// and the element stride along the axis.
__device__ __forceinline__ int64_t tc_col_offset(int axis, int c) {
  constexpr int64_t N = TC_N;
  return axis == 0 ? (int64_t)c * N : (axis == 1 ? (int64_t)(c / N) * N * N + (c % N) : (int64_t)c);
}

// Asynchronous copies (cp.async) of one tile into a stage, already in the
// K-major 128-byte-swizzled operand layout: element (line p, n) of K-block
// n/32 sits at block + p*128 + ((chunk ^ (p % 8)) * 16) + (n % 4) * 4, chunk =
// (n % 32) / 4.  x: 16-byte copies of 4 consecutive n, lanes along the chunks
// of a line; y, z: 4-byte copies, lanes along the lines (coalesced reads).
__device__ __forceinline__ void tc_issue_tile(const float* __restrict__ in, int axis, int colbase,
                                              uint32_t stage) {
  constexpr int64_t N = TC_N;
  if (axis == 0) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int t = threadIdx.x + TC_THREADS * r;
      const int p = t >> 5, ch = t & 31;
      const float* src = in + (int64_t)(colbase + p) * N + 4 * ch;
      const uint32_t dst = stage + (ch >> 3) * (TC_COLS * 128) + p * 128 + (((ch & 7) ^ (p & 7)) << 4);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
  } else {
    const int64_t estride = axis == 1 ? N : N * N;
    const int p = threadIdx.x & 63;
    const float* base = in + tc_col_offset(axis, colbase + p);
#pragma unroll 8
    for (int r = 0; r < 32; ++r) {
      const int n = (threadIdx.x >> 6) + 4 * r;
      const uint32_t dst = stage + (n >> 5) * (TC_COLS * 128) + p * 128 + ((((n & 31) >> 2) ^ (p & 7)) << 4) +
                           ((n & 3) << 2);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(base + n * estride) : "memory");
    }
  }
}

__device__ __forceinline__ void tc_commit_group() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Split a landed stage in place into its TF32 high part and, in the matching
// low stage, the remainder x - hi.
__device__ __forceinline__ void tc_split_stage(float* hi, float* lo) {
#pragma unroll
  for (int r = 0; r < TC_B_BYTES / 16 / TC_THREADS; ++r) {
    const int e = 4 * (threadIdx.x + TC_THREADS * r);
    float4 x = *reinterpret_cast<const float4*>(hi + e);
    float4 h, l;
    h.x = tf32_rna(x.x); l.x = x.x - h.x;
    h.y = tf32_rna(x.y); l.y = x.y - h.y;
    h.z = tf32_rna(x.z); l.z = x.z - h.z;
    h.w = tf32_rna(x.w); l.w = x.w - h.w;
    *reinterpret_cast<float4*>(hi + e) = h;
    *reinterpret_cast<float4*>(lo + e) = l;
  }
}

__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_pass(const __grid_constant__ PassJobs<float, float, TC_MAXJ> jobs, int njobs,
          const float* __restrict__ Tm, const float* __restrict__ s2, int* __restrict__ err) {
  extern __shared__ __align__(16) uint8_t tc_smem_raw[];
  const uint32_t raw = smem_u32(tc_smem_raw);
  uint8_t* smem = tc_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint8_t* hi_st = smem;                                     // TC_STAGES x B tile (hi)
  uint8_t* lo_st = smem + TC_STAGES * TC_B_BYTES;            // TC_STAGES x B tile (lo)
  float* ost = reinterpret_cast<float*>(smem + 2 * TC_STAGES * TC_B_BYTES);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * TC_STAGES * TC_B_BYTES + TC_OUT_BYTES);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 2);
  int* nact_s = reinterpret_cast<int*>(tmem_slot + 1);
  int* act = nact_s + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (*err) return;   // an earlier pass timed out: do nothing
  if (tid == 0) {
    int n = 0;
    for (int j = 0; j < njobs; ++j) {
      const int* sk = jobs.j[j].a.skip;
      if (!(sk && *sk)) act[n++] = j;
    }
    *nact_s = n;
  }
  __syncthreads();
  const int ntiles = *nact_s * TC_TILES_PER_JOB;
  const int t_begin = (int)((int64_t)blockIdx.x * ntiles / gridDim.x);
  const int t_end = (int)((int64_t)(blockIdx.x + 1) * ntiles / gridDim.x);
  if (t_begin >= t_end) return;
  auto job_of = [&](int t) -> const PassJob<float, float>& { return jobs.j[act[t / TC_TILES_PER_JOB]]; };
  auto issue = [&](int t) {
    const PassJob<float, float>& jb = job_of(t);
    const int it = t - t_begin;
    tc_issue_tile(jb.in, jb.a.axis, (t % TC_TILES_PER_JOB) * TC_COLS,
                  smem_u32(hi_st + (it % TC_STAGES) * TC_B_BYTES));
  };
  // the first two tiles are in flight while the CTA sets up
  issue(t_begin);
  tc_commit_group();
  if (t_begin + 1 < t_end) issue(t_begin + 1);
  tc_commit_group();

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;

  // T_hi (warps 0-3) and T_lo (warps 4-7) into tensor memory: lane m = row m
  {
    const int hl = warp >> 2;
    const int m = 32 * (warp & 3) + lane;
    const float* src = Tm + (size_t)hl * TC_N * TC_N + m;
#pragma unroll 1
    for (int n0 = 0; n0 < TC_N; n0 += 32) {
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = src[(size_t)(n0 + j) * TC_N];
      tc_st32(tmem + lane_base + (uint32_t)(hl * TC_N + n0), v);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }

  bool ok = true;
  auto wait_mma = [&](int it) {
    if (ok && !tc_wait(smem_u32(&mbar[it & 1]), (uint32_t)((it >> 1) & 1))) {
      ok = false;
      atomicExch(err, 1);
    }
    tc_fence_after();
  };

  auto epilogue = [&](int t, int dbuf) {
    const PassJob<float, float>& jb = job_of(t);
    const PassArgs& a = jb.a;
    const int axis = a.axis;
    const int colbase = (t % TC_TILES_PER_JOB) * TC_COLS;
    const int m = 32 * (warp & 3) + lane;      // output index along the axis
    const int p0 = 32 * (warp >> 2);            // first of this thread's 32 lines
    float v[32];
    tc_ld32(tmem + lane_base + (uint32_t)(2 * TC_N + TC_COLS * dbuf + p0), v);
    const float sc = (float)a.scale;
    if (a.wmode != W_NONE) {
      const float inv_mu = (float)(1.0 / a.mu);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int c = colbase + p0 + j;
        int i, jj, k;
        if (axis == 0) { i = m; jj = c % TC_N; k = c / TC_N; }
        else if (axis == 1) { i = c % TC_N; jj = m; k = c / TC_N; }
        else { i = c % TC_N; jj = c / TC_N; k = m; }
        v[j] *= spectral_weight2<float, TC_N>(a, s2, inv_mu, i, jj, k);
      }
    }
    float* __restrict__ out = jb.out;
    if (axis == 0) {
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        float* dst = out + (int64_t)(colbase + p0 + j) * TC_N + m;
        *dst = a.accumulate ? *dst + sc * v[j] : sc * v[j];
      }
    } else {
      // stage [m][64 lines] with 16-byte chunks swizzled by m % 8, then write rows
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int cj = (p0 >> 2) + q;
        *reinterpret_cast<float4*>(ost + m * TC_COLS + ((cj ^ (m & 7)) << 2)) =
            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      __syncthreads();
      const int64_t estride = axis == 1 ? TC_N : (int64_t)TC_N * TC_N;
      const int64_t cbase = tc_col_offset(axis, colbase);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int e = tid + TC_THREADS * r;
        const int mm = e >> 4, cj = e & 15;
        float4 w = *reinterpret_cast<const float4*>(ost + mm * TC_COLS + ((cj ^ (mm & 7)) << 2));
        float4* dst = reinterpret_cast<float4*>(out + cbase + mm * estride + 4 * cj);
        if (a.accumulate) {
          const float4 pr = *dst;
          w = make_float4(pr.x + sc * w.x, pr.y + sc * w.y, pr.z + sc * w.z, pr.w + sc * w.w);
        } else {
          w = make_float4(sc * w.x, sc * w.y, sc * w.z, sc * w.w);
        }
        *dst = w;
      }
    }
    tc_fence_before();
  };

#pragma unroll 1
  for (int t = t_begin; t < t_end; ++t) {
    const int it = t - t_begin;
    const int st = it % TC_STAGES;
    float* hi = reinterpret_cast<float*>(hi_st + st * TC_B_BYTES);
    float* lo = reinterpret_cast<float*>(lo_st + st * TC_B_BYTES);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncthreads();
    tc_split_stage(hi, lo);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && ok) {
      tc_fence_after();
      const uint32_t d = tmem + (uint32_t)(2 * TC_N + TC_COLS * (it & 1));
      const uint32_t bh = smem_u32(hi), bl = smem_u32(lo);
#pragma unroll 1
      for (int ks = 0; ks < TC_N / 8; ++ks) {
        const uint32_t koff = (uint32_t)((ks >> 2) * (TC_COLS * 128) + (ks & 3) * 32);
        const uint64_t dh = tc_desc_sw128(bh + koff), dl = tc_desc_sw128(bl + koff);
        const uint32_t ahi = tmem + (uint32_t)(8 * ks), alo = tmem + (uint32_t)(TC_N + 8 * ks);
        tc_mma(d, alo, dh, ks > 0);
        tc_mma(d, ahi, dl, 1);
        tc_mma(d, ahi, dh, 1);
      }
      tc_commit(smem_u32(&mbar[it & 1]));
    }
    // stage (it + 2) % 3 was read by the MMAs of tile it - 1: wait for them,
    // then refill it with tile it + 2 and run the epilogue of tile it - 1
    if (it >= 1) wait_mma(it - 1);
    if (t + 2 < t_end) issue(t + 2);
    tc_commit_group();
    if (it >= 1) epilogue(t - 1, (it - 1) & 1);
  }
  {
    const int it = t_end - 1 - t_begin;
    wait_mma(it);
    epilogue(t_end - 1, it & 1);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
  }
}

}  // namespace kfbim
