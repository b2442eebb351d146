// Sparse and pointwise kernels of the KFBI matvec: jump evaluation (Sec. 4.3
// jump conditions), right-hand-side corrections (Sec. 4.3 items 1-4), MAC
// stencils and residual (Sec. 4.2), trace interpolation (Sec. 4.4) and the
// reductions used by CG and GMRES.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_common.cuh"
#include "fastcvt.h"

namespace kfbim {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 1216;  // 8 x 152 SMs

// Index arithmetic of the N^3 grid fields, flat index x = (k N + j) N + i:
// shifts when N is a power of two (lg = log2 N), divisions otherwise (lg < 0,
// N = 96).
struct GridIx {
  int N, lg;
  __device__ __forceinline__ int64_t n3() const { return (int64_t)N * N * N; }
  // element stride along axis b
  __device__ __forceinline__ int64_t stride(int b) const {
    return b == 0 ? 1 : (b == 1 ? (int64_t)N : (int64_t)N * N);
  }
  // field f of a flat index e over consecutive N^3 fields, and e's index x in it
  __device__ __forceinline__ int field(int64_t e, int64_t& x) const {
    const int f = lg >= 0 ? (int)(e >> (3 * lg)) : (int)(e / n3());
    x = e - (int64_t)f * n3();
    return f;
  }
  __device__ __forceinline__ void unflat(int64_t x, int& i, int& j, int& k) const {
    if (lg >= 0) {
      const int m = N - 1;
      i = (int)(x & m);
      j = (int)((x >> lg) & m);
      k = (int)(x >> (2 * lg));
    } else {
      const int64_t q = x / N;
      i = (int)(x - q * N);
      k = (int)(q / N);
      j = (int)(q - (int64_t)k * N);
    }
  }
};

// ------------------------------------------------------------------ jumps
// Jump values at every control point (Sec. 4.3).  One thread per fit row
// (point y, component c'): the fitted value and surface derivatives
// (d_1, d_2, d_11, d_12, d_22) of phi^(c') as a sequential sum over the row's
// neighbours; then, per block of JB points, the 11 x 18 jump map from shared
// memory (one output slot per task, input-major map rows).  All arithmetic is
// FP64.  J is slot-major: J[s * n + y].
// The fit rows are interleaved by groups of 32 (a warp's rows): entry i of
// row r at fit_off[r / 32] + 32 i + r % 32, weight k at fit_w[k ne + that],
// rows padded to their group's longest with zero weights (column 0), so a
// warp reads one entry of each of its rows with one coalesced load per array
// and every row's sum is the one of its CSR order (the padding adds zeros).
constexpr int JB = 32;                 // points per block (3 JB threads)
__global__ void __launch_bounds__(3 * JB)
k_jumps(const double* __restrict__ phi, const double* __restrict__ fpts, int64_t n,
        const int32_t* __restrict__ comp, const int32_t* __restrict__ pid,
        const int64_t* __restrict__ fit_off, const int32_t* __restrict__ fit_col,
        const double* __restrict__ fit_w, int64_t ne, const double* __restrict__ jmap,
        double* __restrict__ J) {
  __shared__ double D[JB * 3][6];
  const int64_t y0 = (int64_t)blockIdx.x * JB;
  {
    const int t = threadIdx.x;                  // row 3 * (y - y0) + c'
    const int64_t y = y0 + t / 3;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    if (y < n) {
      const int64_t rr = 3 * y0 + t;
      const int64_t b = fit_off[rr >> 5], e = fit_off[(rr >> 5) + 1];
      for (int64_t q = b + (rr & 31); q < e; q += 32) {
        const double v = phi[fit_col[q]];
#pragma unroll
        for (int k = 0; k < 6; ++k) acc[k] += fit_w[k * ne + q] * v;
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) D[t][k] = acc[k];
  }
  __syncthreads();
  // slot 0: the density itself at a primary point, its fitted value at a secondary one
  if (threadIdx.x < JB) {
    const int64_t y = y0 + threadIdx.x;
    if (y < n) {
      const int64_t p = pid[y];
      J[y] = (p >= 0) ? phi[p] : D[3 * threadIdx.x + comp[y] - 1][0];
    }
  }
  // slots 1..11: the jump map (input-major jmap[(y * 18 + q) * 11 + r])
  for (int task = threadIdx.x; task < JB * 11; task += 3 * JB) {
    const int yl = task / 11, r = task - yl * 11;
    const int64_t y = y0 + yl;
    if (y >= n) continue;
    const double* M = jmap + (size_t)y * 18 * 11 + r;
    double s = 0.0;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
      for (int k = 0; k < 5; ++k) s += M[(5 * cc + k) * 11] * D[3 * yl + cc][k + 1];
    if (fpts) {
#pragma unroll
      for (int cc = 0; cc < 3; ++cc) s += M[(15 + cc) * 11] * fpts[cc * n + y];
    }
    J[(int64_t)(r + 1) * n + y] = s;
  }
}

// ------------------------------------------------------------ RHS assembly
// f~ on the face grids (f in Omega, 0 outside and on wall faces) and g = 0:
// the extended source of the volume integral (Prop. FBI, Alg. 1 step 2).
__global__ void k_rhs_fill(const double* __restrict__ fgrid, const uint8_t* __restrict__ side1,
                           const uint8_t* __restrict__ side2, const uint8_t* __restrict__ side3,
                           GridIx gx, double* __restrict__ rhs) {
  const int64_t N3 = gx.n3();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 4 * N3;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t x;
    const int f = gx.field(e, x);
    double v = 0.0;
    if (f < 3 && fgrid) {
      const uint8_t* side = f == 0 ? side1 : (f == 1 ? side2 : side3);
      int i, j, k;
      gx.unflat(x, i, j, k);
      const int nrm = f == 0 ? i : (f == 1 ? j : k);
      if (side[x] && nrm > 0) v = fgrid[e];
    }
    rhs[e] = v;
  }
}

// Correction rows (Sec. 4.3 items 1-4): rhs[row] += sum coef * J[src] (CSR
// keyed by target, no atomics).
__global__ void k_corrections(const int64_t* __restrict__ row, const int64_t* __restrict__ ptr,
                              const int64_t* __restrict__ src, const double* __restrict__ coef,
                              int64_t nrows, const double* __restrict__ J, double* __restrict__ rhs) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) s += coef[e] * J[src[e]];
    rhs[row[r]] += s;
  }
}

// ------------------------------------------------------------------ trace
// u^+ at the primary points (Sec. 4.4, Eqs. Interpolation+/-): ten-node
// quadratic interpolation with the jump Taylor terms of the Omega^c nodes.
__global__ void k_trace(const double* __restrict__ u, const double* __restrict__ J, int64_t n_all,
                        int64_t n_prim, const int64_t* __restrict__ prim_of, int N,
                        const int32_t* __restrict__ tcomp, const int32_t* __restrict__ tnode,
                        const double* __restrict__ tw, const double* __restrict__ tcj,
                        double* __restrict__ out) {
  const int64_t N3 = (int64_t)N * N * N;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_prim;
       q += (int64_t)gridDim.x * blockDim.x) {
    const double* uc = u + (int64_t)(tcomp[q] - 1) * N3;
    const int64_t y = prim_of[q];
    double s = 0.0;
#pragma unroll
    for (int i = 0; i < 10; ++i) s += tw[10 * q + i] * uc[tnode[10 * q + i]];
#pragma unroll
    for (int k = 0; k < 10; ++k) s += tcj[10 * q + k] * J[(int64_t)k * n_all + y];
    out[q] = s;
  }
}

// p^+ at every control point (Sec. 4.4, last paragraph: a linear rule is
// enough for the pressure): trilinear interpolation over the eight cell
// centres around the point; a cell in Omega^c contributes p + [p] (slot 10 of
// J at the point), its Omega-side value to zeroth order.
__global__ void k_pressure_trace(const double* __restrict__ p, const double* __restrict__ J,
                                 const double* __restrict__ xyz, int64_t n, int N, double lo, double h,
                                 const uint8_t* __restrict__ side0, double* __restrict__ out) {
  for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < n;
       y += (int64_t)gridDim.x * blockDim.x) {
    int i0[3];
    double t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double sc = (xyz[3 * y + a] - lo) / h - 0.5;
      int f = (int)floor(sc);
      f = f < 0 ? 0 : (f > N - 2 ? N - 2 : f);
      i0[a] = f;
      t[a] = sc - f;
    }
    const double jp = J[10 * n + y];
    double acc = 0.0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int di = c & 1, dj = (c >> 1) & 1, dk = c >> 2;
      const int64_t idx = ((int64_t)(i0[2] + dk) * N + (i0[1] + dj)) * N + (i0[0] + di);
      const double w = (di ? t[0] : 1.0 - t[0]) * (dj ? t[1] : 1.0 - t[1]) * (dk ? t[2] : 1.0 - t[2]);
      acc += w * (p[idx] + (side0[idx] ? 0.0 : jp));
    }
    out[y] = acc;
  }
}

// --------------------------------------------------------- MAC stencils

// r^(c) = f^(c) - G_c p   (face grid c; wall faces 0)
template <typename Tp, typename Tout>
__global__ void k_f_minus_gp(const double* __restrict__ f, const Tp* __restrict__ p, GridIx gx, double h,
                             Tout* __restrict__ r) {
  const int64_t N3 = gx.n3();
  const double ih = 1.0 / h;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 3 * N3;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t x;
    const int c = gx.field(e, x);
    int id[3];
    gx.unflat(x, id[0], id[1], id[2]);
    const int nrm = c == 0 ? id[0] : (c == 1 ? id[1] : id[2]);
    if constexpr (sizeof(Tout) == 4 && sizeof(Tp) == 4) {
      // FP32 result (the MIXED correction): FP32 arithmetic, f rounded by
      // integer operations (no FP64 instruction per element)
      float v = 0.f;
      if (nrm > 0) {
        const int64_t st = gx.stride(c);
        v = f64_to_f32(f[e]) - (float(p[x]) - float(p[x - st])) * float(ih);
      }
      r[e] = Tout(v);
    } else {
      double v = 0.0;
      if (nrm > 0) {
        const int64_t st = gx.stride(c);
        v = f[e] - (double(p[x]) - double(p[x - st])) * ih;
      }
      r[e] = Tout(v);
    }
  }
}

// FP64 residual of the corrected MAC system (Eq. MAC with the lambda_h
// projection): rf = f - (-mu Lap u + G p), rg = g - mean(g) - D u - c p
// (Stokes: c = 0; Navier: the mean is 0 and c = 1/(lambda + mu)).
__global__ void k_mac_residual(const double* __restrict__ f, const double* __restrict__ g,
                               const double* __restrict__ gmean, const double* __restrict__ u,
                               const double* __restrict__ p, GridIx gx, double h, double mu, double cpen,
                               double* __restrict__ rf, double* __restrict__ rg) {
  const int N = gx.N;
  const int64_t N3 = gx.n3();
  const double ih = 1.0 / h, c_lap = -mu / (h * h);
  const double gm = gmean[0];
  // FP64 throughput is the bound here (a small fraction of the FP32 rate on
  // this GPU): the six neighbours are summed first and scaled once
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 4 * N3;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t x;
    const int c = gx.field(e, x);
    int id[3];
    gx.unflat(x, id[0], id[1], id[2]);
    if (c < 3) {
      const int nrm = c == 0 ? id[0] : (c == 1 ? id[1] : id[2]);
      if (nrm == 0) { rf[e] = 0.0; continue; }
      const double* uc = u + (int64_t)c * N3;
      const double u0 = uc[x];
      double pair[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int64_t st = gx.stride(b);
        const int ib = b == 0 ? id[0] : (b == 1 ? id[1] : id[2]);
        double um, up;
        if (b == c) {
          um = (ib - 1 >= 1) ? uc[x - st] : 0.0;
          up = (ib + 1 <= N - 1) ? uc[x + st] : 0.0;
        } else {
          um = (ib > 0) ? uc[x - st] : -u0;
          up = (ib < N - 1) ? uc[x + st] : -u0;
        }
        pair[b] = up + um;
      }
      // nine FP64 operations per value: five adds for the neighbours, the
      // centre by one FMA, the pressure difference and two FMAs for
      // rf = f - dp / h - c_lap (sum - 6 u0)
      const double lap = fma(-6.0, u0, (pair[0] + pair[1]) + pair[2]);
      const double dp = p[x] - p[x - gx.stride(c)];
      rf[e] = fma(-c_lap, lap, fma(-ih, dp, f[e]));
    } else {
      double dif[3];
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const int64_t st = gx.stride(b);
        const int ib = b == 0 ? id[0] : (b == 1 ? id[1] : id[2]);
        const double* ub = u + (int64_t)b * N3;
        const double lo = (ib >= 1) ? ub[x] : 0.0;
        const double hi = (ib + 1 <= N - 1) ? ub[x + st] : 0.0;
        dif[b] = hi - lo;
      }
      rg[x] = fma(-ih, (dif[0] + dif[1]) + dif[2], fma(-cpen, p[x], g[x] - gm));
    }
  }
}

// ------------------------------------------------------------ reductions
// partial[blockIdx.x] = sum x*y (y == nullptr: sum x; x == y allowed)
template <typename Ta, typename Tb>
__global__ void k_dot_partial(const Ta* __restrict__ x, const Tb* __restrict__ y, int64_t n,
                              double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    s += y ? double(x[e]) * double(y[e]) : double(x[e]);
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// partial[b] = this block's compensated FP32 sum of x[e]^2 over a grid-stride
// range of FP64 values rounded to FP32 by integer operations: a norm for the
// refinement's stopping test (relative accuracy about 1e-7) without FP64
// instructions per element.  Finished by k_merge_partials.
__global__ void k_norm2_partial(const double* __restrict__ x, int64_t n, float2* __restrict__ partial) {
  __shared__ float2 sh[32];
  CgAcc<float> a[1];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float v = f64_to_f32(x[e]);
    a[0].add_prod(v, v);
  }
  block_merge<1>(a, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = make_float2(a[0].s, a[0].c);
}

// out = scale * the merged sum of nb compensated pairs (fixed order, one block)
__global__ void k_merge_partials(const float2* __restrict__ partial, int nb, double scale, double* __restrict__ out) {
  __shared__ float2 sh[32];
  CgAcc<float> a[1];
  for (int b = threadIdx.x; b < nb; b += blockDim.x) a[0].merge(partial[b].x, partial[b].y);
  block_merge<1>(a, sh);
  if (threadIdx.x == 0) out[0] = scale * a[0].value();
}

// out[j] = scale * sum_b partial[j * nb + b]  (fixed order, one block per j)
__global__ void k_sum_partials(const double* __restrict__ partial, int nb, double scale,
                               double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += partial[(int64_t)blockIdx.x * nb + b];
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = scale * s;
}

// ----------------------------------------------------------------- CG
// q_S = q + q2 + q3 + cdiag d (the three component terms and, for the
// Navier system, the c p block; summed in place into q);
// dq = d . q_S; alpha = rr / (dq + sumd^2 rank1)
template <typename T>
__global__ void k_cg_alpha(const T* __restrict__ d, T* __restrict__ q, const T* __restrict__ q2,
                           const T* __restrict__ q3, int64_t n, CGScalars* s,
                           double* __restrict__ partial) {
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  const T cd = T(s->cdiag);
  CgAcc<T> acc;   // a thread's few terms, compensated in FP32 (MIXED); FP64 from the block sum on
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T qs = q[e] + q2[e] + q3[e] + cd * d[e];
    q[e] = qs;
    acc.add_prod(d[e], qs);
  }
  if (last_block_sum(acc.value(), partial, &s->ticket[0], sh, &total) && threadIdx.x == 0) {
    const double den = total + s->sumd * s->sumd * s->rank1;
    s->dq = den;
    s->alpha = (den != 0.0) ? s->rr / den : 0.0;
  }
}

// x += alpha d; r -= alpha (q_S + sumd rank1); rr_new = r . r; beta; convergence flag
template <typename T>
__global__ void k_cg_update(T* __restrict__ x, T* __restrict__ r, const T* __restrict__ d,
                            const T* __restrict__ q, int64_t n, CGScalars* s,
                            double* __restrict__ partial) {
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  // element arithmetic in T (FP32 in MIXED); a thread's few squares summed
  // with compensation (CgAcc), the block and grid sums in FP64
  const T a = T(s->alpha);
  const T c1 = T(s->sumd * s->rank1);
  CgAcc<T> acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[e] - a * (q[e] + c1);
    x[e] = x[e] + a * d[e];
    r[e] = rv;
    acc.add_prod(rv, rv);
  }
  if (last_block_sum(acc.value(), partial, &s->ticket[1], sh, &total) && threadIdx.x == 0) {
    s->beta = (s->rr != 0.0) ? total / s->rr : 0.0;
    s->rr = total;
    s->iters += 1;
  }
}

// d = r + beta d; sumd = sum d; done once rr <= stop
template <typename T>
__global__ void k_cg_direction(T* __restrict__ d, const T* __restrict__ r, int64_t n, CGScalars* s,
                               double* __restrict__ partial) {
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  const T b = T(s->beta);
  CgAcc<T> acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = r[e] + b * d[e];
    d[e] = v;
    acc.add(v);
  }
  if (last_block_sum(acc.value(), partial, &s->ticket[2], sh, &total) && threadIdx.x == 0) {
    s->sumd = total;
    if (!(s->rr > s->stop)) s->done = 1;
  }
}

// The three CG kernels for a batch of independent CG runs in one launch each:
// blockIdx.y selects the run (its vectors, scalars and partial buffer), the
// blocks of one run reduce exactly as in the single-run kernels.
constexpr int kCgBatchMax = 64;
template <typename T>
struct CgBatchArgs {
  T *x[kCgBatchMax], *r[kCgBatchMax], *d[kCgBatchMax], *q[kCgBatchMax];
  const T *q2[kCgBatchMax], *q3[kCgBatchMax];
  CGScalars* s[kCgBatchMax];
  double* partial[kCgBatchMax];
};

template <typename T>
__global__ void k_cg_alpha_b(const __grid_constant__ CgBatchArgs<T> A, int64_t n) {
  const int b = blockIdx.y;
  CGScalars* s = A.s[b];
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  const T* d = A.d[b];
  T* q = A.q[b];
  const T *q2 = A.q2[b], *q3 = A.q3[b];
  const T cd = T(s->cdiag);
  CgAcc<T> acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T qs = q[e] + q2[e] + q3[e] + cd * d[e];
    q[e] = qs;
    acc.add_prod(d[e], qs);
  }
  if (last_block_sum(acc.value(), A.partial[b], &s->ticket[0], sh, &total) && threadIdx.x == 0) {
    const double den = total + s->sumd * s->sumd * s->rank1;
    s->dq = den;
    s->alpha = (den != 0.0) ? s->rr / den : 0.0;
  }
}

template <typename T>
__global__ void k_cg_update_b(const __grid_constant__ CgBatchArgs<T> A, int64_t n) {
  const int b = blockIdx.y;
  CGScalars* s = A.s[b];
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  T *x = A.x[b], *r = A.r[b];
  const T *d = A.d[b], *q = A.q[b];
  const T a = T(s->alpha);
  const T c1 = T(s->sumd * s->rank1);
  CgAcc<T> acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T rv = r[e] - a * (q[e] + c1);
    x[e] = x[e] + a * d[e];
    r[e] = rv;
    acc.add_prod(rv, rv);
  }
  if (last_block_sum(acc.value(), A.partial[b], &s->ticket[1], sh, &total) && threadIdx.x == 0) {
    s->beta = (s->rr != 0.0) ? total / s->rr : 0.0;
    s->rr = total;
    s->iters += 1;
  }
}

template <typename T>
__global__ void k_cg_direction_b(const __grid_constant__ CgBatchArgs<T> A, int64_t n) {
  const int b = blockIdx.y;
  CGScalars* s = A.s[b];
  __shared__ double sh[32];
  __shared__ double total;
  if (s->done) return;
  T* d = A.d[b];
  const T* r = A.r[b];
  const T be = T(s->beta);
  CgAcc<T> acc;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const T v = r[e] + be * d[e];
    d[e] = v;
    acc.add(v);
  }
  if (last_block_sum(acc.value(), A.partial[b], &s->ticket[2], sh, &total) && threadIdx.x == 0) {
    s->sumd = total;
    if (!(s->rr > s->stop)) s->done = 1;
  }
}

// initial scalars: rr = bb = b.b, sumd = sum b, stop = tol^2 bb
template <typename T>
__global__ void k_cg_init(const T* __restrict__ b, int64_t n, CGScalars* s, double tol2, double rank1,
                          double cdiag, double* __restrict__ partial) {
  double s0 = 0.0, s1 = 0.0;
  bool last;
  if constexpr (sizeof(T) == 4) {
    // FP32 right-hand side: compensated FP32 sums of b.b and sum b, merged
    // through the block and the grid without FP64 arithmetic
    __shared__ float2 shf[2 * 32];
    CgAcc<float> a[2];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      const float v = b[e];
      a[0].add_prod(v, v);
      a[1].add(v);
    }
    double out[2];
    last = last_block_merge<2>(a, reinterpret_cast<float2*>(partial), &s->ticket[0], shf, out);
    s0 = out[0];
    s1 = out[1];
  } else {
    __shared__ double sh[32];
    __shared__ bool is_last;
    double a0 = 0.0, a1 = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      const double v = double(b[e]);
      a0 += v * v;
      a1 += v;
    }
    a0 = block_sum<double>(a0, sh);
    a1 = block_sum<double>(a1, sh);
    if (threadIdx.x == 0) {
      partial[2 * blockIdx.x] = a0;
      partial[2 * blockIdx.x + 1] = a1;
      __threadfence();
      is_last = (atomicAdd(&s->ticket[0], 1u) == gridDim.x - 1);
    }
    __syncthreads();
    last = is_last;
    if (last) {
      __threadfence();
      for (int bk = threadIdx.x; bk < (int)gridDim.x; bk += blockDim.x) {
        s0 += ((volatile double*)partial)[2 * bk];
        s1 += ((volatile double*)partial)[2 * bk + 1];
      }
      s0 = block_sum<double>(s0, sh);
      s1 = block_sum<double>(s1, sh);
      if (threadIdx.x == 0) s->ticket[0] = 0u;
    }
  }
  if (last && threadIdx.x == 0) {
    s->rr = s0;
    s->bb = s0;
    s->sumd = s1;
    s->stop = tol2 * s0;
    s->rank1 = rank1;
    s->cdiag = cdiag;
    s->done = (s0 > s->stop) ? 0 : 1;
    s->iters = 0;
  }
}

// --------------------------------------------------------- vector helpers
// Streaming steps of the Schur solve (Sec. 4.2 items i-iii: right-hand side,
// velocity recovery, pressure gauge) and of the FP64 refinement.
// y += a x
__global__ void k_axpy(const double* __restrict__ x, double a, double* __restrict__ y, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] += a * x[e];
}

// out = b1 + b2 + b3
template <typename T>
__global__ void k_sum3(const T* __restrict__ b1, const T* __restrict__ b2, const T* __restrict__ b3,
                       T* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = b1[e] + b2[e] + b3[e];
}

// out = g + b1 + b2 + b3
template <typename Ta, typename Tb>
__global__ void k_sum4(const Ta* __restrict__ g, const Tb* __restrict__ b1, const Tb* __restrict__ b2,
                       const Tb* __restrict__ b3, Tb* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
  {
    if constexpr (sizeof(Ta) == 8 && sizeof(Tb) == 4)
      out[e] = f64_to_f32(g[e]) + b1[e] + b2[e] + b3[e];   // FP32 right-hand side, FP32 sums
    else
      out[e] = Tb(double(g[e]) + double(b1[e]) + double(b2[e]) + double(b3[e]));
  }
}

template <typename Ta, typename Tb>
__global__ void k_convert(const Ta* __restrict__ a, Tb* __restrict__ b, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    b[e] = Tb(a[e]);
}

template <typename Ta>
__global__ void k_add_to(const Ta* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
  {
    if constexpr (sizeof(Ta) == 4)
      b[e] += f32_to_f64(a[e]);   // exact widening by integer operations, one FP64 add
    else
      b[e] += double(a[e]);
  }
}

// b[e] = a[e] + shift[0] * sc   (pressure gauge)
__global__ void k_shift(double* __restrict__ b, const double* __restrict__ shift, double sc, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    b[e] += sc * shift[0];
}

// -------------------------------------------------------------- GMRES
// Classical Gram-Schmidt twice for the Arnoldi step of GMRES (Alg. 1 step 3).
// partial[j * nb + b] = sum_e V[j][e] w[e]
__global__ void k_multidot_partial(const double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                                   int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  const int j = blockIdx.y;
  const double* v = V + (int64_t)j * ld;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    s += v[e] * w[e];
  s = block_sum<double>(s, sh);
  if (threadIdx.x == 0) partial[(int64_t)j * gridDim.x + blockIdx.x] = s;
}

// w -= sum_j h[j] V[j]   (sign = -1)  or  w = sum_j h[j] V[j] (sign = 0)
__global__ void k_multi_axpy(const double* __restrict__ V, int64_t ld, const double* __restrict__ hcoef,
                             int k, double* __restrict__ w, int64_t n, int assign) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int j = 0; j < k; ++j) s += hcoef[j] * V[(int64_t)j * ld + e];
    w[e] = assign ? s : w[e] - s;
  }
}

__global__ void k_scale_copy(const double* __restrict__ a, double sc_host, const double* __restrict__ sc_dev,
                             double* __restrict__ b, int64_t n) {
  const double sc = sc_dev ? sc_host / sc_dev[0] : sc_host;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    b[e] = sc * a[e];
}

}  // namespace kfbim

namespace kfbim {

// ------------------------------------------------------------- adjoint
// Not in the paper (it solves forward problems only): the transpose of the
// matvec of Prop. DBI, for gradients with respect to the boundary data.
// Transposes of the linear maps phi -> J (jumps), J -> rhs (corrections) and
// (u, J) -> trace, each a gather over a transposed CSR built once on the
// host (fixed summation order, no atomics).

// rhs[0 : 3 N^3] = ubar with the wall faces (normal index 0) zeroed, rhs[3 N^3 :] = 0.
__global__ void k_adjoint_rhs(const double* __restrict__ ubar, GridIx gx, double* __restrict__ rhs) {
  const int64_t N3 = gx.n3();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < 4 * N3;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t x;
    const int f = gx.field(e, x);
    double v = 0.0;
    if (f < 3) {
      int i, j, k;
      gx.unflat(x, i, j, k);
      const int nrm = f == 0 ? i : (f == 1 ? j : k);
      if (nrm > 0) v = ubar[e];
    }
    rhs[e] = v;
  }
}

// ubar[key[r]] = sum_e w[e] lam[q[e]]: the trace rows transposed onto the
// face-grid nodes they read (ubar zeroed by the caller).
__global__ void k_trace_T_u(const int64_t* __restrict__ key, const int64_t* __restrict__ ptr,
                            const int32_t* __restrict__ q, const double* __restrict__ w, int64_t nkeys,
                            const double* __restrict__ lam, double* __restrict__ ubar) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nkeys;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) s += w[e] * lam[q[e]];
    ubar[key[r]] = s;
  }
}

// Jbar[k][y] = tcj[q][k] lam[q] for the primary point y of trace row q
// (each point has at most one trace row; Jbar zeroed by the caller).
__global__ void k_trace_T_J(const double* __restrict__ lam, int64_t n_all, int64_t n_prim,
                            const int64_t* __restrict__ prim_of, const double* __restrict__ tcj,
                            double* __restrict__ Jbar) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n_prim;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t y = prim_of[q];
#pragma unroll
    for (int k = 0; k < 10; ++k) Jbar[(int64_t)k * n_all + y] = tcj[10 * q + k] * lam[q];
  }
}

// Jbar[key[r]] += sum_e coef[e] rbar[row[e]]: the correction rows transposed
// (key = slot * n_all + point).
__global__ void k_corrections_T(const int64_t* __restrict__ key, const int64_t* __restrict__ ptr,
                                const int64_t* __restrict__ row, const double* __restrict__ coef,
                                int64_t nkeys, const double* __restrict__ rbar, double* __restrict__ Jbar) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nkeys;
       r += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = ptr[r]; e < ptr[r + 1]; ++e) s += coef[e] * rbar[row[e]];
    Jbar[key[r]] += s;
  }
}

// Per point y: the jump map transposed, Dbar[(3y + c')][s] (s = 0 value, 1..5
// the fitted derivatives d_1, d_2, d_11, d_12, d_22 of phi^(c')).  Slot 0 of a
// secondary point is its fitted value; of a primary point, phi itself (added
// in k_fit_T).
__global__ void k_jumps_T(const double* __restrict__ Jbar, int64_t n, const int32_t* __restrict__ comp,
                          const int32_t* __restrict__ pid, const double* __restrict__ jmap,
                          double* __restrict__ Dbar) {
  for (int64_t y = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; y < n;
       y += (int64_t)gridDim.x * blockDim.x) {
    double jb[11];
#pragma unroll
    for (int r = 0; r < 11; ++r) jb[r] = Jbar[(int64_t)(r + 1) * n + y];
    const double* M = jmap + (size_t)y * 18 * 11;
    const int c = comp[y] - 1;
    const double j0 = (pid[y] < 0) ? Jbar[y] : 0.0;
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
      double* D = Dbar + (size_t)(3 * y + cc) * 6;
      D[0] = (cc == c) ? j0 : 0.0;
#pragma unroll
      for (int s = 0; s < 5; ++s) {
        const double* m = M + (5 * cc + s) * 11;
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < 11; ++r) acc += m[r] * jb[r];
        D[s + 1] = acc;
      }
    }
  }
}

// phibar[col] = Jbar[0][point of col] + sum over the fit entries reading col
// of sum_s fit_w[s][q] Dbar[row][s]  (the surface fit transposed; q are the
// entries' positions in the interleaved fit layout of k_jumps).
__global__ void k_fit_T(const int64_t* __restrict__ ptr, const int32_t* __restrict__ q,
                        const int32_t* __restrict__ rr, const double* __restrict__ fit_w, int64_t fit_nnz,
                        const double* __restrict__ Dbar, const double* __restrict__ Jbar,
                        const int64_t* __restrict__ prim_of, int64_t n_prim, double* __restrict__ out) {
  for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < n_prim;
       col += (int64_t)gridDim.x * blockDim.x) {
    double s = Jbar[prim_of[col]];
    for (int64_t e = ptr[col]; e < ptr[col + 1]; ++e) {
      const int64_t qe = q[e];
      const double* D = Dbar + (size_t)rr[e] * 6;
#pragma unroll
      for (int k = 0; k < 6; ++k) s += fit_w[k * fit_nnz + qe] * D[k];
    }
    out[col] = s;
  }
}

}  // namespace kfbim
