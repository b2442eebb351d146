// FP32 Schur-complement CG iteration in three kernels (Sec. 4.2, Eq. linearS1
// and items i-iii), for N = 32, 64, 128.
//
// The Schur operator is applied in spectral form,
//   S d = (1/mu) sum_c B_c^-1 Lambda_c B_c d (+ rank-one / c d terms),
// B_c = DCT-II along axis c and DST-II along the other two axes, Lambda_c =
// sin^2(a_c) / sum_b sin^2(a_b).  The transforms along z come first: terms 1
// and 2 share DST-II along z, term 3 takes DCT-II along z.  After that every
// (x, y) plane of the two z-transformed fields is independent, so one CTA per
// plane does the rest of the three terms in shared memory:
//   W12 = T1 + T2 with T1 = (C_x S_y)^-1 L1 (C_x S_y) Z1, T2 = (S_x C_y)^-1 L2 (S_x C_y) Z1,
//   W3  = (S_x S_y)^-1 L3 (S_x S_y) Z3,
// the weights taking the plane's z mode.  The inverse z transforms of W12
// (DST-III) and W3 (DCT-III) are summed into q.
//
// The vector update of iteration k waits for alpha_k, which is known only
// once the reduction of d.q over the whole grid is done, so it is carried
// into the first kernel of iteration k + 1, which touches every element
// anyway; the next r.r (for beta and the stopping test) then comes from its
// expansion
//   |r - alpha q|^2 = r.r - 2 alpha r.q + alpha^2 q.q
// with r.r, r.q and q.q summed beside d.q over the stored vectors.  r.r is
// that of the stored r, never the previous expansion: the expansion carries
// an absolute error of the FP32 rounding times the r.r it started from, and
// carried on from one iteration to the next those errors would add up to
// about 1e-7 of the first r.r, far above a stopping level of 1e-11 of it.
// One CG iteration:
//   k_cg_zfwd  x += alpha d, r -= alpha q (pending update), d = r + beta d,
//              Z1 = S_z d, Z3 = C_z d, sum(d)          (4 reads, 5 writes)
//   k_cg_xy    W12, W3 in place of Z1, Z3              (2 reads, 2 writes)
//   k_cg_zinv  q = S_z^-1 W12 + C_z^-1 W3 + c d + rank-one; d.q, r.r, r.q,
//              q.q; alpha, the next r.r, beta          (4 reads, 1 write)
// i.e. 18 N^3 values moved per iteration, against 28 for the transform
// passes of Schur apply run one axis at a time plus 14 for the CG vectors;
// k_cg_fin applies the last pending update once the run stops.
//
// Transforms: the real DCT-II/DST-II (and inverses) of transforms.cuh via
// Makhoul's reordering, two real lines per complex FFT of length N (or the
// DCT-II and DST-II of one line together, since the DST-II input is the
// DCT-II input with its second half negated).  A team of M = N/16 threads
// computes one complex FFT: a radix-16 DFT in registers, a twiddle, an
// exchange through the shared memory of the team's own two lines and radix-M
// DFTs in registers.  Within a warp the teams only synchronise with
// __syncwarp.
//
// Shared-memory layouts avoid bank conflicts for the access patterns of the
// team FFT (stride 2 and runs of 8 along a line, 4 teams per warp):
//   plane: element x of row y at y N + (x ^ plane_sw(y)); the plane kernel
//   works along rows only and transposes the plane between its x and y passes,
//   z tile: element z of line l (32 lines) at 32 z + (l ^ tile_sw(z)),
//   exchange: in the z kernels the team's own two lines (real parts in one,
//   imaginary parts in the other, index c at position xpi(c)); in the plane
//   kernel a separate buffer per team (rows of M + 1, teams 8 banks apart),
//   which keeps its register use within the 128 of 512 threads.  The plane
//   kernel runs its twelve line operations through one copy of the FFT.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cg_common.cuh"
#include "transforms.cuh"
#include "transforms2.cuh"

namespace kfbim {
namespace slab {

template <int N>
struct Cfg {
  static constexpr int M = N / 16;                        // threads per complex FFT
  static constexpr int NS = 16 / M;                       // radix-M DFTs per thread
  static constexpr int PLANE_TEAMS = N / 2;               // xy kernel: one pair of lines per team
  static constexpr int PLANE_THREADS = PLANE_TEAMS * M;
  static constexpr int TILE = 32;                         // z kernels: lines per CTA
  static constexpr int TILE_THREADS = TILE * M;           // one line per team
};

template <int N>
struct XySmem {
  static constexpr size_t plane = sizeof(float) * N * N;
  // two planes (Z1 -> P and Q; Z3 -> P after them), the teams' exchange
  // buffers (real and imaginary arrays) and the tables
  static constexpr size_t xch = sizeof(float) * Cfg<N>::PLANE_TEAMS * ((16 * (Cfg<N>::M + 1) + 31) / 32 * 32 + 8);
  static constexpr size_t bytes = 2 * plane + 2 * xch + sizeof(C2<float>) * 3 * N + sizeof(float) * 2 * N;
};

template <int N>
struct ZSmem {
  static constexpr size_t tile = sizeof(float) * N * Cfg<N>::TILE;
  static constexpr size_t bytes = 2 * tile + sizeof(C2<float>) * 3 * N;
};

// Row swizzle of a plane: bits 0, 3 and 4 of the column index, from the row
// index mod 16, chosen so that the rows 8w + 2t (t = 0..3; likewise the odd
// rows) that the four teams of a warp work on map a stride-2 run and an
// aligned run of 8 columns to disjoint banks.  The plane kernel only ever
// works along rows (it transposes the plane between its x and y passes), so
// a row's swizzle is fixed and an access costs one XOR.
__device__ __forceinline__ int plane_sw(int y) {
  const int y0 = y & 1, y1 = (y >> 1) & 1, y2 = (y >> 2) & 1, y3 = (y >> 3) & 1;
  return (y0 ^ y1 ^ y3) | (y1 << 3) | (y2 << 4);
}

// Line swizzle of a z tile (32 lines): bits 2..4 of the line index, from
// z mod 16, bijective on even z, odd z, z < 8 and z >= 8 of each 16; the four
// teams of a warp take lines 4w + t (bits 0, 1).  Multiples of 4 keep
// 16-byte groups of lines together for vector copies.
__host__ __device__ __forceinline__ constexpr int tile_sw(int z) { return (((z >> 1) ^ ((z & 1) << 2)) & 7) << 2; }

// Position along the team's two lines of logical exchange index c (the
// team's lines double as its exchange buffer: real parts in line a,
// imaginary parts in line b).  Flipping bits 0..2 by bits 4..6 makes the
// exchange's three access patterns (8 consecutive indices; stride 16; the
// natural index of the FFT output) fall on distinct banks with the swizzles
// above.
__host__ __device__ __forceinline__ constexpr int xpi(int c) { return c ^ ((c >> 4) & 7); }

// Row y of a plane: element x at y N + (x ^ plane_sw(y)).
struct PlaneRow {
  float* p;
  int sw;
  __device__ __forceinline__ float& operator[](int x) const { return p[x ^ sw]; }
};
template <int N>
__device__ __forceinline__ PlaneRow plane_row(float* plane, int y) {
  return {plane + y * N, plane_sw(y)};
}
struct TileCol {
  float* p;
  int l;
  __device__ __forceinline__ float& operator[](int z) const { return p[z * 32 + (l ^ tile_sw(z))]; }
};

// The exchange buffer of a team's complex FFT, logical index c = s M + m in
// the first step and the natural index k of the FFT output Z[k] after it.
// XLines: the team's own two lines (in place; the post-processing reads all
// of Z before it writes the lines).  XBuf: a separate buffer of the team
// (separate real and imaginary arrays, rows of M + 1 floats).
template <class LA, class LB>
struct XLines {
  LA A;
  LB B;
  static constexpr bool in_place = true;
  static constexpr bool blocked = true;
  __device__ __forceinline__ float& re(int c) const { return A[xpi(c)]; }
  __device__ __forceinline__ float& im(int c) const { return B[xpi(c)]; }
};
template <class LA, class LB>
__device__ __forceinline__ XLines<LA, LB> xlines(const LA& A, const LB& B) {
  return {A, B};
}
template <int N>
struct XBuf {
  float* xr;
  float* xi;
  static constexpr bool in_place = false;
  static constexpr bool blocked = false;
  static constexpr int TS = (16 * (Cfg<N>::M + 1) + 31) / 32 * 32 + 8;   // team stride, 8 banks apart
  __device__ __forceinline__ float& re(int c) const { return xr[c + c / Cfg<N>::M]; }
  __device__ __forceinline__ float& im(int c) const { return xi[c + c / Cfg<N>::M]; }
};

// One complex FFT of length N by a team of M threads (lane m) through the
// exchange X.  On entry v[r] = z[m + M r], r = 0..15, the inputs already read
// from the lines; on return X holds Z[k] at logical index k, INV:
// exp(+2 pi i n k / N).  Four steps: Y[m][s] = DFT16_r z[m + M r], times
// w_N^{m s}, exchanged, then Z[s + 16 k] = DFT_M over m of the twiddled
// Y[m][s], lane m taking s = NS m + q.
template <int N, bool INV, class X>
__device__ __forceinline__ void team_fft(C2<float> (&v)[16], const X& x, const C2<float>* tw, int m) {
  using C = Cfg<N>;
  constexpr int M = C::M, NS = C::NS;
  dft_reg<16, INV, float>(v);
  __syncwarp();   // the team has read its inputs and the previous output
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    C2<float> y = v[s];
    if (s != 0) {
      C2<float> w = tw[2 * m * s];   // exp(-2 pi i m s / N) from the table over 2N
      if (INV) w.y = -w.y;
      y = cmul(y, w);
    }
    x.re(s * M + m) = y.x;
    x.im(s * M + m) = y.y;
  }
  __syncwarp();
  C2<float> w2[NS][M];
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int c = (X::blocked ? NS * m + q : q * M + m) * M + k;
      w2[q][k] = {x.re(c), x.im(c)};
    }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    dft_reg<M, INV, float>(w2[q]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int c = (X::blocked ? NS * m + q : q * M + m) + 16 * k;
      x.re(c) = w2[q][k].x;
      x.im(c) = w2[q][k].y;
    }
  }
  __syncwarp();
}

// team_fft for the separate exchange (X::blocked false) with the output left
// in registers: lane m returns Z[m + M j] in z[j], j = 0..15 (the radix-M
// step's results, k = q M + m + 16 k' with j = q + NS k').  zx_store writes
// them to the exchange at their natural index when a post-processing needs
// a general permutation of Z.
template <int N, bool INV, class X>
__device__ __forceinline__ void team_fft_reg(C2<float> (&v)[16], const X& x, const C2<float>* tw, int m,
                                             C2<float> (&z)[16]) {
  using C = Cfg<N>;
  constexpr int M = C::M, NS = C::NS;
  static_assert(!X::blocked, "register output needs the interleaved stage-two order");
  dft_reg<16, INV, float>(v);
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    C2<float> y = v[s];
    if (s != 0) {
      C2<float> w = tw[2 * m * s];
      if (INV) w.y = -w.y;
      y = cmul(y, w);
    }
    x.re(s * M + m) = y.x;
    x.im(s * M + m) = y.y;
  }
  __syncwarp();
  C2<float> w2[NS][M];
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int c = (q * M + m) * M + k;
      w2[q][k] = {x.re(c), x.im(c)};
    }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    dft_reg<M, INV, float>(w2[q]);
#pragma unroll
    for (int k = 0; k < M; ++k) z[q + NS * k] = w2[q][k];
  }
}

template <int N, class X>
__device__ __forceinline__ void zx_store(const X& x, const C2<float> (&z)[16], int m) {
  constexpr int M = Cfg<N>::M;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    x.re(m + M * j) = z[j].x;
    x.im(m + M * j) = z[j].y;
  }
  __syncwarp();
}

// Forward output from the FFT registers (team_fft_reg): Z[N - k] of mode
// k = m + M r lies with lane (M - m) mod M of the team, register 15 - r (or
// (16 - r) mod 16 for m = 0), and arrives by a shuffle; put(k, xa, xb) as
// post_fwd.
template <int N, class F>
__device__ __forceinline__ void post_fwd_reg(const C2<float> (&z)[16], const C2<float>* qN, int m, F&& put) {
  constexpr int M = Cfg<N>::M;
  const int lane = threadIdx.x & 31;
  const int partner = (lane & ~(M - 1)) | ((M - m) & (M - 1));
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    // what this lane sends: the value its partner needs, Z at register 15 - r
    // (partner m != 0) or (16 - r) mod 16 (m = 0, its own partner)
    const C2<float> snd = m ? z[15 - r] : z[(16 - r) & 15];
    const float zcx = __shfl_sync(0xffffffffu, snd.x, partner);
    const float zcy = __shfl_sync(0xffffffffu, snd.y, partner);
    const float zkx = z[r].x, zky = z[r].y;
    const float vax = 0.5f * (zkx + zcx), vay = 0.5f * (zky - zcy);
    const float vbx = 0.5f * (zky + zcy), vby = -0.5f * (zkx - zcx);
    const int k = m + M * r;
    const C2<float> q = qN[k];
    put(k, q.x * vax - q.y * vay, q.x * vbx - q.y * vby);
  }
}

// Forward input of a pair of lines (DCT-II or DST-II each; DST-II negates the
// second half of Makhoul's reordering v_n = x_{2n}, v_{N-1-n} = x_{2n+1}).
template <int N, class LA, class LB>
__device__ __forceinline__ void pre_fwd_pair(C2<float> (&v)[16], const LA& A, const LB& B, bool dsta, bool dstb,
                                             int m) {
  constexpr int M = Cfg<N>::M;
  __syncwarp();   // the team's earlier writes to the lines are visible
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int n = m + M * r;
    const bool hi = r >= 8;   // n >= N / 2
    const int i = hi ? 2 * (N - 1 - n) + 1 : 2 * n;
    float a = A[i], b = B[i];
    if (hi && dsta) a = -a;
    if (hi && dstb) b = -b;
    v[r] = {a, b};
  }
}

// Forward input of one line whose DCT-II (real part) and DST-II (imaginary
// part) are wanted together.
template <int N, class L>
__device__ __forceinline__ void pre_fwd_cs(C2<float> (&v)[16], const L& A, int m) {
  constexpr int M = Cfg<N>::M;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int n = m + M * r;
    const bool hi = r >= 8;
    const float a = A[hi ? 2 * (N - 1 - n) + 1 : 2 * n];
    v[r] = {a, hi ? -a : a};
  }
}

// Forward output: for k = m + M r the transforms of both packed lines at
// mode k, X_k = Re(exp(-i pi k / 2N) V_k) (a DCT-II line puts it at position
// k, a DST-II line at N - 1 - k), handed to put(k, xa, xb).  In place, every
// value is computed before any put, once the whole team has read Z.
template <int N, class X, class F>
__device__ __forceinline__ void post_fwd(const X& x, const C2<float>* qN, int m, F&& put) {
  constexpr int M = Cfg<N>::M;
  auto value = [&](int k, float& va, float& vb) {
    const int kc = (N - k) & (N - 1);
    const float zkx = x.re(k), zky = x.im(k), zcx = x.re(kc), zcy = x.im(kc);
    const float vax = 0.5f * (zkx + zcx), vay = 0.5f * (zky - zcy);
    const float vbx = 0.5f * (zky + zcy), vby = -0.5f * (zkx - zcx);
    const C2<float> q = qN[k];
    va = q.x * vax - q.y * vay;
    vb = q.x * vbx - q.y * vby;
  };
  if constexpr (X::in_place) {
    float oa[16], ob[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) value(m + M * r, oa[r], ob[r]);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) put(m + M * r, oa[r], ob[r]);
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      float va, vb;
      value(m + M * r, va, vb);
      put(m + M * r, va, vb);
    }
  }
}

// Inverse input of a pair of lines (DCT-III when dst = false, DST-III when
// true): V_k = conj(q_k) (x_k - i x_{N-k}) with the DST-III line read backwards.
template <int N, class LA, class LB>
__device__ __forceinline__ void pre_inv_pair(C2<float> (&v)[16], const LA& A, const LB& B, bool dsta, bool dstb,
                                             const C2<float>* qN, int m) {
  constexpr int M = Cfg<N>::M;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int k = m + M * r;
    const bool k0 = (k == 0);
    const float xa = dsta ? A[N - 1 - k] : A[k];
    const float xna = k0 ? 0.f : (dsta ? A[k - 1] : A[N - k]);
    const float xb = dstb ? B[N - 1 - k] : B[k];
    const float xnb = k0 ? 0.f : (dstb ? B[k - 1] : B[N - k]);
    const C2<float> q = qN[k];
    const float vax = q.x * xa - q.y * xna, vay = -q.x * xna - q.y * xa;
    const float vbx = q.x * xb - q.y * xnb, vby = -q.x * xnb - q.y * xb;
    v[r] = {vax - vby, vay + vbx};
  }
}

// Inverse output: x_{2n} = v_n, x_{2n+1} = v_{N-1-n} (1/N; DST-III negates the
// odd outputs); for o = m + M r, put(o, xa, xb), in place after the whole
// team has read Z.
template <int N, class X, class F>
__device__ __forceinline__ void post_inv(const X& x, bool dsta, bool dstb, int m, F&& put) {
  constexpr int M = Cfg<N>::M;
  constexpr float invN = 1.0f / N;
  auto value = [&](int o, float& va, float& vb) {
    const bool odd = (o & 1) != 0;
    const int c = odd ? N - 1 - (o >> 1) : (o >> 1);
    va = x.re(c) * ((dsta && odd) ? -invN : invN);
    vb = x.im(c) * ((dstb && odd) ? -invN : invN);
  };
  if constexpr (X::in_place) {
    float oa[16], ob[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) value(m + M * r, oa[r], ob[r]);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) put(m + M * r, oa[r], ob[r]);
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      float va, vb;
      value(m + M * r, va, vb);
      put(m + M * r, va, vb);
    }
  }
}

// Inverse output with run-time kinds and scales: x_{2n} = v_n, x_{2n+1} =
// v_{N-1-n} times sa (line a) and sb (line b), a DST-III line negating its
// odd outputs; put(o, xa, xb) for o = m + M r.  The exchange X is a separate
// buffer (written by the team's FFT only).
template <int N, class X, class F>
__device__ __forceinline__ void post_inv_rt(const X& x, int ka, int kb, float sa, float sb, int m, F&& put) {
  constexpr int M = Cfg<N>::M;
  static_assert(!X::in_place, "run-time kinds with a separate exchange only");
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int o = m + M * r;
    const bool odd = (o & 1) != 0;
    const int c = odd ? N - 1 - (o >> 1) : (o >> 1);
    put(o, x.re(c) * ((ka && odd) ? -sa : sa), x.im(c) * ((kb && odd) ? -sb : sb));
  }
}

// sin^2 weights (Lambda_c / mu) of the Schur terms at modes (ax, ay, az):
// s2[a] = 4 sin^2(pi a / 2N) for the DCT modes, s2[N + a] = 4 sin^2(pi (a+1) / 2N)
// for the DST modes; the numerator is the DCT axis's.
__device__ __forceinline__ float schur_w(float num, float sum, float inv_mu) {
  return __fdividef(num, sum) * inv_mu;   // sum >= 4 sin^2(pi / 2N) > 0, far from the fast path's limits
}

template <int N>
__device__ __forceinline__ void load_tables(C2<float>* tw, C2<float>* qN, float* s2, const C2<float>* __restrict__ twg,
                                            const C2<float>* __restrict__ qg, const float* __restrict__ s2g,
                                            int threads) {
  for (int e = threadIdx.x; e < 3 * N; e += threads) {
    if (e < 2 * N) tw[e] = twg[e];
    else qN[e - 2 * N] = qg[e - 2 * N];
  }
  if (s2)
    for (int e = threadIdx.x; e < 2 * N; e += threads) s2[e] = s2g[e];
}

// Plane y-major, N^2 floats from global memory into the swizzled layout.
template <int N, int THREADS>
__device__ __forceinline__ void load_plane(float* P, const float* __restrict__ g) {
  constexpr int PER = N * N / THREADS;
  float t[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) t[j] = g[threadIdx.x + j * THREADS];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = threadIdx.x + j * THREADS;
    const int y = e / N, x = e % N;
    P[y * N + (x ^ plane_sw(y))] = t[j];
  }
}

// In-place transpose of a swizzled plane (every thread reads its share, then
// writes it to the mirrored position; barriers before and after).
template <int N, int THREADS>
__device__ __forceinline__ void transpose_plane(float* P) {
  constexpr int PER = N * N / THREADS;
  float t[PER];
  __syncthreads();
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = threadIdx.x + j * THREADS;
    const int y = e / N, x = e % N;
    t[j] = P[y * N + (x ^ plane_sw(y))];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e = threadIdx.x + j * THREADS;
    const int y = e / N, x = e % N;
    P[x * N + (y ^ plane_sw(x))] = t[j];
  }
  __syncthreads();
}

// ------------------------------------------------- z-tile lane addressing
// In a z tile, element z of line l sits at tl(z) ^ l with tl(z) = 32 z ^
// tile_sw(z), and exchange index c of the team's lines at tl(xpi(c)) ^ l.  Both
// maps are XOR-linear in the bits of their argument, so for the FFT's access
// patterns, an index of the form (lane part) + (constant part) with disjoint
// bits, the address is (the lane's precomputed part) ^ (a compile-time
// constant): one XOR per access instead of the swizzle arithmetic.
__host__ __device__ __forceinline__ constexpr int tl(int z) { return (z << 5) ^ tile_sw(z); }
__host__ __device__ __forceinline__ constexpr int tlx(int c) { return tl(xpi(c)); }

// One lane of a z-tile team: line l (the tile column), lane m < M.
template <int N>
struct ZLane {
  static constexpr int M = N / 16, NS = 16 / M;
  int m;
  int e_m, e_2m, e_mm1, e_nm;      // tl(m), tl(2m), tl of the k-1 and N-k lane parts, each ^ l
  int x_m, x_16m, x_nsm, x_mp, x_mh;   // tlx of m, 16 m, NS m, the partner -m mod M, m >> 1 (odd: ^ tlx(N-1))
  __device__ __forceinline__ ZLane(int m_, int l) : m(m_) {
    e_m = tl(m) ^ l;
    e_2m = tl(2 * m) ^ l;
    e_mm1 = tl(m ? m - 1 : M - 1) ^ l;   // k - 1 = (m - 1) + M r, or (M - 1) + M (r - 1) for m = 0
    e_nm = tl(m ? M - m : 0) ^ l;        // N - k = (M - m) + M (15 - r), or M (16 - r) for m = 0
    x_m = tlx(m) ^ l;
    x_16m = tlx(16 * m) ^ l;
    x_nsm = tlx(NS * m) ^ l;
    x_mp = tlx((M - m) & (M - 1)) ^ l;
    x_mh = tlx(m >> 1) ^ ((m & 1) ? tlx(N - 1) : 0) ^ l;
  }
};

// The team FFT of team_fft with the exchange in the z tile's lines D (real)
// and E (imaginary) at the lane's XOR addresses.
template <int N, bool INV>
__device__ __forceinline__ void zteam_fft(C2<float> (&v)[16], float* D, float* E, const ZLane<N>& L,
                                          const C2<float>* tw) {
  constexpr int M = ZLane<N>::M, NS = ZLane<N>::NS;
  const int m = L.m;
  dft_reg<16, INV, float>(v);
  __syncwarp();
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    C2<float> y = v[s];
    if (s != 0) {
      C2<float> w = tw[2 * m * s];
      if (INV) w.y = -w.y;
      y = cmul(y, w);
    }
    const int a = L.x_m ^ tlx(s * M);
    D[a] = y.x;
    E[a] = y.y;
  }
  __syncwarp();
  C2<float> w2[NS][M];
#pragma unroll
  for (int q = 0; q < NS; ++q)
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int a = L.x_16m ^ tlx(q * M + k);   // c = (NS m + q) M + k = 16 m + q M + k
      w2[q][k] = {D[a], E[a]};
    }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NS; ++q) {
    dft_reg<M, INV, float>(w2[q]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
      const int a = L.x_nsm ^ tlx(q + 16 * k);   // c = NS m + q + 16 k
      D[a] = w2[q][k].x;
      E[a] = w2[q][k].y;
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------ the kernels
// The buffers of up to MAXB independent CG runs on one grid (blockIdx.y
// selects the run): each run's blocks reduce exactly as a single run's, so a
// run's arithmetic does not depend on the batch it is part of.
template <int MAXB>
struct SlabArgs {
  float* x[MAXB];
  float* r[MAXB];
  float* d[MAXB];
  float* q[MAXB];
  float* z1[MAXB];
  float* z3[MAXB];
  CGScalars* s[MAXB];
  double* partial[MAXB];
};

// The pending update x += alpha d, r -= alpha q (alpha = 0 in the first
// iteration: nothing pending); d = r + beta d; Z1 = DST-II_z d, Z3 = DCT-II_z d;
// sumd = sum d.  CTA: 32 lines along z at x = x0 .. x0 + 31, y fixed (grid
// N/32 x N blocks per run).
template <int N, int MAXB>
__global__ void __launch_bounds__(Cfg<N>::TILE_THREADS, 4)
k_cg_zfwd(const __grid_constant__ SlabArgs<MAXB> args, const C2<float>* __restrict__ twg,
          const C2<float>* __restrict__ qg) {
  using C = Cfg<N>;
  constexpr int T = C::TILE_THREADS, M = C::M;
  constexpr int PER = N * 8 / T, HALF = PER / 2;   // float4 groups of the tile per thread (4)
  __shared__ float2 sh[32];
  const int b = blockIdx.y;
  CGScalars* s = args.s[b];
  if (s->done) return;
  float* __restrict__ x = args.x[b];
  float* __restrict__ r = args.r[b];
  float* __restrict__ d = args.d[b];
  const float* __restrict__ q = args.q[b];
  float* __restrict__ z1 = args.z1[b];
  float* __restrict__ z3 = args.z3[b];
  double* __restrict__ partial = args.partial[b];
  extern __shared__ __align__(16) unsigned char smz[];
  float* D = reinterpret_cast<float*>(smz);
  float* E = D + N * C::TILE;
  C2<float>* tw = reinterpret_cast<C2<float>*>(E + N * C::TILE);
  C2<float>* qN = tw + 2 * N;
  const int xb = blockIdx.x % (N / C::TILE), y = blockIdx.x / (N / C::TILE);
  const int x0 = xb * C::TILE;
  const double alpha = s->alpha;
  const bool pending = alpha != 0.0;
  const float a = float(alpha), beta = float(s->beta);
  CgAcc<float> acc[1];
#pragma unroll
  for (int h = 0; h < PER; h += HALF) {
    float4 rv[HALF], dv[HALF], xv[HALF], qv[HALF];
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const int e4 = threadIdx.x + (h + j) * T;
      const int64_t g = ((int64_t)(e4 >> 3) * N + y) * N + x0 + (e4 & 7) * 4;
      rv[j] = *reinterpret_cast<const float4*>(r + g);
      dv[j] = *reinterpret_cast<const float4*>(d + g);
      if (pending) {
        xv[j] = *reinterpret_cast<const float4*>(x + g);
        qv[j] = *reinterpret_cast<const float4*>(q + g);
      }
    }
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const int e4 = threadIdx.x + (h + j) * T;
      const int z = e4 >> 3, c4 = (e4 & 7) * 4;
      const int64_t g = ((int64_t)z * N + y) * N + x0 + c4;
      if (pending) {
        xv[j].x += a * dv[j].x;
        xv[j].y += a * dv[j].y;
        xv[j].z += a * dv[j].z;
        xv[j].w += a * dv[j].w;
        rv[j].x -= a * qv[j].x;
        rv[j].y -= a * qv[j].y;
        rv[j].z -= a * qv[j].z;
        rv[j].w -= a * qv[j].w;
        *reinterpret_cast<float4*>(x + g) = xv[j];
        *reinterpret_cast<float4*>(r + g) = rv[j];
      }
      float4 nv;
      nv.x = rv[j].x + beta * dv[j].x;
      nv.y = rv[j].y + beta * dv[j].y;
      nv.z = rv[j].z + beta * dv[j].z;
      nv.w = rv[j].w + beta * dv[j].w;
      *reinterpret_cast<float4*>(d + g) = nv;
      *reinterpret_cast<float4*>(D + z * 32 + (c4 ^ tile_sw(z))) = nv;
      acc[0].add(nv.x);
      acc[0].add(nv.y);
      acc[0].add(nv.z);
      acc[0].add(nv.w);
    }
  }
  // the tables are read from the FFT on: their loads queue behind the tile's
  load_tables<N>(tw, qN, nullptr, twg, qg, nullptr, T);
  __syncthreads();
  {
    // DCT-II and DST-II of line tm along z in one FFT (pre: Makhoul's order,
    // the second half negated for the DST; post: both transforms at mode k)
    const int tm = threadIdx.x / M, m = threadIdx.x % M;
    const ZLane<N> L(m, tm);
    C2<float> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const bool hi = r >= 8;   // n = m + M r >= N / 2: element 2(N-1-n)+1 = (2N-1) ^ 2n
      const float a = D[L.e_2m ^ (hi ? tl(2 * N - 1) ^ tl(2 * M * r) : tl(2 * M * r))];
      v[r] = {a, hi ? -a : a};
    }
    zteam_fft<N, false>(v, D, E, L, tw);
    float oc[16], os[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int k = m + M * r;
      const int ak = L.x_m ^ tlx(M * r);
      const int ac = L.x_mp ^ (m ? tlx(M * (15 - r)) : tlx(M * ((16 - r) & 15)));
      const float zkx = D[ak], zky = E[ak], zcx = D[ac], zcy = E[ac];
      const float vax = 0.5f * (zkx + zcx), vay = 0.5f * (zky - zcy);
      const float vbx = 0.5f * (zky + zcy), vby = -0.5f * (zkx - zcx);
      const C2<float> q = qN[k];
      oc[r] = q.x * vax - q.y * vay;
      os[r] = q.x * vbx - q.y * vby;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      E[L.e_m ^ tl(M * r)] = oc[r];                        // DCT-II mode k -> Z3
      D[L.e_m ^ tl(N - 1) ^ tl(M * r)] = os[r];            // DST-II at N-1-k -> Z1
    }
  }
  __syncthreads();
  for (int e4 = threadIdx.x; e4 < N * 8; e4 += T) {
    const int z = e4 >> 3, c4 = (e4 & 7) * 4;
    const int64_t g = ((int64_t)z * N + y) * N + x0 + c4;
    const int a = z * 32 + (c4 ^ tile_sw(z));
    *reinterpret_cast<float4*>(z1 + g) = *reinterpret_cast<const float4*>(D + a);
    *reinterpret_cast<float4*>(z3 + g) = *reinterpret_cast<const float4*>(E + a);
  }
  double sum[1];
  if (last_block_merge<1>(acc, reinterpret_cast<float2*>(partial), &s->ticket[2], sh, sum) && threadIdx.x == 0)
    s->sumd = sum[0];
}

// Makhoul input of a forward line pair with the kinds known only at run
// time (kind 1: DST-II, the second half negated; B may be A, for the DCT-II
// and DST-II of one line).
template <int N, class LA, class LB>
__device__ __forceinline__ void pre_fwd_rt(C2<float> (&v)[16], const LA& A, const LB& B, int ka, int kb, int m) {
  constexpr int M = Cfg<N>::M;
  __syncwarp();
  const float sa = ka ? -1.f : 1.f, sb = kb ? -1.f : 1.f;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int n = m + M * r;
    const bool hi = r >= 8;
    const int i = hi ? 2 * (N - 1 - n) + 1 : 2 * n;
    const float a = A[i], b = B[i];
    v[r] = {hi ? sa * a : a, hi ? sb * b : b};
  }
}

// Makhoul input of an inverse line pair (kind 0: DCT-III, 1: DST-III) at run
// time, conjugated: the forward FFT of conj(V) is the conjugate of the
// inverse FFT of V, so one FFT code serves both directions.
template <int N, class LA, class LB>
__device__ __forceinline__ void pre_inv_rt(C2<float> (&v)[16], const LA& A, const LB& B, int ka, int kb,
                                           const C2<float>* qN, int m) {
  constexpr int M = Cfg<N>::M;
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int k = m + M * r;
    const bool k0 = (k == 0);
    const float xa = A[ka ? N - 1 - k : k];
    const float xna = k0 ? 0.f : A[ka ? k - 1 : N - k];
    const float xb = B[kb ? N - 1 - k : k];
    const float xnb = k0 ? 0.f : B[kb ? k - 1 : N - k];
    const C2<float> q = qN[k];
    const float vax = q.x * xa - q.y * xna, vay = -q.x * xna - q.y * xa;
    const float vbx = q.x * xb - q.y * xnb, vby = -q.x * xnb - q.y * xb;
    v[r] = {vax - vby, -(vay + vbx)};
  }
}

// The twelve line operations of k_cg_xy, per team (two lines each), all
// along rows; the y passes work on the transposed plane (row = x mode):
//   0, 1   x forward of Z1: DCT-II (term 1, into P) and DST-II (term 2, into Q)
//          of rows 2t, 2t + 1                          [then P, Q transposed]
//   2, 3   y of term 1 on P: DST-II with its weight, DST-III (rows 2t, 2t + 1)
//   4, 5   y of term 2 on Q: DCT-II with its weight, DCT-III
//                                                  [then P, Q transposed back]
//   6, 7   x inverse: DCT-III of P plus DST-III of Q, rows 2t, 2t + 1 -> W12
//   (Z3 into P)
//   8      x forward of Z3: DST-II of rows 2t, 2t + 1     [then P transposed]
//   9, 10  y of term 3: DST-II with its weight, DST-III [then P transposed back]
//   11     x inverse: DST-III of rows 2t, 2t + 1 -> W3
// One loop runs them all through one copy of the FFT code (a fully unrolled
// kernel with a copy per operation does not fit the instruction cache).
constexpr int kXyOps = 12;

// The (x, y) part of the three Schur terms on plane kz = blockIdx.x of the
// z-transformed fields of run blockIdx.y, in place: Z1 -> W12 = T1 + T2,
// Z3 -> W3 = T3.
template <int N, int MAXB>
__global__ void __launch_bounds__(Cfg<N>::PLANE_THREADS, 1)
k_cg_xy(const __grid_constant__ SlabArgs<MAXB> args, const C2<float>* __restrict__ twg,
        const C2<float>* __restrict__ qg, const float* __restrict__ s2g, float inv_mu) {
  using C = Cfg<N>;
  constexpr int T = C::PLANE_THREADS, M = C::M, TS = XBuf<N>::TS;
  constexpr float invN = 1.0f / N;
  const int b = blockIdx.y;
  if (args.s[b]->done) return;
  float* __restrict__ z1 = args.z1[b];
  float* __restrict__ z3 = args.z3[b];
  extern __shared__ __align__(16) unsigned char smx[];
  float* P = reinterpret_cast<float*>(smx);
  float* Q = P + N * N;
  float* Xr = Q + N * N;
  float* Xi = Xr + C::PLANE_TEAMS * TS;
  C2<float>* tw = reinterpret_cast<C2<float>*>(Xi + C::PLANE_TEAMS * TS);
  C2<float>* qN = tw + 2 * N;
  float* s2 = reinterpret_cast<float*>(qN + N);
  const int kz = blockIdx.x;
  const int64_t off = (int64_t)kz * N * N;
  load_tables<N>(tw, qN, s2, twg, qg, s2g, T);
  const int tm = threadIdx.x / M, m = threadIdx.x % M;
  const XBuf<N> X{Xr + tm * TS, Xi + tm * TS};
  load_plane<N, T>(P, z1 + off);
  __syncthreads();   // tables and plane
  const int l0 = 2 * tm;   // this team's pair of rows
#pragma unroll 1
  for (int op = 0; op < kXyOps; ++op) {
    if (op == 8) {
      load_plane<N, T>(P, z3 + off);
      __syncthreads();
    }
    const bool inv = op == 3 || op == 5 || op == 6 || op == 7 || op == 10 || op == 11;
    const bool qplane = op == 4 || op == 5;
    const int row = (op == 1 || op == 7) ? l0 + 1 : l0;
    int ka = 1, kb = 1, term = 0;
    PlaneRow A, B, DB;
    if (op <= 1) {
      A = B = plane_row<N>(P, row);   // one row: DCT-II into P, DST-II into Q
      DB = plane_row<N>(Q, row);
      ka = 0;
    } else if (op == 6 || op == 7) {
      A = plane_row<N>(P, row);       // DCT-III of term 1 and DST-III of term 2
      B = plane_row<N>(Q, row);
      DB = B;
      ka = 0;
    } else {
      float* pl = qplane ? Q : P;
      A = plane_row<N>(pl, l0);
      B = plane_row<N>(pl, l0 + 1);
      DB = B;
      if (qplane) ka = kb = 0;
      term = op == 2 ? 1 : (op == 4 ? 2 : (op == 9 ? 3 : 0));
    }
    C2<float> v[16], zr[16];
    if (inv) pre_inv_rt<N>(v, A, B, ka, kb, qN, m);
    else pre_fwd_rt<N>(v, A, B, ka, kb, m);
    team_fft_reg<N, false>(v, X, tw, m, zr);
    if (!inv) {
      // weights of the y passes (row = x mode, position = y mode): sin^2 of
      // the DCT axis over the sum of the three axes' sin^2, over mu
      const float az = term == 3 ? s2[kz] : s2[N + kz];
      const float ax0 = s2[(term == 1 ? 0 : N) + l0], ax1 = s2[(term == 1 ? 0 : N) + l0 + 1];
      post_fwd_reg<N>(zr, qN, m, [&](int k, float va, float vb) {
        const int oa = ka ? N - 1 - k : k, ob = kb ? N - 1 - k : k;
        if (term) {
          const float ay = s2[(term == 2 ? 0 : N) + oa];
          const float n0 = term == 1 ? ax0 : (term == 2 ? ay : az);
          const float n1 = term == 1 ? ax1 : (term == 2 ? ay : az);
          va *= schur_w(n0, ax0 + ay + az, inv_mu);
          vb *= schur_w(n1, ax1 + ay + az, inv_mu);
        }
        A[oa] = va;
        DB[ob] = vb;
      });
    } else {
      float* outa = nullptr;
      float* outb = nullptr;
      if (op == 6 || op == 7) outa = z1 + off + (int64_t)row * N;
      if (op == 11) {
        outa = z3 + off + (int64_t)l0 * N;
        outb = outa + N;
      }
      zx_store<N>(X, zr, m);
      // 1/N, and the conjugation of the imaginary part
      post_inv_rt<N>(X, ka, kb, invN, -invN, m, [&](int o, float va, float vb) {
        if (op == 6 || op == 7) outa[o] = va + vb;
        else if (op == 11) {
          outa[o] = va;
          outb[o] = vb;
        } else {
          A[o] = va;
          B[o] = vb;
        }
      });
    }
    if (op == 1 || op == 5 || op == 8 || op == 10) {
      transpose_plane<N, T>(P);
      if (op == 1 || op == 5) transpose_plane<N, T>(Q);
    } else if (op == 7) {
      __syncthreads();
    }
  }
}

// q = DST-III_z W12 + DCT-III_z W3 + cdiag d + rank1 sumd; d.q, r.r, r.q,
// q.q; alpha, the next r.r and beta, done once that r.r <= stop.  Tiles as k_cg_zfwd.
template <int N, int MAXB>
__global__ void __launch_bounds__(Cfg<N>::TILE_THREADS, 4)
k_cg_zinv(const __grid_constant__ SlabArgs<MAXB> args, const C2<float>* __restrict__ twg,
          const C2<float>* __restrict__ qg) {
  using C = Cfg<N>;
  constexpr int T = C::TILE_THREADS, M = C::M;
  constexpr int PER = N * 8 / T;   // float4 groups of the tile per thread (4)
  __shared__ float2 sh[4 * 32];
  const int b = blockIdx.y;
  CGScalars* s = args.s[b];
  if (s->done) return;
  const float* __restrict__ w12 = args.z1[b];
  const float* __restrict__ w3 = args.z3[b];
  const float* __restrict__ d = args.d[b];
  float* __restrict__ q = args.q[b];
  double* __restrict__ partial = args.partial[b];
  extern __shared__ __align__(16) unsigned char smi[];
  float* D = reinterpret_cast<float*>(smi);
  float* E = D + N * C::TILE;
  C2<float>* tw = reinterpret_cast<C2<float>*>(E + N * C::TILE);
  C2<float>* qN = tw + 2 * N;
  const int xb = blockIdx.x % (N / C::TILE), y = blockIdx.x / (N / C::TILE);
  const int x0 = xb * C::TILE;
  {
    float4 av[PER], bv[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e4 = threadIdx.x + j * T;
      const int64_t g = ((int64_t)(e4 >> 3) * N + y) * N + x0 + (e4 & 7) * 4;
      av[j] = *reinterpret_cast<const float4*>(w12 + g);
      bv[j] = *reinterpret_cast<const float4*>(w3 + g);
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int e4 = threadIdx.x + j * T;
      const int z = e4 >> 3, c4 = (e4 & 7) * 4;
      const int a = z * 32 + (c4 ^ tile_sw(z));
      *reinterpret_cast<float4*>(D + a) = av[j];
      *reinterpret_cast<float4*>(E + a) = bv[j];
    }
  }
  load_tables<N>(tw, qN, nullptr, twg, qg, nullptr, T);   // read from the FFT on
  __syncthreads();
  {
    // DST-III of line tm of W12 (D) plus DCT-III of line tm of W3 (E) in one
    // inverse FFT: V_k = conj(q_k) (x_k - i x_{N-k}), the DST-III line read
    // backwards (x_k -> D[N-1-k], x_{N-k} -> D[k-1])
    const int tm = threadIdx.x / M, m = threadIdx.x % M;
    const ZLane<N> L(m, tm);
    C2<float> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int k = m + M * r;
      const bool k0 = (k == 0);
      const float xa = D[L.e_m ^ tl(N - 1) ^ tl(M * r)];
      const float xna = k0 ? 0.f : D[L.e_mm1 ^ (m ? tl(M * r) : (r ? tl(M * (r - 1)) : 0))];
      const float xb = E[L.e_m ^ tl(M * r)];
      const float xnb = k0 ? 0.f : E[L.e_nm ^ (m ? tl(M * (15 - r)) : tl(M * (16 - r)))];
      const C2<float> q = qN[k];
      const float vax = q.x * xa - q.y * xna, vay = -q.x * xna - q.y * xa;
      const float vbx = q.x * xb - q.y * xnb, vby = -q.x * xnb - q.y * xb;
      v[r] = {vax - vby, vay + vbx};
    }
    zteam_fft<N, true>(v, D, E, L, tw);
    // x_{2n} = v_n, x_{2n+1} = v_{N-1-n} over N; the DST-III line negates the odd outputs
    constexpr float invN = 1.0f / N;
    const float sa = (m & 1) ? -invN : invN;
    float oa[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const int a = L.x_mh ^ tlx((M / 2) * r);
      oa[r] = D[a] * sa + E[a] * invN;
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 16; ++r) D[L.e_m ^ tl(M * r)] = oa[r];
  }
  __syncthreads();
  // q = the three terms + c d + rank-one; d.q, r.r, r.q and q.q for alpha
  // and the expansion of the next r.r
  const float cd = float(s->cdiag), c1 = float(s->sumd * s->rank1);
  const float* __restrict__ r = args.r[b];
  float4 dv[PER], rv[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e4 = threadIdx.x + j * T;
    const int64_t g = ((int64_t)(e4 >> 3) * N + y) * N + x0 + (e4 & 7) * 4;
    dv[j] = *reinterpret_cast<const float4*>(d + g);
    rv[j] = *reinterpret_cast<const float4*>(r + g);
  }
  // d.q and r.r (alpha, the stopping test) exact to about 2^-48: every
  // product split by FMA, all sums compensated; r.q and q.q (only in the
  // expansion) sum the four products of a float4 by FMA first (within 3
  // roundings of their magnitudes) and those sums compensated
  CgAcc<float> acc[4];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int e4 = threadIdx.x + j * T;
    const int z = e4 >> 3, c4 = (e4 & 7) * 4;
    const int64_t g = ((int64_t)z * N + y) * N + x0 + c4;
    const float4 t = *reinterpret_cast<const float4*>(D + z * 32 + (c4 ^ tile_sw(z)));
    const float4 dw = dv[j], rw = rv[j];
    float4 qv;
    qv.x = t.x + cd * dw.x + c1;
    qv.y = t.y + cd * dw.y + c1;
    qv.z = t.z + cd * dw.z + c1;
    qv.w = t.w + cd * dw.w + c1;
    *reinterpret_cast<float4*>(q + g) = qv;
    acc[0].add_prod(dw.x, qv.x);
    acc[0].add_prod(dw.y, qv.y);
    acc[0].add_prod(dw.z, qv.z);
    acc[0].add_prod(dw.w, qv.w);
    acc[1].add_prod(rw.x, rw.x);
    acc[1].add_prod(rw.y, rw.y);
    acc[1].add_prod(rw.z, rw.z);
    acc[1].add_prod(rw.w, rw.w);
    acc[2].add(fmaf(rw.w, qv.w, fmaf(rw.z, qv.z, fmaf(rw.y, qv.y, rw.x * qv.x))));
    acc[3].add(fmaf(qv.w, qv.w, fmaf(qv.z, qv.z, fmaf(qv.y, qv.y, qv.x * qv.x))));
  }
  double sum[4];
  if (last_block_merge<4>(acc, reinterpret_cast<float2*>(partial), &s->ticket[0], sh, sum) &&
      threadIdx.x == 0) {
    const double dq = sum[0], rr = sum[1];
    const double al = (dq != 0.0) ? rr / dq : 0.0;
    const double rr1 = rr - 2.0 * al * sum[2] + al * al * sum[3];   // |r - alpha q|^2
    s->dq = dq;
    s->alpha = al;
    s->beta = (rr != 0.0) ? rr1 / rr : 0.0;
    s->rr = rr1;
    s->iters += 1;
    if (!(rr1 > s->stop)) s->done = 1;
  }
}

// The update still pending when a run stops: x += alpha d (float4 vectors,
// n4 = N^3 / 4; blockIdx.y = run).
constexpr int FIN_THREADS = 256;
template <int MAXB>
__global__ void __launch_bounds__(FIN_THREADS)
k_cg_fin(const __grid_constant__ SlabArgs<MAXB> args, int64_t n4) {
  const int b = blockIdx.y;
  const float a = float(args.s[b]->alpha);
  if (a == 0.f) return;
  float4* __restrict__ x4 = reinterpret_cast<float4*>(args.x[b]);
  const float4* __restrict__ d4 = reinterpret_cast<const float4*>(args.d[b]);
  for (int64_t e = (int64_t)blockIdx.x * FIN_THREADS + threadIdx.x; e < n4; e += (int64_t)gridDim.x * FIN_THREADS) {
    float4 xv = x4[e];
    const float4 dv = d4[e];
    xv.x += a * dv.x;
    xv.y += a * dv.y;
    xv.z += a * dv.z;
    xv.w += a * dv.w;
    x4[e] = xv;
  }
}

}  // namespace slab
}  // namespace kfbim
