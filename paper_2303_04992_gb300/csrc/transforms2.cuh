// Transform pass with compile-time N: the same real transforms as
// transforms.cuh (DCT-II/III, DST-II/III via Makhoul's reordering, DST-I via
// the odd extension, two real lines per complex FFT), but each complex FFT of
// length L is a four-step FFT with a radix-16 DFT in registers, a twiddle, one
// shared-memory exchange and a radix-(L/16) DFT in registers:
//   z[m + M r] --DFT16 over r--> Y[m][s] * w_L^{m s} --DFT_M over m--> Z[s + 16 k],
//   M = L / 16 threads per line pair.
// Staging rows are padded (stride N + 1) so that column accesses of the
// strided axes are free of bank conflicts.  One CTA holds LPC2 = 32 lines
// (128 B coalesced rows for FP32 on the y and z axes).
#pragma once

#include <type_traits>

#include "fastcvt.h"
#include "transforms.cuh"

namespace kfbim {

constexpr int LPC2 = 32;
constexpr int PASS2_THREADS = 128;

template <int R>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}

// cos and sin of 2 pi j / 16 for j in 0..15 (exact octant symmetry)
__host__ __device__ constexpr double cos16(int j) {
  constexpr double c1 = 0.92387953251128675613, c2 = 0.70710678118654752440, c3 = 0.38268343236508977173;
  j &= 15;
  return j == 0 ? 1.0 : j == 1 ? c1 : j == 2 ? c2 : j == 3 ? c3 : j == 4 ? 0.0 : j == 5 ? -c3
       : j == 6 ? -c2 : j == 7 ? -c1 : j == 8 ? -1.0 : j == 9 ? -c1 : j == 10 ? -c2 : j == 11 ? -c3
       : j == 12 ? 0.0 : j == 13 ? c3 : j == 14 ? c2 : c1;
}
__host__ __device__ constexpr double sin16(int j) { return cos16(j - 4); }

// exp(-+ 2 pi i j / 16), sign + for the inverse transform (j a compile-time constant)
template <typename T, bool INV>
__device__ __forceinline__ C2<T> w16(int j) {
  return {T(cos16(j)), INV ? T(sin16(j)) : T(-sin16(j))};
}

// In-register DFT of R <= 16 points, natural order in and out (radix-2 DIT).
template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_reg(C2<T>* v) {
  if constexpr (R > 1) {
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int j = bitrev<R>(i);
      if (j > i) {
        const C2<T> t = v[i];
        v[i] = v[j];
        v[j] = t;
      }
    }
#pragma unroll
    for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
      for (int i = 0; i < R; i += len) {
#pragma unroll
        for (int k = 0; k < len / 2; ++k) {
          const C2<T> a = v[i + k];
          C2<T> b = v[i + k + len / 2];
          if (k != 0) b = cmul(b, w16<T, INV>(k * (16 / len)));
          v[i + k] = {a.x + b.x, a.y + b.y};
          v[i + k + len / 2] = {a.x - b.x, a.y - b.y};
        }
      }
    }
  }
}

// cos and sin of 2 pi j / 24 for j in 0..23 (multiples of 15 degrees)
__host__ __device__ constexpr double cos24(int j) {
  constexpr double c15 = 0.96592582628906828675, c30 = 0.86602540378443864676, c45 = 0.70710678118654752440,
                   c60 = 0.5, c75 = 0.25881904510252076235;
  j = ((j % 24) + 24) % 24;
  const int q = j % 12;   // cos(x + 180) = -cos x
  const double v = q == 0 ? 1.0 : q == 1 ? c15 : q == 2 ? c30 : q == 3 ? c45 : q == 4 ? c60 : q == 5 ? c75
                 : q == 6 ? 0.0 : q == 7 ? -c75 : q == 8 ? -c60 : q == 9 ? -c45 : q == 10 ? -c30 : -c15;
  return j < 12 ? v : -v;
}
__host__ __device__ constexpr double sin24(int j) { return cos24(j - 6); }

// In-register DFT of 24 points, natural order in and out: x[n], n = 8 n1 + n2,
// as X[k1 + 3 k2] = sum_n2 w_8^(n2 k2) [w_24^(n2 k1) sum_n1 x[8 n1 + n2] w_3^(n1 k1)]
// (three-point DFTs, the twiddle, then three eight-point DFTs).
template <bool INV, typename T>
__device__ __forceinline__ void dft24(C2<T>* v) {
  const T sg = INV ? T(1) : T(-1);
  const T h = T(0.86602540378443864676);   // sin 60 degrees
  C2<T> a[3][8];
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2) {
    const C2<T> x0 = v[n2], x1 = v[8 + n2], x2 = v[16 + n2];
    const C2<T> s = {x1.x + x2.x, x1.y + x2.y}, d = {x1.x - x2.x, x1.y - x2.y};
    a[0][n2] = {x0.x + s.x, x0.y + s.y};
    // x0 - s / 2 -+ i sin60 d  (the sign of the forward transform, exp(-2 pi i / 3))
    const C2<T> m = {x0.x - T(0.5) * s.x, x0.y - T(0.5) * s.y};
    a[1][n2] = {m.x - sg * h * d.y, m.y + sg * h * d.x};
    a[2][n2] = {m.x + sg * h * d.y, m.y - sg * h * d.x};
  }
#pragma unroll
  for (int k1 = 1; k1 < 3; ++k1)
#pragma unroll
    for (int n2 = 1; n2 < 8; ++n2) {
      const C2<T> w = {T(cos24(n2 * k1)), INV ? T(sin24(n2 * k1)) : T(-sin24(n2 * k1))};
      a[k1][n2] = cmul(a[k1][n2], w);
    }
#pragma unroll
  for (int k1 = 0; k1 < 3; ++k1) {
    dft_reg<8, INV, T>(a[k1]);
#pragma unroll
    for (int k2 = 0; k2 < 8; ++k2) v[k1 + 3 * k2] = a[k1][k2];
  }
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dft_any(C2<T>* v) {
  if constexpr (R == 24) dft24<INV, T>(v);
  else dft_reg<R, INV, T>(v);
}

template <int L>
struct Fft2Shape {
  // L = R M: a DFT of R points in each thread's registers, then R / M DFTs of
  // M points per thread.  R = 16 for the power-of-two lengths; R = 24 (3 x 8)
  // for the lengths 96 and 192 of the N = 96 grid, so that M (4 or 8) divides R.
  static constexpr int R = (L & (L - 1)) == 0 ? 16 : 24;
  static constexpr int M = L / R;                                    // threads per pair
  static constexpr int PPR_MAX = (PASS2_THREADS / M < LPC2 / 2) ? PASS2_THREADS / M : LPC2 / 2;
  // pairs per round: a power of two, so that the rounds cover the CTA's pairs
  static constexpr int PPR = PPR_MAX >= 16 ? 16 : (PPR_MAX >= 8 ? 8 : (PPR_MAX >= 4 ? 4 : (PPR_MAX >= 2 ? 2 : 1)));
  static constexpr int X = PPR * R * (M + 1);                        // exchange entries
  static constexpr int Z = PPR * (L + 1);                            // output entries (padded rows)
  static_assert(R % M == 0 || M == 2 * R, "four-step split");
};

template <typename T, int N>
struct Pass2Smem {
  static constexpr int RS = N + 1;                 // padded staging row
  using A = Fft2Shape<N>;
  using B = Fft2Shape<2 * N>;
  static constexpr size_t staging = sizeof(T) * LPC2 * RS;
  static constexpr size_t stage_al = (staging + 15) / 16 * 16;
  static constexpr int XA = A::X > A::Z ? A::X : A::Z;
  static constexpr int XB = B::X > B::Z ? B::X : B::Z;
  // the exchange buffer also receives the FFT output (after a barrier); the
  // twiddle, post-twiddle and eigenvalue tables (4 KB in FP32) are read
  // through the L1 cache, which keeps an FP32 CTA within a sixth of the
  // shared memory: six CTAs per SM up to N = 128, so that the 1536 CTAs of a
  // three-job stage at N = 128 run in two waves of 912 slots instead of three
  // of 760 (at N = 256 the staging rows hold four per SM)
  static constexpr size_t xbuf = sizeof(C2<T>) * (XA > XB ? XA : XB);
  static constexpr size_t bytes = stage_al + xbuf;
};

// Where the lines of a transform come from and go to.  Lines are taken in
// pairs (2p, 2p + 1): the two real lines of one complex FFT.
// The staged lines of a CTA in shared memory (row stride N + 1).
template <typename T>
struct SmemLines {
  T* Rb;
  int RS;
  __device__ __forceinline__ T a(int p, int i) const { return Rb[(2 * p) * RS + i]; }
  __device__ __forceinline__ T b(int p, int i) const { return Rb[(2 * p + 1) * RS + i]; }
  __device__ __forceinline__ void put(int p, int o, T va, T vb) const {
    Rb[(2 * p) * RS + o] = va;
    Rb[(2 * p + 1) * RS + o] = vb;
  }
};
// An input value in the working type: FP64 input of an FP32 pass is rounded
// by integer operations (fastcvt.h; the conversion instruction runs on the
// FP64 pipe, a small fraction of the FP32 rate on this GPU).
template <typename T, typename Tin>
__device__ __forceinline__ T to_work(Tin v) {
  if constexpr (sizeof(T) == 4 && sizeof(Tin) == 8) return f64_to_f32(v);
  else return T(v);
}

// The CTA's lines straight from global memory: element i of line l at
// base[l * ls + i * es].
template <typename T, typename Tin>
struct GlobalLines {
  const Tin* base;
  int64_t ls, es;
  __device__ __forceinline__ T a(int p, int i) const {
    return to_work<T>(base[(int64_t)(2 * p) * ls + (int64_t)i * es]);
  }
  __device__ __forceinline__ T b(int p, int i) const {
    return to_work<T>(base[(int64_t)(2 * p + 1) * ls + (int64_t)i * es]);
  }
};
// Results straight to global memory (out = scale * v, or out += scale * v).
// Adjacent lines (ls == 1, the y and z passes) are written as one 2-vector.
template <typename T, typename Tout>
struct GlobalOut {
  Tout* base;
  int64_t ls, es;
  T sc;
  int acc;
  __device__ __forceinline__ void put(int p, int o, T va, T vb) const {
    Tout* q = base + (int64_t)(2 * p) * ls + (int64_t)o * es;
    if (acc) {
      va = T(q[0]) + sc * va;
      vb = T(q[ls]) + sc * vb;
    } else {
      va = sc * va;
      vb = sc * vb;
    }
    if constexpr (sizeof(Tout) == 4 || sizeof(Tout) == 8) {
      if (ls == 1) {
        using V2 = typename std::conditional<sizeof(Tout) == 4, float2, double2>::type;
        *reinterpret_cast<V2*>(q) = V2{Tout(va), Tout(vb)};
        return;
      }
    }
    q[0] = Tout(va);
    q[ls] = Tout(vb);
  }
};

// One real transform of the CTA's LPC2 lines, read through `src` and written
// through `dst` (which may be the same staged lines).
// KIND: 0 DCT-II family, 1 DST-II family, 2 DST-I.  INV: inverse.
// lines_fast: the output loop runs along the lines (coalesced for the y and z
// passes, whose lines are adjacent in memory) instead of along the index.
template <typename T, int N, int KIND, bool INV, class Src, class Dst>
__device__ void xform2(const Src& src, const Dst& dst, bool lines_fast, C2<T>* Xb, C2<T>* Zb, const C2<T>* tw,
                       const C2<T>* qN) {
  constexpr int L = (KIND == 2) ? 2 * N : N;
  constexpr int R = Fft2Shape<L>::R;
  constexpr int M = L / R;
  constexpr int XS = M + 1;                       // padded exchange row
  constexpr int ZS = L + 1;                       // padded output row
  constexpr int PAIRS = LPC2 / 2;
  constexpr int PPR = Fft2Shape<L>::PPR;          // pairs per round
  constexpr int ROUNDS = PAIRS / PPR;
  // DST-I is its own inverse up to the factor 2/N: both directions use the forward FFT
  constexpr bool FINV = (KIND == 2) ? false : INV;
  const int tid = threadIdx.x;
  const int pl = tid / M, m = tid - pl * M;       // pair within round, thread within pair
#pragma unroll 1
  for (int round = 0; round < ROUNDS; ++round) {
    const int p = round * PPR + pl;
    const bool active = pl < PPR;
    C2<T>* Xp = Xb + pl * (R * XS);
    C2<T>* Zp = Zb + pl * ZS;             // Zb aliases Xb
    if (active) {
      C2<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int n = m + M * r;
        C2<T> z;
        if constexpr (KIND == 2) {
          T a = 0, b = 0;
          if (n > 0 && n < N) { a = src.a(p, n); b = src.b(p, n); }
          else if (n > N) { a = -src.a(p, L - n); b = -src.b(p, L - n); }
          z = {a, b};
        } else if constexpr (!INV) {
          const int i = (n < N / 2) ? 2 * n : 2 * (N - 1 - n) + 1;
          T a = src.a(p, i), b = src.b(p, i);
          if (KIND == 1 && n >= N / 2) { a = -a; b = -b; }
          z = {a, b};
        } else {
          const int k = n;
          T xa, xna, xb, xnb;
          if constexpr (KIND == 1) {
            xa = src.a(p, N - 1 - k); xb = src.b(p, N - 1 - k);
            xna = k > 0 ? src.a(p, k - 1) : T(0); xnb = k > 0 ? src.b(p, k - 1) : T(0);
          } else {
            xa = src.a(p, k); xb = src.b(p, k);
            xna = k > 0 ? src.a(p, N - k) : T(0); xnb = k > 0 ? src.b(p, N - k) : T(0);
          }
          const C2<T> q = qN[k];                  // V = conj(q) (x_k - i x_{N-k})
          const C2<T> VA = {q.x * xa - q.y * xna, -q.x * xna - q.y * xa};
          const C2<T> VB = {q.x * xb - q.y * xnb, -q.x * xnb - q.y * xb};
          z = {VA.x - VB.y, VA.y + VB.x};
        }
        v[r] = z;
      }
      dft_any<R, FINV, T>(v);
#pragma unroll
      for (int s = 0; s < R; ++s) {
        if (s != 0 && m != 0) {
          // w_L^{m s} = exp(-2 pi i m s / L) = tw[(m s) * (2N / L)], table over the full circle
          C2<T> w = tw[(m * s) * (2 * N / L)];
          if (FINV) w.y = -w.y;
          v[s] = cmul(v[s], w);
        }
        Xp[s * XS + m] = v[s];
      }
    }
    __syncthreads();
    if constexpr (M <= R) {
      // step C: R/M DFTs of length M per thread, all read before the output
      // overwrites the exchange buffer
      constexpr int NS = R / M;
      C2<T> w[NS][M];
      if (active) {
#pragma unroll
        for (int q = 0; q < NS; ++q)
#pragma unroll
          for (int k = 0; k < M; ++k) w[q][k] = Xp[(q * M + m) * XS + k];
      }
      __syncthreads();
      if (active) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
          dft_reg<M, FINV, T>(w[q]);
#pragma unroll
          for (int k = 0; k < M; ++k) Zp[q * M + m + R * k] = w[q][k];
        }
      }
    } else {
      // step C for M = 2R (L = 512, the DST-I at N = 256; one warp per line
      // pair): Z[s + R k] = sum_m Y[m][s] w_M^{m k}.  Lane m takes s = m / 2
      // and the half m0 = m % 2 of the m index: a DFT of length R over m1 of
      // U[k'] = sum_m1 Y[2 m1 + m0][s] w_R^{m1 k'}, then the radix-2 step with
      // the partner lane m ^ 1, Z[s + R k] = U0[k'] + w_M^k' U1[k'] and
      // Z[s + R (k' + R)] = U0[k'] - w_M^k' U1[k'] (lane m0 = 0 writes the
      // first, lane m0 = 1 the second half).
      static_assert(M == 2 * R && PPR * M == PASS2_THREADS, "one warp per pair");
      const int s = m >> 1, m0 = m & 1;
      C2<T> u[R];
#pragma unroll
      for (int m1 = 0; m1 < R; ++m1) u[m1] = Xp[s * XS + 2 * m1 + m0];
      __syncthreads();
      dft_reg<R, FINV, T>(u);
#pragma unroll
      for (int k = 0; k < R; ++k) {
        const C2<T> o = {__shfl_xor_sync(0xffffffffu, u[k].x, 1), __shfl_xor_sync(0xffffffffu, u[k].y, 1)};
        C2<T> w = tw[k * (2 * N / M)];   // w_M^k = exp(-+ 2 pi i k / M)
        if (FINV) w.y = -w.y;
        const C2<T> u0 = m0 ? o : u[k];
        const C2<T> t1 = cmul(m0 ? u[k] : o, w);
        Zp[s + R * (k + R * m0)] = m0 ? C2<T>{u0.x - t1.x, u0.y - t1.y} : C2<T>{u0.x + t1.x, u0.y + t1.y};
      }
    }
    __syncthreads();
    // post-processing: output o of both lines of pair pr from the FFT row
    auto post = [&](int pr, int o) {
      const C2<T>* Z = Zb + pr * ZS;
      T va, vb;
      if constexpr (KIND == 2) {
        const T sc = INV ? T(1) / T(N) : T(0.5);
        const C2<T> z = Z[o];
        va = (o == 0) ? T(0) : -z.y * sc;
        vb = (o == 0) ? T(0) : z.x * sc;
      } else if constexpr (!INV) {
        const int k = (KIND == 1) ? (N - 1 - o) : o;
        const C2<T> zk = Z[k], zc = Z[k == 0 ? 0 : N - k];
        const C2<T> VA = {T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
        const C2<T> VB = {T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
        const C2<T> q = qN[k];
        va = q.x * VA.x - q.y * VA.y;
        vb = q.x * VB.x - q.y * VB.y;
      } else {
        const int n = (o & 1) ? (N - 1 - (o >> 1)) : (o >> 1);
        const C2<T> z = Z[n];
        const T sc = (KIND == 1 && (o & 1)) ? -T(1) / T(N) : T(1) / T(N);
        va = z.x * sc;
        vb = z.y * sc;
      }
      dst.put(round * PPR + pr, o, va, vb);
    };
    if (lines_fast) {
      for (int e = tid; e < PPR * N; e += PASS2_THREADS) post(e % PPR, e / PPR);
    } else {
      for (int e = tid; e < PPR * N; e += PASS2_THREADS) post(e / N, e % N);
    }
    __syncthreads();
  }
}

template <typename T, int N, class Src, class Dst>
__device__ __forceinline__ void xform2_dispatch(int type, const Src& src, const Dst& dst, bool lines_fast, C2<T>* Xb,
                                                C2<T>* Zb, const C2<T>* tw, const C2<T>* qN) {
  switch (type) {
    case X_DCT2F: xform2<T, N, 0, false>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    case X_DCT2I: xform2<T, N, 0, true>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    case X_DST2F: xform2<T, N, 1, false>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    case X_DST2I: xform2<T, N, 1, true>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    case X_DST1F: xform2<T, N, 2, false>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    case X_DST1I: xform2<T, N, 2, true>(src, dst, lines_fast, Xb, Zb, tw, qN); break;
    default: break;
  }
}

template <typename T, int N>
__device__ __forceinline__ T spectral_weight2(const PassArgs& a, const T* __restrict__ s2, T inv_mu,
                                              int i, int j, int k) {
  const T sum = s2[a.kind[0] * N + i] + s2[a.kind[1] * N + j] + s2[a.kind[2] * N + k];
  const int ac = a.wc == 0 ? i : (a.wc == 1 ? j : k);
  // correctly rounded reciprocal: the same value as T(1) / sum
  T isum;
  if constexpr (sizeof(T) == 4) isum = __frcp_rn(sum);
  else isum = __drcp_rn(sum);
  if (a.wmode == W_SCHUR) return s2[ac] * isum * inv_mu;
  if (ac == 0) return T(0);
  const T h = T(a.h);
  if (a.wmode == W_POISSON) return h * h * isum * inv_mu;
  return T(-2) * h * sqrt(T(0.25) * s2[ac]) * isum * inv_mu;   // W_RHS
}

// The staged lines of a CTA, written with the spectral weight applied (the
// fused middle pass: first transform, weight, second transform).
template <typename T, int N>
struct WeightedSmemLines {
  T* Rb;
  int RS;
  const PassArgs* a;
  const T* s2;
  T inv_mu;
  int line0, axis;
  __device__ __forceinline__ T w(int l, int n) const {
    const int line = line0 + l;
    int i, j, k;
    if (axis == 0) { i = n; j = line % N; k = line / N; }
    else if (axis == 1) { i = line % N; j = n; k = line / N; }
    else { i = line % N; j = line / N; k = n; }
    return spectral_weight2<T, N>(*a, s2, inv_mu, i, j, k);
  }
  __device__ __forceinline__ void put(int p, int o, T va, T vb) const {
    Rb[(2 * p) * RS + o] = va * w(2 * p, o);
    Rb[(2 * p + 1) * RS + o] = vb * w(2 * p + 1, o);
  }
};

// Up to three independent passes in one launch (blockIdx.y selects the job):
// the three components' transforms of one stage of the Schur apply, the
// Schur right-hand side or the velocity recovery.
template <typename Tin, typename Tout>
struct PassJob {
  const Tin* in;
  Tout* out;
  PassArgs a;
};
// Up to MAXJ jobs per launch: 3 for one instance, 48 for a batch of 16
// instances (kernel parameters of up to ~5 KB).
template <typename Tin, typename Tout, int MAXJ>
struct PassJobs {
  PassJob<Tin, Tout> j[MAXJ];
};

template <typename Tin, typename T, typename Tout, int N, int MAXJ>
__global__ void __launch_bounds__(PASS2_THREADS, (sizeof(T) == 4 ? (N <= 128 ? 6 : 4) : 2))
k_axis_pass2(const __grid_constant__ PassJobs<Tin, Tout, MAXJ> jobs, const C2<T>* __restrict__ tw,
             const C2<T>* __restrict__ qN, const T* __restrict__ s2) {
  using S = Pass2Smem<T, N>;
  extern __shared__ __align__(16) unsigned char smem2[];
  const PassJob<Tin, Tout>& job = jobs.j[blockIdx.y];
  const PassArgs& a = job.a;
  if (a.skip && *a.skip) return;
  const Tin* __restrict__ in = job.in;
  Tout* __restrict__ out = job.out;
  T* Rb = reinterpret_cast<T*>(smem2);
  C2<T>* Xb = reinterpret_cast<C2<T>*>(smem2 + S::stage_al);
  C2<T>* Zb = Xb;
  const C2<T>* tws = tw;
  const C2<T>* qs = qN;
  const T* s2s = s2;   // the eigenvalue table, read by the weight
  constexpr int RS = S::RS;
  const int line0 = blockIdx.x * LPC2;
  const int axis = a.axis;
  const int64_t NN = (int64_t)N * N;
  // lines: x: line = k N + j (contiguous); y: (k, i), base k N^2 + i; z: (j, i), base j N + i
  const int64_t stride = axis == 0 ? 1 : (axis == 1 ? N : NN);
  const int64_t base0 = axis == 0 ? (int64_t)line0 * N
                                  : (axis == 1 ? (int64_t)(line0 / N) * NN + (line0 % N) : (int64_t)line0);
  // for y and z the LPC2 lines of a CTA are consecutive in x (LPC2 divides N)
  const int64_t ls = axis == 0 ? (int64_t)N : 1;          // line stride
  const int64_t es = stride;                               // element stride
  const GlobalLines<T, Tin> gin{in + base0, ls, es};
  const bool lines_fast = axis != 0;
  if (a.wmode == W_NONE && a.type1 == X_NONE) {
    // plain pass: lines gathered from global memory into the FFT registers,
    // results written from the post-processing straight to global memory
    const GlobalOut<T, Tout> gout{out + base0, ls, es, T(a.scale), a.accumulate};
    xform2_dispatch<T, N>(a.type0, gin, gout, lines_fast, Xb, Zb, tws, qs);
    return;
  }
  const SmemLines<T> st{Rb, RS};
  if (a.wmode != W_NONE) {
    const WeightedSmemLines<T, N> wst{Rb, RS, &a, s2s, T(1.0 / a.mu), line0, axis};
    xform2_dispatch<T, N>(a.type0, gin, wst, false, Xb, Zb, tws, qs);
  } else {
    xform2_dispatch<T, N>(a.type0, gin, st, false, Xb, Zb, tws, qs);
  }
  if (a.type1 != X_NONE) {
    const GlobalOut<T, Tout> gout{out + base0, ls, es, T(a.scale), a.accumulate};
    xform2_dispatch<T, N>(a.type1, st, gout, lines_fast, Xb, Zb, tws, qs);
    return;
  }
  // weighted single transform: staged lines -> global
  const T sc = T(a.scale);
  constexpr int PER = LPC2 * N / PASS2_THREADS;
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const int e = threadIdx.x + q * PASS2_THREADS;
    int l, n;
    int64_t g;
    if (axis == 0) { l = e / N; n = e - l * N; g = base0 + e; }
    else { n = e / LPC2; l = e - n * LPC2; g = base0 + l + n * stride; }
    out[g] = a.accumulate ? Tout(T(out[g]) + sc * Rb[l * RS + n]) : Tout(sc * Rb[l * RS + n]);
  }
}

}  // namespace kfbim
