// Real-to-real trigonometric transforms along one axis of an N^3 field, the
// building block of the FFT Poisson solver (Sec. 4.2 item ii) and of the
// spectral form of the Schur operator.
//
// Transforms of a line x_0..x_{N-1} (unnormalised forward, exact inverse):
//   DCT2F: X_a = sum_n x_n cos(pi a (n+1/2)/N),  a = 0..N-1        (cell values)
//   DST2F: X_{b-1} = sum_n x_n sin(pi b (n+1/2)/N),  b = 1..N      (zero-wall ghosts)
//   DST1F: X_a = sum_{n>=1} x_n sin(pi a n / N),  a = 1..N-1, X_0 = 0 (wall faces)
// DCT2/DST2 go through one length-N complex FFT per pair of lines (Makhoul's
// reordering; DST-II as DCT-II of (-1)^n x_n read backwards); DST1 through one
// length-2N complex FFT per pair of lines of the odd extension.  The FFT is a
// radix-2 Stockham in shared memory.
//
// One CTA transforms LPC lines.  For the x axis the lines are contiguous; for
// y and z the CTA takes LPC lines adjacent in x so that global loads and stores
// are coalesced across lines.  A pass may apply a first transform, a pointwise
// spectral weight and a second transform along the same axis before the store
// (the fused middle pass of a 3D transform pair).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kfbim {

enum Xform : int { X_NONE = 0, X_DCT2F, X_DCT2I, X_DST2F, X_DST2I, X_DST1F, X_DST1I };

enum WeightMode : int {
  W_NONE = 0,
  W_SCHUR = 1,    // sin^2(a_c)/sum sin^2 / mu     (component c, DCT along c)
  W_POISSON = 2,  // h^2 / (mu sum 4 sin^2)        (face grid c, DST-I along c)
  W_RHS = 3       // -2 h sin(a_c) / (mu sum 4 sin^2)  (face c -> cell basis c)
};

constexpr int LPC = 16;      // lines per CTA
constexpr int PASS_THREADS = 256;

struct PassArgs {
  int N;
  int axis;          // 0 x, 1 y, 2 z
  int type0, type1;  // type1 may be X_NONE
  int wmode, wc;     // weight mode, component axis (0..2) of the weight
  int kind[3];       // mode index of spectral axis b: idx (0) or idx + 1 (1)
  double mu, h;
  int accumulate;    // out += scale * result (else out = scale * result)
  double scale;
  const int* skip;   // nullable: the pass does nothing when *skip != 0
};

template <typename T>
struct C2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// Radix-2 Stockham FFT of P sequences of length L (power of two) held in smem
// buffer a (b is scratch).  tw[t] = exp(-2 pi i t / (2N)), t < N; twiddles of
// length L use stride 2N / L.  Returns the buffer holding the result.
template <typename T>
__device__ C2<T>* fft_stockham(C2<T>* a, C2<T>* b, int L, int P, const C2<T>* __restrict__ tw,
                               int twstride, bool inverse) {
  const int half = L >> 1;
  for (int Ns = 1; Ns < L; Ns <<= 1) {
    const int tstep = (half / Ns) * twstride;
    for (int w = threadIdx.x; w < P * half; w += blockDim.x) {
      const int p = w / half, j = w - p * half;
      const C2<T>* in = a + p * L;
      C2<T>* out = b + p * L;
      const C2<T> v0 = in[j];
      C2<T> v1 = in[j + half];
      const int k = j & (Ns - 1);
      C2<T> t = tw[k * tstep];
      if (inverse) t.y = -t.y;
      v1 = cmul(v1, t);
      const int idx = ((j - k) << 1) + k;
      out[idx] = {v0.x + v1.x, v0.y + v1.y};
      out[idx + Ns] = {v0.x - v1.x, v0.y - v1.y};
    }
    __syncthreads();
    C2<T>* s = a;
    a = b;
    b = s;
  }
  return a;
}

__device__ __forceinline__ int mak_perm(int n, int N) {
  // position in x of entry n of Makhoul's reordered sequence
  return (n < (N >> 1)) ? 2 * n : 2 * (N - 1 - n) + 1;
}

// Apply transform `type` to the LPC lines held in R (R[l*N + n]), in place.
template <typename T>
__device__ void line_transform(T* R, C2<T>* CA, C2<T>* CB, int N, int type,
                               const C2<T>* __restrict__ tw, const C2<T>* __restrict__ qN) {
  const int P = LPC / 2;
  if (type == X_NONE) return;
  if (type == X_DST1F || type == X_DST1I) {
    const int L = 2 * N;
    for (int e = threadIdx.x; e < P * L; e += blockDim.x) {
      const int p = e / L, n = e - p * L;
      T va = 0, vb = 0;
      if (n > 0 && n < N) {
        va = R[(2 * p) * N + n];
        vb = R[(2 * p + 1) * N + n];
      } else if (n > N) {
        va = -R[(2 * p) * N + (L - n)];
        vb = -R[(2 * p + 1) * N + (L - n)];
      }
      CA[e] = {va, vb};
    }
    __syncthreads();
    C2<T>* Z = fft_stockham(CA, CB, L, P, tw, 1, false);
    const T sc = (type == X_DST1I) ? T(1) / T(N) : T(0.5);  // (2/N) * (1/2)
    for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
      const int l = e / N, k = e - l * N;
      const int p = l >> 1;
      T v = 0;
      if (k > 0) {
        const C2<T> z = Z[p * L + k];
        v = (l & 1) ? z.x * sc : -z.y * sc;
      }
      R[e] = v;
    }
    __syncthreads();
    return;
  }
  const bool fwd = (type == X_DCT2F || type == X_DST2F);
  const bool dst = (type == X_DST2F || type == X_DST2I);
  const int L = N;
  if (fwd) {
    for (int e = threadIdx.x; e < P * L; e += blockDim.x) {
      const int p = e / L, n = e - p * L;
      const int src = mak_perm(n, N);
      T va = R[(2 * p) * N + src], vb = R[(2 * p + 1) * N + src];
      if (dst && n >= (N >> 1)) { va = -va; vb = -vb; }
      CA[e] = {va, vb};
    }
    __syncthreads();
    C2<T>* Z = fft_stockham(CA, CB, L, P, tw, 2, false);
    for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
      const int l = e / N, m = e - l * N;
      const int p = l >> 1;
      const int k = dst ? (N - 1 - m) : m;
      const C2<T> zk = Z[p * L + k];
      const C2<T> zc = Z[p * L + ((N - k) & (N - 1))];
      C2<T> V;
      if ((l & 1) == 0) V = {T(0.5) * (zk.x + zc.x), T(0.5) * (zk.y - zc.y)};
      else V = {T(0.5) * (zk.y + zc.y), T(-0.5) * (zk.x - zc.x)};
      const C2<T> q = qN[k];
      R[e] = q.x * V.x - q.y * V.y;
    }
    __syncthreads();
  } else {
    for (int e = threadIdx.x; e < P * L; e += blockDim.x) {
      const int p = e / L, k = e - p * L;
      T wa[2], wb[2];
      for (int s = 0; s < 2; ++s) {
        const T* Rl = R + (2 * p + s) * N;
        T xk, xnk;
        if (dst) {
          xk = Rl[N - 1 - k];
          xnk = (k > 0) ? Rl[k - 1] : T(0);
        } else {
          xk = Rl[k];
          xnk = (k > 0) ? Rl[N - k] : T(0);
        }
        wa[s] = xk;
        wb[s] = -xnk;
      }
      const C2<T> q = qN[k];  // V = conj(q) * W
      const C2<T> VA = {q.x * wa[0] + q.y * wb[0], q.x * wb[0] - q.y * wa[0]};
      const C2<T> VB = {q.x * wa[1] + q.y * wb[1], q.x * wb[1] - q.y * wa[1]};
      CA[e] = {VA.x - VB.y, VA.y + VB.x};
    }
    __syncthreads();
    C2<T>* Z = fft_stockham(CA, CB, L, P, tw, 2, true);
    const T inv = T(1) / T(N);
    for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
      const int l = e / N, nx = e - l * N;
      const int p = l >> 1;
      // nx = mak_perm(n): invert
      const int n = (nx & 1) ? (N - 1 - (nx >> 1)) : (nx >> 1);
      const C2<T> z = Z[p * L + n];
      T v = ((l & 1) ? z.y : z.x) * inv;
      if (dst && (nx & 1)) v = -v;
      R[e] = v;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void line_coords(int axis, int N, int line, int n, int& i, int& j, int& k) {
  if (axis == 0) { i = n; j = line % N; k = line / N; }
  else if (axis == 1) { i = line % N; j = n; k = line / N; }
  else { i = line % N; j = line / N; k = n; }
}

__device__ __forceinline__ int64_t line_base(int axis, int N, int line) {
  if (axis == 0) return (int64_t)line * N;
  if (axis == 1) return (int64_t)(line / N) * N * N + (line % N);
  return (int64_t)line;
}

__device__ __forceinline__ int64_t line_stride(int axis, int N) {
  return axis == 0 ? 1 : (axis == 1 ? N : (int64_t)N * N);
}

template <typename T>
__device__ __forceinline__ T spectral_weight(const PassArgs& a, const double* __restrict__ s2,
                                             int i, int j, int k) {
  const int id[3] = {i, j, k};
  double sum = 0.0;
  for (int b = 0; b < 3; ++b) sum += s2[a.kind[b] * a.N + id[b]];
  const int ac = id[a.wc];
  if (a.wmode == W_SCHUR) return T(s2[ac] / sum / a.mu);
  if (a.wmode == W_POISSON) return (ac == 0) ? T(0) : T(a.h * a.h / (a.mu * sum));
  // W_RHS: sin(pi a / 2N) = sqrt(s2 / 4)
  return (ac == 0) ? T(0) : T(-2.0 * a.h * sqrt(0.25 * s2[ac]) / (a.mu * sum));
}

template <typename Tin, typename T, typename Tout>
__global__ void __launch_bounds__(PASS_THREADS)
k_axis_pass(const Tin* __restrict__ in, Tout* __restrict__ out, PassArgs a,
            const C2<T>* __restrict__ tw, const C2<T>* __restrict__ qN,
            const double* __restrict__ s2) {
  extern __shared__ unsigned char smem_raw[];
  if (a.skip && *a.skip) return;
  const int N = a.N;
  T* R = reinterpret_cast<T*>(smem_raw);
  C2<T>* CA = reinterpret_cast<C2<T>*>(smem_raw + sizeof(T) * LPC * N);
  C2<T>* CB = CA + (LPC / 2) * 2 * N;
  const int line0 = blockIdx.x * LPC;
  const int64_t stride = line_stride(a.axis, N);
  // load (coalesced: along n for x lines, across lines otherwise)
  for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
    int l, n;
    if (a.axis == 0) { l = e / N; n = e - l * N; }
    else { n = e / LPC; l = e - n * LPC; }
    R[l * N + n] = T(in[line_base(a.axis, N, line0 + l) + n * stride]);
  }
  __syncthreads();
  line_transform<T>(R, CA, CB, N, a.type0, tw, qN);
  if (a.wmode != W_NONE) {
    for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
      const int l = e / N, n = e - l * N;
      int i, j, k;
      line_coords(a.axis, N, line0 + l, n, i, j, k);
      R[e] *= spectral_weight<T>(a, s2, i, j, k);
    }
    __syncthreads();
  }
  line_transform<T>(R, CA, CB, N, a.type1, tw, qN);
  const T sc = T(a.scale);
  for (int e = threadIdx.x; e < LPC * N; e += blockDim.x) {
    int l, n;
    if (a.axis == 0) { l = e / N; n = e - l * N; }
    else { n = e / LPC; l = e - n * LPC; }
    const int64_t g = line_base(a.axis, N, line0 + l) + n * stride;
    const T v = sc * R[l * N + n];
    if (a.accumulate) out[g] = Tout(T(out[g]) + v);
    else out[g] = Tout(v);
  }
}

inline size_t pass_smem_bytes(int N, size_t tsize) {
  return tsize * LPC * N + 2 * (LPC / 2) * 2 * N * 2 * tsize;
}

}  // namespace kfbim
