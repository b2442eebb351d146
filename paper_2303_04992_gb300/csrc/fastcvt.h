// Conversions between IEEE 754 binary64 and binary32 by integer operations on
// the encodings (sign bit, biased exponent, significand), for the FP32 steps
// of the MIXED refinement that read or write FP64 fields.  On GB300, FP64
// arithmetic and conversions to or from FP64 run at a small fraction of the
// FP32 and integer rates, so a streaming kernel that converts every element
// is bound by them; these take a few integer operations instead.
//
// Plain C++ (host and device): the CPU test suite compiles this header with
// g++ and compares it with the C++ conversions bit for bit.
#pragma once

#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define KFBIM_CVT_HD __host__ __device__ __forceinline__
#else
#define KFBIM_CVT_HD inline
#endif

namespace kfbim {

KFBIM_CVT_HD uint64_t cvt_bits64(double v) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(v);
#else
  uint64_t b;
  memcpy(&b, &v, sizeof b);
  return b;
#endif
}

KFBIM_CVT_HD double cvt_from_bits64(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}

KFBIM_CVT_HD uint32_t cvt_bits32(float v) {
#ifdef __CUDA_ARCH__
  return (uint32_t)__float_as_uint(v);
#else
  uint32_t b;
  memcpy(&b, &v, sizeof b);
  return b;
#endif
}

KFBIM_CVT_HD float cvt_from_bits32(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float v;
  memcpy(&v, &b, sizeof v);
  return v;
#endif
}

// binary64 -> binary32 rounded to nearest, ties to even, for results in the
// binary32 normal range (magnitude at least 2^-126).  Smaller magnitudes give
// a signed zero (no subnormal results), larger than the binary32 range a
// signed infinity (so does NaN, which the solver's fields never hold).
// The 52-bit significand keeps its top 23 bits; the 29 dropped bits decide
// the rounding, whose carry may run into the exponent (to the next binade,
// or to infinity from the largest one).
KFBIM_CVT_HD float f64_to_f32(double v) {
  const uint64_t b = cvt_bits64(v);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffu) - 1023 + 127;
  const uint32_t m = (uint32_t)(b >> 29) & 0x7fffffu;
  const uint32_t rest = (uint32_t)b & 0x1fffffffu;
  uint32_t r = ((uint32_t)(e < 0 ? 0 : e) << 23) | m;
  r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  r = e <= 0 ? 0u : (e >= 255 ? 0x7f800000u : r);
  return cvt_from_bits32(sign | r);
}

// binary32 -> binary64, exact for zero and normal numbers (a subnormal
// argument gives a signed zero); infinities and NaN keep their class.
KFBIM_CVT_HD double f32_to_f64(float v) {
  const uint32_t b = cvt_bits32(v);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t m = (uint64_t)(b & 0x7fffffu) << 29;
  const uint64_t r = e == 0 ? 0ull : (e == 255 ? (0x7ff0000000000000ull | m) : (((uint64_t)(e + 896) << 52) | m));
  return cvt_from_bits64(sign | r);
}

}  // namespace kfbim
