// Checks the integer-operation conversions of fastcvt.h against the C++
// conversions (round to nearest even on the host) for binary32-normal
// results; prints the number of mismatches per category.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>

#include "fastcvt.h"

static bool same(float a, float b) {
  uint32_t x, y;
  std::memcpy(&x, &a, 4);
  std::memcpy(&y, &b, 4);
  return x == y;
}
static bool same64(double a, double b) {
  uint64_t x, y;
  std::memcpy(&x, &a, 8);
  std::memcpy(&y, &b, 8);
  return x == y;
}

int main() {
  std::mt19937_64 rng(12345);
  long bad_random = 0, bad_ties = 0, bad_back = 0, bad_small = 0, bad_big = 0, n = 0;
  for (int i = 0; i < 2000000; ++i) {
    // random sign, exponent within the binary32 normal range, random significand
    const uint64_t sign = (rng() & 1) << 63;
    const uint64_t e = 1023 - 126 + rng() % 254;   // 2^-126 .. 2^127
    const uint64_t m = rng() & ((1ull << 52) - 1);
    uint64_t b = sign | (e << 52) | m;
    double v;
    std::memcpy(&v, &b, 8);
    const float want = static_cast<float>(v);
    if (std::isfinite(want) && std::fabs(want) >= 1.1754943508222875e-38f && !same(kfbim::f64_to_f32(v), want))
      ++bad_random;
    // exact ties: dropped bits exactly half an ulp, both parities of the kept part
    b = sign | (e << 52) | (m & ~((1ull << 29) - 1)) | (1ull << 28);
    std::memcpy(&v, &b, 8);
    const float wt = static_cast<float>(v);
    if (std::isfinite(wt) && !same(kfbim::f64_to_f32(v), wt)) ++bad_ties;
    // binary32 -> binary64 is exact
    const float f = want;
    if (std::isfinite(f) && std::fabs(f) >= 1.1754943508222875e-38f && !same64(kfbim::f32_to_f64(f), (double)f))
      ++bad_back;
    ++n;
  }
  // below the binary32 normal range: signed zero; above: signed infinity
  const double smalls[] = {1e-300, -1e-300, 1e-40, -3e-39, 0.0, -0.0};
  for (double v : smalls) {
    const float r = kfbim::f64_to_f32(v);
    if (r != 0.0f || std::signbit(r) != std::signbit(v)) ++bad_small;
  }
  const double bigs[] = {1e39, -1e300, 3.4028235677973366e38};
  for (double v : bigs) {
    const float r = kfbim::f64_to_f32(v);
    if (!std::isinf(r) || std::signbit(r) != std::signbit(v)) ++bad_big;
  }
  if (kfbim::f64_to_f32(3.4028234663852886e38) != 3.4028234663852886e38f) ++bad_big;
  std::printf("n %ld\nrandom %ld\nties %ld\nback %ld\nsmall %ld\nbig %ld\n", n, bad_random, bad_ties, bad_back,
              bad_small, bad_big);
  return 0;
}
