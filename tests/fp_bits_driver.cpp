// Checks the integer conversions of csrc/fp_bits.h on the CPU against the
// compiler's own: narrow_rne against a double -> float conversion (round to
// nearest, ties to even) on edge cases (ties either way, carries into the
// exponent and out of the subnormal range, the largest finite float, the
// subnormal boundary and the rounding to zero below it, zeros, Inf, NaN) and
// random bit patterns over every exponent; widen_exact against float ->
// double on every one of the 2^32 floats.  Prints "ok <count>" or the first
// mismatch.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <limits>
#include <random>
#include <vector>

#include "../paper_2110_08389_gb300/csrc/fp_bits.h"

static double from_bits(uint64_t b) {
  double x;
  std::memcpy(&x, &b, sizeof x);
  return x;
}

static bool same(float a, float b) {
  uint32_t x, y;
  std::memcpy(&x, &a, 4);
  std::memcpy(&y, &b, 4);
  return x == y || (std::isnan(a) && std::isnan(b));
}

static bool same64(double a, double b) {
  uint64_t x, y;
  std::memcpy(&x, &a, 8);
  std::memcpy(&y, &b, 8);
  return x == y || (std::isnan(a) && std::isnan(b));
}

int main(int argc, char **argv) {
  const long n = argc > 1 ? std::atol(argv[1]) : 4000000;
  long wcount = 0;
  for (uint64_t k = 0; k < (1ull << 32); ++k) {
    const uint32_t b = (uint32_t)k;
    float x;
    std::memcpy(&x, &b, 4);
    if (!same64((double)x, tmg::widen_exact(x))) {
      std::printf("widen mismatch bits=%08x\n", b);
      return 1;
    }
    ++wcount;
  }
  std::vector<double> xs = {0.0, -0.0, 1.0, -1.0, 0.1, 1.0 / 3.0, 3.0e38, 3.4028234663852886e38,
                            3.4028235677973366e38, 3.5e38, 1e300, -1e300, 1.1754943508222875e-38,
                            1.1754942e-38, 1e-40, 1e-45, 1e-50, 5e-324,
                            std::numeric_limits<double>::infinity(), -std::numeric_limits<double>::infinity(),
                            std::numeric_limits<double>::quiet_NaN()};
  // ties and near-ties around kept bits even and odd, and carries
  for (uint64_t kept : {0x000000ull, 0x000001ull, 0x7ffffeull, 0x7fffffull, 0x123456ull})
    for (uint64_t rest : {0x0ffffffull, 0x10000000ull, 0x10000001ull, 0x1fffffffull, 0x0ull, 0x1ull})
      for (int ex : {1023 - 126, 1023 - 1, 1023, 1023 + 1, 1023 + 127})
        for (uint64_t sg : {0ull, 1ull})
          xs.push_back(from_bits((sg << 63) | ((uint64_t)ex << 52) | (kept << 29) | rest));
  // the subnormal range of the result and the rounding to zero below it
  for (int ex = 1023 - 155; ex <= 1023 - 125; ++ex)
    for (uint64_t frac : {0x0ull, 0x1ull, 0x8000000000000ull, 0xfffffffffffffull, 0x123456789abcdull,
                          0x4000000000000ull, 0xc000000000000ull})
      for (uint64_t sg : {0ull, 1ull}) xs.push_back(from_bits((sg << 63) | ((uint64_t)ex << 52) | frac));
  std::mt19937_64 rng(12345);
  for (long k = 0; k < n; ++k) {
    uint64_t b = rng();
    // exponents mostly around the float range, some beyond it
    const uint64_t ex = 1023 - 160 + (rng() % 330);
    b = (b & 0x800fffffffffffffull) | (ex << 52);
    xs.push_back(from_bits(b));
  }
  long count = 0;
  for (double x : xs) {
    const float want = (float)x, got = tmg::narrow_rne(x);
    if (!same(want, got)) {
      uint64_t b;
      std::memcpy(&b, &x, 8);
      std::printf("mismatch x=%.17g bits=%016llx want=%.9g got=%.9g\n", x, (unsigned long long)b, want, got);
      return 1;
    }
    ++count;
  }
  std::printf("ok %ld\n", count + wcount);
  return 0;
}
