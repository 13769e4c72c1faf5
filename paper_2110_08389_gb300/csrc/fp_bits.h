// fp_bits.h -- conversions between binary32 and binary64 from the IEEE-754
// fields, with integer instructions only.  GB300 issues about two FP64
// instructions per SM per clock, and a conversion to or from a double counts
// as one; the refinement kernels of transfer.cu convert every node once, so
// these keep the FP64 pipe for the arithmetic of the defect.  Every class of
// value (normal, subnormal, zero, overflow, Inf, NaN) is handled by integer
// instructions: a fallback to the conversion instruction would be predicated
// into the common path and cost its FP64 issue slot anyway.  Plain C++ with a host/device
// qualifier, so that tests/fp_bits_driver.cpp checks them on the CPU against
// the compiler's own conversions.
#pragma once
#include <stdint.h>
#include <string.h>

#ifdef __CUDACC__
#define FPB_HD __host__ __device__ __forceinline__
#else
#define FPB_HD inline
#endif

namespace tmg {

FPB_HD uint64_t fpb_bits64(double x) {
#ifdef __CUDA_ARCH__
  return (uint64_t)__double_as_longlong(x);
#else
  uint64_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
FPB_HD uint32_t fpb_bits32(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  uint32_t b;
  memcpy(&b, &x, sizeof b);
  return b;
#endif
}
FPB_HD float fpb_float(uint32_t b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

FPB_HD double fpb_double(uint64_t b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, sizeof x);
  return x;
#endif
}

// Index of the highest set bit of a nonzero 32-bit word.
FPB_HD int fpb_top_bit(uint32_t m) {
#ifdef __CUDA_ARCH__
  return 31 - __clz((int)m);
#else
  return 31 - __builtin_clz(m);
#endif
}

// binary64 -> binary32, rounded to nearest, ties to even.  A normal result
// keeps the top 23 bits of the 52-bit fraction and the 29 dropped bits
// decide the rounding (above half: up; exactly half: up when the kept bits
// are odd); a carry out of the fraction moves into the exponent field, which
// is the correctly rounded result, up to Inf.  A subnormal result is the
// 53-bit significand shifted right to units of 2^-149 and rounded the same
// way (a carry into bit 23 gives the smallest normal, again correctly).
// Doubles above the float range give Inf, Inf stays Inf, NaN stays a quiet
// NaN.  Integer instructions only: no branch of it issues an FP64
// instruction, predicated or not.
FPB_HD float narrow_rne(double x) {
  const uint64_t b = fpb_bits64(x);
  const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ffu);
  const uint64_t frac = b & 0xfffffffffffffull;
  const int e = ex - 1023 + 127;
  uint32_t r;
  if (ex == 0x7ff) {
    r = frac ? 0x7fc00000u | (uint32_t)(frac >> 29) : 0x7f800000u;  // NaN (quiet) or Inf
  } else if (e > 254) {
    r = 0x7f800000u;  // beyond the largest finite float
  } else if (e >= 1) {
    const uint32_t kept = (uint32_t)(frac >> 29), rest = (uint32_t)frac & 0x1fffffffu;
    r = ((uint32_t)e << 23) | kept;
    if (rest > 0x10000000u || (rest == 0x10000000u && (kept & 1u))) r += 1u;
  } else {
    // |x| < 2^-126: q = m * 2^(ex - 1075) / 2^-149 = m >> (30 - e), m the significand
    const int sh = 30 - e;  // >= 30
    const uint64_t m = ex ? (frac | (1ull << 52)) : frac;  // a double subnormal is far below 2^-149
    if (sh > 54 || m == 0) {
      r = 0u;
    } else {
      const uint64_t q = m >> sh, rest = m & ((1ull << sh) - 1), half = 1ull << (sh - 1);
      r = (uint32_t)q;
      if (rest > half || (rest == half && (q & 1u))) r += 1u;
    }
  }
  return fpb_float(sign | r);
}

// binary32 -> binary64, exact: the sign, the exponent rebiased from 127 to
// 1023, the fraction moved up by 29 bits; a subnormal float is normalised
// (its top set bit becomes the hidden bit); zero, Inf and NaN keep their
// class (NaN its payload).  Integer instructions only.
FPB_HD double widen_exact(float x) {
  const uint32_t b = fpb_bits32(x);
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  const uint32_t ex = (b >> 23) & 0xffu, frac = b & 0x7fffffu;
  uint64_t r;
  if (ex == 0xffu) {
    r = (0x7ffull << 52) | ((uint64_t)frac << 29);
  } else if (ex != 0u) {
    r = ((uint64_t)(ex + 896u) << 52) | ((uint64_t)frac << 29);
  } else if (frac == 0u) {
    r = 0u;
  } else {
    // frac * 2^-149 = 1.f * 2^(p - 149), p the top set bit of frac
    const int p = fpb_top_bit(frac);
    r = ((uint64_t)(p + 874) << 52) | (((uint64_t)frac << (52 - p)) & 0xfffffffffffffull);
  }
  return fpb_double(sign | r);
}

}  // namespace tmg
