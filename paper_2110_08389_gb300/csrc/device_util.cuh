// device_util.cuh -- small device helpers shared by the line-solve kernels.
#pragma once
#include "mg_internal.h"

namespace tmg {

// The four coefficient arrays of a level (W_i, E_i over x; S_j, N_j over y).
template <typename T>
struct Coefs {
  const T *W, *E, *S, *N;
};
template <typename T>
inline Coefs<T> level_coefs(const Level &L);
template <>
inline Coefs<double> level_coefs<double>(const Level &L) { return {L.W64, L.E64, L.S64, L.N64}; }
template <>
inline Coefs<float> level_coefs<float>(const Level &L) { return {L.W32, L.E32, L.S32, L.N32}; }

// Reciprocal used by the eliminations.  FP32: the fast reciprocal (within 2
// ulp), ample for the FP32 correction equation.  FP64: Newton-Raphson
// iteration r <- r + r (1 - x r), which doubles the number of correct bits per
// step, started from the FP32 reciprocal (24 bits -> 48 -> 96); two fused
// steps replace the much slower IEEE double division.  Valid while |x| and
// 1/|x| lie inside the float range (grid spacings above ~1e-18).
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) {
  double r = (double)__frcp_rn((float)x);
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

}  // namespace tmg
