// device_util.cuh -- small device helpers shared by the line-solve kernels.
#pragma once
#include <utility>

#include "fp_bits.h"
#include "mg_internal.h"

namespace tmg {

// Checked builds (compiled with -DMG_CHECK, see build.py): every kernel
// validates the indices it decodes from its descriptors (node positions,
// junctions, tiles, sequences) and the ranges it derives from the level's
// shape before it touches memory with them.  A value out of range is
// recorded in this translation unit's check word, with the source line of
// the first check that failed, and replaced by the lower bound, so that the
// access stays inside the arrays and the kernel runs on (no trap, no early
// exit); the C ABI reads and clears the words after each call (mg_check_word)
// and returns MG_ERR_INVALID_ARG.  In other builds MG_RANGE is the value
// itself.
#ifdef MG_CHECK
#ifndef MG_CHECK_TU
#define MG_CHECK_TU "?"
#endif
static __device__ unsigned g_check_word;
static __device__ unsigned g_check_line;
__device__ __forceinline__ void mg_check_fail(unsigned line) {
  atomicOr(&g_check_word, 1u);
  atomicCAS(&g_check_line, 0u, line);
}
__device__ __forceinline__ int mg_range(int v, int lo, int hi, unsigned line) {
  if (v < lo || v > hi) {
    mg_check_fail(line);
    return lo;
  }
  return v;
}
#define MG_RANGE(v, lo, hi) ::tmg::mg_range((int)(v), (int)(lo), (int)(hi), __LINE__)
// true if c holds; else records it (the caller then skips the work)
__device__ __forceinline__ bool mg_ok_if(bool c, unsigned line) {
  if (!c) mg_check_fail(line);
  return c;
}
#define MG_OK_IF(c) ::tmg::mg_ok_if((c), __LINE__)
namespace {
unsigned read_check_word_tu(unsigned *line) {
  unsigned v = 0, l = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, g_check_word, sizeof(v)) != cudaSuccess) return ~0u;
  cudaMemcpyFromSymbol(&l, g_check_line, sizeof(l));
  cudaMemcpyToSymbol(g_check_word, &z, sizeof(z));
  cudaMemcpyToSymbol(g_check_line, &z, sizeof(z));
  *line = l;
  return v;
}
struct CheckWordReg {
  CheckWordReg() { register_check_reader(MG_CHECK_TU, &read_check_word_tu); }
} g_check_word_reg;
}  // namespace
#else
#define MG_RANGE(v, lo, hi) (v)
#define MG_OK_IF(c) true
#endif

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
// 1/|x| lie inside the float range (grid spacings above ~1e-18).  The seed's
// conversions to float and back use integer instructions (fp_bits.h, the
// same values as the conversion instructions), which keeps them off the
// FP64 pipe.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) {
  double r = widen_exact(__frcp_rn(narrow_rne(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

// Programmatic dependent launch.  Kernels of the cycle are launched with
// launch_pdl, so a kernel's CTAs may start while the previous kernel in the
// stream is still running.  Each such kernel calls pdl_trigger() first (its
// own dependents may then be scheduled) and pdl_wait() before its first
// access to data that an earlier kernel writes or reads (u, f, scratch): the
// wait returns once the previous grid has completed and its writes are
// visible.  Only constant data (descriptors, coefficients) is read before it.
// Both are no-ops in a kernel launched without the attribute.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Grids of at most this many CTAs are launched with the attribute.  Early
// start pays on the small levels, whose kernels are a few microseconds of
// latency each; for the large multi-wave grids of the fine levels it was
// measured slower on GB300.  4097^2 FP32+refine solve: 11.5 ms without PDL,
// 12.3 ms with it on every kernel, 11.4 ms with this limit; V(1,1) cycle on
// 129^2: 240 us without PDL, 180 us with it; 256 mixed batched problems:
// 0.256 s without, 0.247 s with this limit.
constexpr unsigned PDL_MAX_CTAS = 304;

// Launch with the attribute if `pdl`.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_ex(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                             Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
  return launch_ex(grid.x * grid.y * grid.z <= PDL_MAX_CTAS, kern, grid, block, smem, s, std::forward<Args>(args)...);
}

}  // namespace tmg
