// tile_math.cuh -- the chunk arithmetic shared by the 2D tiled line path
// (tiles.cu) and the 3D one (tiles3.cu): the partition method of Sec. 3's
// line solves on 32-node chunks (two reduced rows per chunk, and the chunk
// interior by Thomas between known ends), with the coefficients of a lane's
// slots given by the along-run coefficients staged per warp and the lane's
// perpendicular coefficient sum.
#pragma once
#include "device_util.cuh"

namespace tmg {
namespace {

__device__ __forceinline__ float rcp_t(float x) { return __fdividef(1.0f, x); }
// Newton-Raphson reciprocal from the FP32 one (as recip, device_util.cuh)
__device__ __forceinline__ double rcp_t(double x) {
  double r = widen_exact(__frcp_rn(narrow_rne(x)));
  double e = fma(-x, r, 1.0);
  r = fma(r, e, r);
  e = fma(-x, r, 1.0);
  return fma(r, e, r);
}

template <typename T>
struct __align__(4 * sizeof(T)) TRow {
  T a, c, y, z;  // a x_prev + x + c x_next = y   (z unused)
};

// Coefficients of slot q for a lane with m active slots and flags fl:
// a (predecessor), c (successor), b (diagonal).  The along coefficients of
// the tile's 32 positions are the same for every lane; each warp stages them
// once in shared memory (co[0][q] = predecessor side, co[1][q] = successor).
template <typename T>
__device__ __forceinline__ void abc(const T (&co)[2][32], int q, int m, int fl, T cross, T &a, T &b, T &c) {
  const T lo = co[0][q], hi = co[1][q];
  b = -(cross + (lo + hi));
  a = (q == 0 && (fl & TL_FIRST)) ? T(0) : lo;
  c = (q == m - 1 && (fl & TL_LAST_W)) ? T(0) : hi;
}

// The chunk's two reduced rows: eliminate nodes 1..m-2 towards node m-1 (hi
// row, in terms of x_0 and x_m) and nodes m-2..1 towards node 0 (lo row, in
// terms of x_{-1} and x_{m-1}); the two sweeps are interleaved.  FULL: m is
// CMAX, so every guard resolves at compile time.  COUP: also the rows'
// couplings a and c (they depend only on the coefficients; without COUP
// only the right-hand sides y are formed, a and c are left 0).
template <typename T, bool FULL, bool COUP = true>
__device__ __forceinline__ void reduce_rows(const T (&co)[2][32], int m_rt, int fl, T cross, const T (&d)[CMAX],
                                            TRow<T> &rlo, TRow<T> &rhi) {
  const int m = FULL ? CMAX : m_rt;
  T a0, b0, c0;
  abc(co, 0, m, fl, cross, a0, b0, c0);
  rhi.a = T(0); rhi.c = T(0); rhi.y = T(0); rhi.z = T(0);
  rlo.z = T(0);
  if (!COUP) { rlo.a = T(0); rlo.c = T(0); }
  if (m <= 2) {
    const T rb = rcp_t(b0);
    if (COUP) { rlo.a = a0 * rb; rlo.c = c0 * rb; }
    rlo.y = d[0] * rb;
  }
  if (m >= 2) {
    T a1, b1, c1;
    abc(co, 1, m, fl, cross, a1, b1, c1);
    T ri = rcp_t(b1);
    T al = COUP ? a1 * ri : T(0), ga = c1 * ri, de = d[1] * ri;
    T ah = T(0), ch = T(0), dh = T(0);
#pragma unroll
    for (int k = 1; k <= CMAX - 2; ++k) {
      const int qf = k + 1;
      if (qf < m) {
        T a, b, c;
        abc(co, qf, m, fl, cross, a, b, c);
        const T r = rcp_t(b - a * ga);
        if (COUP) al = -a * al * r;
        ga = c * r;
        de = (d[qf] - a * de) * r;
      }
      const int qb = CMAX - 1 - k;
      if (qb <= m - 2) {
        T a, b, c;
        abc(co, qb, m, fl, cross, a, b, c);
        if (qb == m - 2) {
          const T r = rcp_t(b);
          ah = a * r; dh = d[qb] * r;
          if (COUP) ch = c * r;
        } else {
          const T r = rcp_t(b - c * ah);
          ah = a * r;
          if (COUP) ch = -c * ch * r;
          dh = (d[qb] - c * dh) * r;
        }
      }
    }
    rhi.a = COUP ? al : T(0); rhi.c = COUP ? ga : T(0); rhi.y = de;
    if (m >= 3) {
      const T r = rcp_t(b0 - c0 * ah);
      if (COUP) { rlo.a = a0 * r; rlo.c = -c0 * ch * r; }
      rlo.y = (d[0] - c0 * dh) * r;
    }
  }
}

// Interior nodes 1..m-2 of a chunk by Thomas between the known end values
// xlo (node 0) and xhi (node m-1), into x (cpv: the multipliers).
template <typename T, bool FULL>
__device__ __forceinline__ void expand_rows(const T (&co)[2][32], int m_rt, int fl, T cross, const T (&dv)[CMAX],
                                            T xlo, T xhi, T *x, T *cpv) {
  const int m = FULL ? CMAX : m_rt;
  T dprev = xlo;
#pragma unroll
  for (int q = 1; q < CMAX - 1; ++q) {
    if (q <= m - 2) {
      T a, b, c;
      abc(co, q, m, fl, cross, a, b, c);
      T dq = dv[q] - a * dprev;
      if (q == m - 2) dq -= c * xhi;
      const T r = (q == 1) ? rcp_t(b) : rcp_t(b - a * cpv[q - 1]);
      cpv[q] = c * r;
      dprev = dq * r;
      x[q] = dprev;
    }
  }
  T xn = dprev;
#pragma unroll
  for (int q = CMAX - 3; q >= 1; --q) {
    if (q <= m - 3) {
      xn = x[q] - cpv[q] * xn;
      x[q] = xn;
    }
  }
  x[0] = xlo;
  x[m - 1] = xhi;
}

}  // namespace
}  // namespace tmg
