// cluster_math.h -- the arithmetic of the cluster pass (cluster.cu) on one
// chunk: host- and device-callable, so that the CPU tests run the same
// eliminations on the cluster plan (cluster_host.h).
//
// Sec. 3, Eq. mLThomas: each leg of a block is eliminated from its wall end
// towards the junction, the junction row couples the legs' last unknowns, and
// back-substitution recovers the legs.  Here a leg's 32-node chunks are first
// reduced to two normalised rows each (partition method: a x_prev + x +
// c x_next = y), the leg is solved on those rows, and each chunk's interior
// is then recovered between its known end values.
#pragma once

#if defined(__CUDACC__)
#define CL_HD __host__ __device__ __forceinline__
#else
#define CL_HD inline
#endif

namespace tmg {
namespace clmath {

// Reciprocal: fast FP32 reciprocal on the device, division on the host.
CL_HD float rcp(float x) {
#if defined(__CUDA_ARCH__)
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}
CL_HD double rcp(double x) { return 1.0 / x; }

template <typename T>
struct Row {
  T a, c, y, n;  // n unused (padding to four values)
};

// Chunk of m <= 32 nodes of a leg: row q is lo(q) x_{q-1} + b_q x_q + hi(q)
// x_{q+1} = d[q] with b_q = -(cross + lo(q) + hi(q)); the predecessor of node
// 0 is a wall (coupling dropped) when FIRST, the successor of node m-1 is a
// wall when LAST_W.  CO provides lo(q), hi(q): the coefficients to the
// predecessor and successor along the run.
template <typename T, typename CO>
CL_HD void abc(const CO &co, int q, int m, bool first, bool last_w, T cross, T &a, T &b, T &c) {
  const T lo = co.lo(q), hi = co.hi(q);
  b = -(cross + (lo + hi));
  a = (q == 0 && first) ? T(0) : lo;
  c = (q == m - 1 && last_w) ? T(0) : hi;
}

// The chunk's two reduced rows (partition method): eliminate nodes 1..m-2
// towards node m-1 (hi row, in terms of x_0 and x_m) and nodes m-2..1
// towards node 0 (lo row, in terms of x_{-1} and x_{m-1}).  m = 1: lo only.
template <typename T, typename CO, typename D>
CL_HD void chunk_reduce(const CO &co, int m, bool first, bool last_w, T cross, const D &d, Row<T> &rlo,
                        Row<T> &rhi) {
  T a0, b0, c0;
  abc(co, 0, m, first, last_w, cross, a0, b0, c0);
  rhi.a = rhi.c = rhi.y = rhi.n = T(0);
  rlo.n = T(0);
  if (m <= 2) {
    const T rb = rcp(b0);
    rlo.a = a0 * rb; rlo.c = c0 * rb; rlo.y = d(0) * rb;
  }
  if (m < 2) return;
  T a1, b1, c1;
  abc(co, 1, m, first, last_w, cross, a1, b1, c1);
  const T ri = rcp(b1);
  T al = a1 * ri, ga = c1 * ri, de = d(1) * ri;
  T ah = T(0), ch = T(0), dh = T(0);
#pragma unroll
  for (int k = 1; k <= 30; ++k) {
    const int qf = k + 1;
    if (qf < m) {
      T a, b, c;
      abc(co, qf, m, first, last_w, cross, a, b, c);
      const T r = rcp(b - a * ga);
      al = -a * al * r;
      ga = c * r;
      de = (d(qf) - a * de) * r;
    }
    const int qb = 31 - k;
    if (qb <= m - 2) {
      T a, b, c;
      abc(co, qb, m, first, last_w, cross, a, b, c);
      if (qb == m - 2) {
        const T r = rcp(b);
        ah = a * r; ch = c * r; dh = d(qb) * r;
      } else {
        const T r = rcp(b - c * ah);
        ah = a * r;
        ch = -c * ch * r;
        dh = (d(qb) - c * dh) * r;
      }
    }
  }
  rhi.a = al; rhi.c = ga; rhi.y = de;
  if (m >= 3) {
    const T r = rcp(b0 - c0 * ah);
    rlo.a = a0 * r; rlo.c = -c0 * ch * r; rlo.y = (d(0) - c0 * dh) * r;
  }
}

// Interior nodes 1..m-2 of a chunk by Thomas between the known end values
// xlo (node 0) and xhi (node m-1); X provides x(q) (read and written) and the
// multipliers are kept in cp[] (length 32).
template <typename T, typename CO, typename D, typename X>
CL_HD void chunk_expand(const CO &co, int m, bool first, bool last_w, T cross, const D &d, T xlo, T xhi,
                        X &x, T *cp) {
  T dprev = xlo;
#pragma unroll
  for (int q = 1; q < 31; ++q) {
    if (q <= m - 2) {
      T a, b, c;
      abc(co, q, m, first, last_w, cross, a, b, c);
      T dq = d(q) - a * dprev;
      if (q == m - 2) dq -= c * xhi;
      const T r = (q == 1) ? rcp(b) : rcp(b - a * cp[q - 1]);
      cp[q] = c * r;
      dprev = dq * r;
      x.set(q, dprev);
    }
  }
  T xn = dprev;
#pragma unroll
  for (int q = 29; q >= 1; --q) {
    if (q <= m - 3) {
      xn = x.get(q) - cp[q] * xn;
      x.set(q, xn);
    }
  }
  // the ends (compile-time indices: X may be a register array)
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    if (q == 0) x.set(0, xlo);
    else if (q == m - 1) x.set(q, xhi);
  }
}

}  // namespace clmath
}  // namespace tmg
