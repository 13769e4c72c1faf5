// warp_common.cuh -- pieces of the warp-path line solve shared by the 2D
// (warp_line.cu) and 3D (grid3d.cu) kernels: the shared-memory slot swizzle
// and the per-thread forward sweep / back-substitution of the partition
// method.
#pragma once
#include "device_util.cuh"

namespace tmg {

// slot of sequence node s in the per-warp arrays: an XOR swizzle that keeps
// both access patterns (32t + l and lK + q) free of bank conflicts
__device__ __forceinline__ int wslot(int s) { return s ^ ((s >> 5) & 31); }

// Step 2 for the thread owning nodes base .. base+K-1: the forward sweep over
// its interior nodes 0..K-2 (rows  x_q + c'_q x_{q+1} = y'_q + z'_q x_J +
// w'_q S_prev), then x_0 = Y0 + Z0 x_J + W0 S_prev + V0 S_own by a backward
// pass of multiply-adds.  K = 1: no interior (x_0 is the next separator).
template <typename T, int K>
struct Sweep {
  T cq[K], yq[K], zq[K], wq[K];  // entries 0..K-2 used
  T Y0 = T(0), Z0 = T(0), W0 = T(0), V0 = T(1);  // x_0 (as the next thread sees its own first node)
  T yl = T(0), zl = T(0), wl = T(1), cl = T(0);  // x_{K-2} = yl + zl x_J + wl S_prev - cl S_own
  __device__ __forceinline__ void run(int base, const T *sa, const T *sb, const T *sc, const T *sd, const T *sz) {
    if constexpr (K > 1) {
      {
        const int sl = wslot(base);
        const T r = recip(sb[sl]);
        cq[0] = sc[sl] * r;
        yq[0] = sd[sl] * r;
        zq[0] = sz[sl] * r;
        wq[0] = -sa[sl] * r;
      }
#pragma unroll
      for (int q = 1; q < K - 1; ++q) {
        const int sl = wslot(base + q);
        const T a = sa[sl];
        const T r = recip(sb[sl] - a * cq[q - 1]);
        cq[q] = sc[sl] * r;
        yq[q] = (sd[sl] - a * yq[q - 1]) * r;
        zq[q] = (sz[sl] - a * zq[q - 1]) * r;
        wq[q] = -a * wq[q - 1] * r;
      }
      yl = yq[K - 2]; zl = zq[K - 2]; wl = wq[K - 2]; cl = cq[K - 2];
      Y0 = yl; Z0 = zl; W0 = wl; V0 = -cl;
#pragma unroll
      for (int q = K - 3; q >= 0; --q) {
        Y0 = yq[q] - cq[q] * Y0;
        Z0 = zq[q] - cq[q] * Z0;
        W0 = wq[q] - cq[q] * W0;
        V0 = -cq[q] * V0;
      }
    }
  }
  // Step 4: interior values for both columns from the separators S_prev =
  // (sym, szm) and S_own = (sy, sz), written over the a (value) and b (x_J
  // column) slots.
  __device__ __forceinline__ void back(int base, T sym, T szm, T sy, T sz, T *sa, T *sb) const {
    sa[wslot(base + K - 1)] = sy;
    sb[wslot(base + K - 1)] = sz;
    T xy = sy, xz = sz;
#pragma unroll
    for (int q = K - 2; q >= 0; --q) {
      xy = yq[q] + wq[q] * sym - cq[q] * xy;
      xz = zq[q] + wq[q] * szm - cq[q] * xz;
      const int sl = wslot(base + q);
      sa[sl] = xy;
      sb[sl] = xz;
    }
  }
};

}  // namespace tmg
