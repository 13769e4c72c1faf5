// warp_line.cu -- one colour pass of a line smoother (tweed, wireframe, zebra)
// on the small levels: one warp per sequence of whole blocks, no CTA barrier.
//
// Every block of the colour is solved exactly, the other colour held fixed
// (Sec. 3).  The blocks given to a warp are laid end to end as one
// tridiagonal system of at most 32*K unknowns (couplings between different
// chains are zero), plus at most one junction node J that is coupled to up
// to four of them (the centre of a tweed cross or T, Eq. mLThomas; the corner
// where a wireframe ring is closed, Eq. CircTri; a lone point block).  Row s:
//     a_s x_{s-1} + b_s x_s + c_s x_{s+1} = d_s - k_s x_J,
// and the junction row  C_J x_J + sum_e k'_e x_{s_e} = r_J.
//
// The solve (the partition method of the line kernel, regrouped for a warp):
//   1. coalesced staging: lane l handles nodes 32t + l; a, b, c, d and
//      z = -k go to shared memory.
//   2. lane l owns nodes lK .. lK+K-1.  Its interior nodes 0..K-2 are
//      eliminated by one forward Thomas sweep in which the unknown separator
//      S_{l-1} (the last node of lane l-1) and x_J are carried as extra
//      columns:  x_q + c'_q x_{q+1} = y'_q + z'_q x_J + w'_q S_{l-1}.
//      A backward pass of multiply-adds gives x_0 in terms of S_{l-1}, S_l
//      and x_J.
//   3. the separators form a tridiagonal system of 32 rows, one per lane
//      (the row of node lK+K-1 with x_{lK+K-2} and x_{(l+1)K} substituted),
//      solved by parallel cyclic reduction over warp shuffles for two
//      right-hand sides: S_l = Y_l + Z_l x_J.
//   4. back-substitution of the interior, again for both columns:
//      x_s = X_s + x_J X'_s.
//   5. the junction row fixes x_J (lanes 0..3 hold its attached nodes),
//      then x_s is written back coalesced.
#include "packed.h"
#include "warp_common.cuh"

namespace tmg {
namespace {

template <typename T>
__device__ __forceinline__ T by_dir(unsigned d, T e, T w, T n, T s) {
  return d == 0u ? e : (d == 1u ? w : (d == 2u ? n : s));
}

// Step 1 for a sequence of NT*K nodes handled by NT threads: thread t stages
// nodes NT*k + t (coalesced), U at a time; the next batch's descriptors are
// loaded while the current batch's data is in flight.  Writes a (coupling to
// the predecessor), b (diagonal; 1 on unused slots), c (to the successor),
// z = -k (to the junction), d (right-hand side with the other colour's
// neighbours moved over) and the node's offset in u (-1 on unused slots).
template <typename T, int K, int NT>
__device__ __forceinline__ void stage_nodes(const uint2 *__restrict__ nd, int t, const Coefs<T> &cp, int nx1,
                                            int ny1, const T *__restrict__ u, const T *__restrict__ f, T *sa, T *sb, T *sc,
                                            T *sd, T *sz, int *sp) {
  constexpr int U = K < 8 ? K : 8;
  uint2 cur[U];
#pragma unroll
  for (int k = 0; k < U; ++k) cur[k] = __ldg(nd + NT * k + t);
  pdl_wait();  // u and f from here on
#pragma unroll
  for (int t0 = 0; t0 < K; t0 += U) {
    uint2 nxt[U];
#pragma unroll
    for (int k = 0; k < U; ++k)
      if (t0 + U < K) nxt[k] = __ldg(nd + NT * (t0 + U + k) + t);
    T fv[U], ue[U], uw[U], un[U], us[U], ce[U], cw[U], cn[U], cs[U];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      // checked builds: a node must be an interior node of the level (else
      // its slot is treated as unused)
      if ((cur[k].y & WN_VALID) && !MG_OK_IF((cur[k].x & 0xFFFFu) >= 1u && (int)(cur[k].x & 0xFFFFu) <= nx1 - 2 &&
                                               (cur[k].x >> 16) >= 1u && (int)(cur[k].x >> 16) <= ny1 - 2))
        cur[k] = make_uint2(0u, 0u);
      const unsigned fl = cur[k].y;
      const int i = (int)(cur[k].x & 0xFFFFu), j = (int)(cur[k].x >> 16);
      const unsigned in = ((fl & WN_PRED) ? 1u << (fl & 3u) : 0u) | ((fl & WN_SUCC) ? 1u << ((fl >> 3) & 3u) : 0u) |
                          ((fl & WN_JUNC) ? 1u << ((fl >> 6) & 3u) : 0u);
      const unsigned out = (fl & WN_VALID) ? (0xFu & ~in) : 0u;
      const size_t p = (size_t)j * nx1 + i;
      fv[k] = (fl & WN_VALID) ? __ldg(f + p) : T(0);
      ue[k] = (out & 1u) ? u[p + 1] : T(0);
      uw[k] = (out & 2u) ? u[p - 1] : T(0);
      un[k] = (out & 4u) ? u[p + nx1] : T(0);
      us[k] = (out & 8u) ? u[p - nx1] : T(0);
      ce[k] = __ldg(cp.E + i);
      cw[k] = __ldg(cp.W + i);
      cn[k] = __ldg(cp.N + j);
      cs[k] = __ldg(cp.S + j);
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      const unsigned fl = cur[k].y;
      const bool valid = (fl & WN_VALID) != 0u;
      const int s = NT * (t0 + k) + t, sl = wslot(s);
      sa[sl] = (fl & WN_PRED) ? by_dir(fl & 3u, ce[k], cw[k], cn[k], cs[k]) : T(0);
      sc[sl] = (fl & WN_SUCC) ? by_dir((fl >> 3) & 3u, ce[k], cw[k], cn[k], cs[k]) : T(0);
      sz[sl] = (fl & WN_JUNC) ? -by_dir((fl >> 6) & 3u, ce[k], cw[k], cn[k], cs[k]) : T(0);
      sb[sl] = valid ? -((cw[k] + ce[k]) + (cs[k] + cn[k])) : T(1);
      sd[sl] = fv[k] - ce[k] * ue[k] - cw[k] * uw[k] - cn[k] * un[k] - cs[k] * us[k];
      sp[s] = valid ? (int)((cur[k].x >> 16) * (unsigned)nx1 + (cur[k].x & 0xFFFFu)) : -1;
    }
    if (t0 + U < K) {
#pragma unroll
      for (int k = 0; k < U; ++k) cur[k] = nxt[k];
    }
  }
}

// The junction of a sequence: its coefficient towards attached node e
// (thread e < 4) and, from rhs(), its row's right-hand side r_J (thread 0).
template <typename T>
struct Junction {
  uint4 jb;
  bool has_j;
  int natt;
  unsigned att = 0;  // directions from the junction to its attached nodes
  T kp = T(0), rJ = T(0), cJ = T(1), ce = T(0), cw = T(0), cn = T(0), cs = T(0);
  size_t p = 0;
  __device__ __forceinline__ Junction(const WBlock *__restrict__ blks, int seq, int t, const Coefs<T> &cp, int nx1,
                                      int ny1, int nslot) {
    jb = __ldg(reinterpret_cast<const uint4 *>(blks) + seq);
    has_j = (jb.y & 0xFFu) != 0u;
    natt = (int)((jb.y >> 8) & 0xFFu);
    // checked builds: the junction must be interior, with at most 4 attached
    // nodes inside the sequence (else the sequence has no junction)
    if (has_j && !MG_OK_IF(natt <= 4 && (jb.x & 0xFFFFu) >= 1u && (int)(jb.x & 0xFFFFu) <= nx1 - 2 &&
                           (jb.x >> 16) >= 1u && (int)(jb.x >> 16) <= ny1 - 2 && (int)(jb.z & 0xFFFFu) < nslot &&
                           (int)(jb.z >> 16) < nslot && (int)(jb.w & 0xFFFFu) < nslot && (int)(jb.w >> 16) < nslot)) {
      has_j = false;
      natt = 0;
    }
    const unsigned adirs = (jb.y >> 16) & 0xFFu;
    if (has_j && t < 4) {
      const int ji = (int)(jb.x & 0xFFFFu), jj = (int)(jb.x >> 16);
      p = (size_t)jj * nx1 + ji;
      ce = __ldg(cp.E + ji); cw = __ldg(cp.W + ji); cn = __ldg(cp.N + jj); cs = __ldg(cp.S + jj);
      for (int q = 0; q < natt; ++q) att |= 1u << ((adirs >> (2 * q)) & 3u);
      if (t < natt) kp = by_dir((adirs >> (2 * t)) & 3u, ce, cw, cn, cs);
      cJ = -((cw + ce) + (cs + cn));
    }
  }
  // after pdl_wait(): r_J = f_J minus the junction's neighbours outside the block
  __device__ __forceinline__ void rhs(int t, int nx1, const T *__restrict__ u, const T *__restrict__ f) {
    if (has_j && t == 0) {
      T r = __ldg(f + p);
      if (!(att & 1u)) r -= ce * u[p + 1];
      if (!(att & 2u)) r -= cw * u[p - 1];
      if (!(att & 4u)) r -= cn * u[p + nx1];
      if (!(att & 8u)) r -= cs * u[p - nx1];
      rJ = r;
    }
  }
  // Step 5, called by all lanes of one warp once the value (xa) and x_J
  // (xb) columns of the attached nodes are in shared memory: x_J from the
  // junction row (valid in lane 0).
  __device__ __forceinline__ T solve(int lane, const T *xa, const T *xb) const {
    T sy = T(0), sz = T(0);
    if (lane < natt) {
      const unsigned word = lane < 2 ? jb.z : jb.w;
      const int s = (int)((word >> (16 * (lane & 1))) & 0xFFFFu);
      sy = kp * xa[wslot(s)];
      sz = kp * xb[wslot(s)];
    }
    sy += __shfl_xor_sync(0xFFFFFFFFu, sy, 1);
    sz += __shfl_xor_sync(0xFFFFFFFFu, sz, 1);
    sy += __shfl_xor_sync(0xFFFFFFFFu, sy, 2);
    sz += __shfl_xor_sync(0xFFFFFFFFu, sz, 2);
    return (rJ - sy) / (cJ + sz);
  }
};

template <typename T, int K>
__global__ void __launch_bounds__(32) warp_line_kernel(const WNode *__restrict__ nodes,
                                                       const WBlock *__restrict__ blks, Coefs<T> cp, int nx1,
                                                       int ny1, T *__restrict__ u, const T *__restrict__ f,
                                                       const PassArgs<T> *__restrict__ tab,
                                                       const int *__restrict__ active) {
  if (tab) {  // packed launch: blockIdx.y selects the problem
    if (!active[blockIdx.y]) return;
    const PassArgs<T> a = tab[blockIdx.y];
    cp = a.c;
    u = a.u;
    f = a.f;
  }
  constexpr int N = 32 * K;
  extern __shared__ __align__(16) unsigned char wsm[];
  T *sa = reinterpret_cast<T *>(wsm);
  T *sb = sa + N, *sc = sb + N, *sd = sc + N, *sz = sd + N;
  int *sp = reinterpret_cast<int *>(sz + N);
  const int lane = threadIdx.x;
  const uint2 *nd = reinterpret_cast<const uint2 *>(nodes) + (size_t)blockIdx.x * N;

  pdl_trigger();
  // ---- the warp's junction
  Junction<T> jn(blks, blockIdx.x, lane, cp, nx1, ny1, N);

  // ---- 1. staging (waits for the previous kernel after its first descriptors)
  stage_nodes<T, K, 32>(nd, lane, cp, nx1, ny1, u, f, sa, sb, sc, sd, sz, sp);
  jn.rhs(lane, nx1, u, f);
  __syncwarp();

  // ---- 2. forward sweep over the lane's interior nodes 0..K-2
  const int base = lane * K;
  Sweep<T, K> sw;
  sw.run(base, sa, sb, sc, sd, sz);

  // ---- 3. separator rows, then cyclic reduction across the lanes
  const int ss = wslot(base + K - 1);
  T A, C, Ry, Rz;
  {
    T Yn = __shfl_down_sync(0xFFFFFFFFu, sw.Y0, 1), Zn = __shfl_down_sync(0xFFFFFFFFu, sw.Z0, 1);
    T Wn = __shfl_down_sync(0xFFFFFFFFu, sw.W0, 1), Vn = __shfl_down_sync(0xFFFFFFFFu, sw.V0, 1);
    if (lane == 31) { Yn = T(0); Zn = T(0); Wn = T(0); Vn = T(0); }
    const T a = sa[ss], c = sc[ss];
    const T B = sb[ss] - a * sw.cl + c * Wn;
    const T r = recip(B);
    A = a * sw.wl * r;
    C = c * Vn * r;
    Ry = (sd[ss] - a * sw.yl - c * Yn) * r;
    Rz = (sz[ss] - a * sw.zl - c * Zn) * r;
  }
#pragma unroll
  for (int dd = 1; dd < 32; dd <<= 1) {
    T Am = __shfl_up_sync(0xFFFFFFFFu, A, dd), Cm = __shfl_up_sync(0xFFFFFFFFu, C, dd);
    T Ym = __shfl_up_sync(0xFFFFFFFFu, Ry, dd), Zm = __shfl_up_sync(0xFFFFFFFFu, Rz, dd);
    T Ap = __shfl_down_sync(0xFFFFFFFFu, A, dd), Cp = __shfl_down_sync(0xFFFFFFFFu, C, dd);
    T Yp = __shfl_down_sync(0xFFFFFFFFu, Ry, dd), Zp = __shfl_down_sync(0xFFFFFFFFu, Rz, dd);
    if (lane < dd) { Am = T(0); Cm = T(0); Ym = T(0); Zm = T(0); }
    if (lane + dd >= 32) { Ap = T(0); Cp = T(0); Yp = T(0); Zp = T(0); }
    const T r = recip(T(1) - A * Cm - C * Ap);
    const T nA = -A * Am * r, nC = -C * Cp * r;
    const T nY = (Ry - A * Ym - C * Yp) * r, nZ = (Rz - A * Zm - C * Zp) * r;
    A = nA; C = nC; Ry = nY; Rz = nZ;
  }

  // ---- 4. back-substitution of the interior for both columns; the results
  // overwrite the lane's own a (value column) and b (x_J column) slots
  {
    T Sym = __shfl_up_sync(0xFFFFFFFFu, Ry, 1), Szm = __shfl_up_sync(0xFFFFFFFFu, Rz, 1);
    if (lane == 0) { Sym = T(0); Szm = T(0); }
    sw.back(base, Sym, Szm, Ry, Rz, sa, sb);
  }
  __syncwarp();

  // ---- 5. junction value, then all values back to u
  T xJ = T(0);
  if (jn.has_j) {
    xJ = __shfl_sync(0xFFFFFFFFu, jn.solve(lane, sa, sb), 0);
    if (lane == 0) u[jn.p] = xJ;
  }
#pragma unroll
  for (int t = 0; t < K; ++t) {
    const int s = 32 * t + lane;
    const int p = sp[s];
    if (p >= 0) {
      const int sl = wslot(s);
      u[p] = sa[sl] + xJ * sb[sl];
    }
  }
}

// The same solve for sequences of 32*W*K nodes on a CTA of W warps: the
// separator system has 32*W rows and its cyclic reduction runs through
// shared memory, one barrier per step.
template <typename T, int K, int W>
__global__ void __launch_bounds__(32 * W) seq_line_kernel(const WNode *__restrict__ nodes,
                                                          const WBlock *__restrict__ blks, Coefs<T> cp, int nx1,
                                                          int ny1, T *__restrict__ u, const T *__restrict__ f,
                                                          const PassArgs<T> *__restrict__ tab,
                                                          const int *__restrict__ active) {
  if (tab) {  // packed launch: blockIdx.y selects the problem
    if (!active[blockIdx.y]) return;
    const PassArgs<T> a = tab[blockIdx.y];
    cp = a.c;
    u = a.u;
    f = a.f;
  }
  constexpr int NT = 32 * W, N = NT * K;
  extern __shared__ __align__(16) unsigned char wsm[];
  T *sa = reinterpret_cast<T *>(wsm);
  T *sb = sa + N, *sc = sb + N, *sd = sc + N, *sz = sd + N;
  T *rep = sz + N;       // [4][NT]: x_0 of every thread (Y0, Z0, W0, V0)
  T *red = rep + 4 * NT;  // [2][4][NT]: separator rows (A, C, Y, Z), double-buffered
  T *xjs = red + 8 * NT;  // the junction value
  int *sp = reinterpret_cast<int *>(xjs + 2);
  const int t = threadIdx.x, lane = t & 31;
  const uint2 *nd = reinterpret_cast<const uint2 *>(nodes) + (size_t)blockIdx.x * N;
  pdl_trigger();
  Junction<T> jn(blks, blockIdx.x, t, cp, nx1, ny1, N);

  stage_nodes<T, K, NT>(nd, t, cp, nx1, ny1, u, f, sa, sb, sc, sd, sz, sp);
  jn.rhs(t, nx1, u, f);
  __syncthreads();

  const int base = t * K;
  Sweep<T, K> sw;
  sw.run(base, sa, sb, sc, sd, sz);
  rep[t] = sw.Y0; rep[NT + t] = sw.Z0; rep[2 * NT + t] = sw.W0; rep[3 * NT + t] = sw.V0;
  __syncthreads();

  const int ss = wslot(base + K - 1);
  T A, C, Ry, Rz;
  {
    const bool last = t == NT - 1;
    const T Yn = last ? T(0) : rep[t + 1], Zn = last ? T(0) : rep[NT + t + 1];
    const T Wn = last ? T(0) : rep[2 * NT + t + 1], Vn = last ? T(0) : rep[3 * NT + t + 1];
    const T a = sa[ss], c = sc[ss];
    const T r = recip(sb[ss] - a * sw.cl + c * Wn);
    A = a * sw.wl * r;
    C = c * Vn * r;
    Ry = (sd[ss] - a * sw.yl - c * Yn) * r;
    Rz = (sz[ss] - a * sw.zl - c * Zn) * r;
  }
  red[t] = A; red[NT + t] = C; red[2 * NT + t] = Ry; red[3 * NT + t] = Rz;
  __syncthreads();
  int cur = 0;
#pragma unroll
  for (int dd = 1; dd < NT; dd <<= 1) {
    const T *rb = red + 4 * NT * cur;
    T Am = T(0), Cm = T(0), Ym = T(0), Zm = T(0), Ap = T(0), Cp = T(0), Yp = T(0), Zp = T(0);
    if (t >= dd) { Am = rb[t - dd]; Cm = rb[NT + t - dd]; Ym = rb[2 * NT + t - dd]; Zm = rb[3 * NT + t - dd]; }
    if (t + dd < NT) { Ap = rb[t + dd]; Cp = rb[NT + t + dd]; Yp = rb[2 * NT + t + dd]; Zp = rb[3 * NT + t + dd]; }
    const T r = recip(T(1) - A * Cm - C * Ap);
    const T nA = -A * Am * r, nC = -C * Cp * r;
    const T nY = (Ry - A * Ym - C * Yp) * r, nZ = (Rz - A * Zm - C * Zp) * r;
    A = nA; C = nC; Ry = nY; Rz = nZ;
    cur ^= 1;
    T *wb = red + 4 * NT * cur;
    wb[t] = A; wb[NT + t] = C; wb[2 * NT + t] = Ry; wb[3 * NT + t] = Rz;
    __syncthreads();
  }
  {
    const T *rb = red + 4 * NT * cur;
    const T Sym = t > 0 ? rb[2 * NT + t - 1] : T(0), Szm = t > 0 ? rb[3 * NT + t - 1] : T(0);
    sw.back(base, Sym, Szm, Ry, Rz, sa, sb);
  }
  __syncthreads();

  T xJ = T(0);
  if (jn.has_j) {
    if (t < 32) {
      const T x = jn.solve(lane, sa, sb);
      if (t == 0) { xjs[0] = x; u[jn.p] = x; }
    }
    __syncthreads();
    xJ = xjs[0];
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const int s = NT * k + t;
    const int p = sp[s];
    if (p >= 0) {
      const int sl = wslot(s);
      u[p] = sa[sl] + xJ * sb[sl];
    }
  }
}

template <typename T, int K, int W>
constexpr size_t seq_smem() {
  return (size_t)32 * W * K * (5 * sizeof(T) + sizeof(int)) + sizeof(T) * (12 * 32 * W + 2);
}

// One launch: the problem (u, f) alone, or (pk.tab != nullptr) the pk.count
// problems of a packed group on grid rows.
template <typename T>
struct WarpLaunch {
  T *u;
  const T *f;
  PackedLaunch pk;
};

template <typename T, int K>
cudaError_t launch_k(const Level &L, const WarpList &w, const WarpLaunch<T> &a, cudaStream_t s) {
  const size_t smem = (size_t)32 * K * (5 * sizeof(T) + sizeof(int));
  count_launch(1);
  return launch_pdl(warp_line_kernel<T, K>, dim3(w.nwarp, a.pk.count), dim3(32), smem, s, (const WNode *)w.node,
                    (const WBlock *)w.blk, level_coefs<T>(L), L.nx + 1, L.ny + 1, a.u, a.f,
                    static_cast<const PassArgs<T> *>(a.pk.tab), a.pk.active);
}

template <typename T, int K, int W>
cudaError_t launch_kw(const Level &L, const WarpList &w, const WarpLaunch<T> &a, cudaStream_t s) {
  count_launch(1);
  return launch_pdl(seq_line_kernel<T, K, W>, dim3(w.nwarp, a.pk.count), dim3(32 * W), seq_smem<T, K, W>(), s,
                    (const WNode *)w.node, (const WBlock *)w.blk, level_coefs<T>(L), L.nx + 1, L.ny + 1, a.u, a.f,
                    static_cast<const PassArgs<T> *>(a.pk.tab), a.pk.active);
}

template <typename T, int K>
cudaError_t launch_multi(const Level &L, const WarpList &w, const WarpLaunch<T> &a, cudaStream_t s) {
  switch (w.W) {
    case 2: return launch_kw<T, K, 2>(L, w, a, s);
    case 4: return launch_kw<T, K, 4>(L, w, a, s);
    case 8: return launch_kw<T, K, 8>(L, w, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int K, int W>
cudaError_t opt_in() {
  return cudaFuncSetAttribute(seq_line_kernel<T, K, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)seq_smem<T, K, W>());
}
template <typename T, int K>
cudaError_t opt_in_all() {
  cudaError_t e = opt_in<T, K, 2>();
  if (e == cudaSuccess) e = opt_in<T, K, 4>();
  if (e == cudaSuccess) e = opt_in<T, K, 8>();
  return e;
}

template <typename T>
cudaError_t launch_shape(const Level &L, const WarpList &w, const WarpLaunch<T> &a, cudaStream_t s) {
  if (w.nwarp == 0 || a.pk.count == 0) return cudaSuccess;
  if (w.W == 1) {
    switch (w.K) {
      case 1: return launch_k<T, 1>(L, w, a, s);
      case 2: return launch_k<T, 2>(L, w, a, s);
      case 4: return launch_k<T, 4>(L, w, a, s);
      case 8: return launch_k<T, 8>(L, w, a, s);
      case 16:
        if constexpr (sizeof(T) == 4) return launch_k<T, 16>(L, w, a, s);
        return cudaErrorInvalidValue;
      default: return cudaErrorInvalidValue;
    }
  }
  switch (w.K) {
    case 1: return launch_multi<T, 1>(L, w, a, s);
    case 2: return launch_multi<T, 2>(L, w, a, s);
    case 4: return launch_multi<T, 4>(L, w, a, s);
    case 8: return launch_multi<T, 8>(L, w, a, s);
    case 16:
      if constexpr (sizeof(T) == 4) return launch_multi<T, 16>(L, w, a, s);
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

template <typename T>
cudaError_t launch_warp_pass(const Level &L, const WarpList &w, T *u, const T *f, cudaStream_t s) {
  return launch_shape<T>(L, w, WarpLaunch<T>{u, f, PackedLaunch{nullptr, nullptr, 1}}, s);
}

template <typename T>
cudaError_t launch_warp_pass_packed(const Level &L, const WarpList &w, const PackedLaunch &pk, cudaStream_t s) {
  return launch_shape<T>(L, w, WarpLaunch<T>{nullptr, nullptr, pk}, s);
}
template cudaError_t launch_warp_pass_packed<float>(const Level &, const WarpList &, const PackedLaunch &,
                                                    cudaStream_t);
template cudaError_t launch_warp_pass_packed<double>(const Level &, const WarpList &, const PackedLaunch &,
                                                     cudaStream_t);

cudaError_t prepare_warp_kernels() {
  cudaError_t e = opt_in_all<float, 1>();
  if (e == cudaSuccess) e = opt_in_all<float, 2>();
  if (e == cudaSuccess) e = opt_in_all<float, 4>();
  if (e == cudaSuccess) e = opt_in_all<float, 8>();
  if (e == cudaSuccess) e = opt_in_all<float, 16>();
  if (e == cudaSuccess) e = opt_in_all<double, 1>();
  if (e == cudaSuccess) e = opt_in_all<double, 2>();
  if (e == cudaSuccess) e = opt_in_all<double, 4>();
  if (e == cudaSuccess) e = opt_in_all<double, 8>();
  return e;
}

template cudaError_t launch_warp_pass<double>(const Level &, const WarpList &, double *, const double *, cudaStream_t);
template cudaError_t launch_warp_pass<float>(const Level &, const WarpList &, float *, const float *, cudaStream_t);

}  // namespace tmg
