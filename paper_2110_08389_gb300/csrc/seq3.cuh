// seq3.cuh -- the 3D warp-path kernels (Sec. 7), included by grid3d.cu (tweed
// lists, at most one junction per sequence) and grid3d_wf.cu (wireframe
// lists: ring junctions and edge skeletons), so that the two families
// compile in parallel and neither carries the other's code.
//
// A sequence holds the chains of whole blocks in 32*W*K slots, one CTA of W
// warps: the partition method of the 2D warp path (warp_common.cuh) with
// six directions, and each junction eliminated by superposition (its
// chains solved for the data and for a unit junction value, then the
// junction row).
#pragma once
#include "solve.h"
#include "warp_common.cuh"

namespace tmg {

namespace {

template <typename T>
struct C6 {
  const T *W, *E, *S, *N, *B, *T_;
};
template <typename T>
C6<T> coefs3(const Level3 &L);
template <>
C6<double> coefs3<double>(const Level3 &L) {
  return {L.c64[0], L.c64[1], L.c64[2], L.c64[3], L.c64[4], L.c64[5]};
}
template <>
C6<float> coefs3<float>(const Level3 &L) {
  return {L.c32[0], L.c32[1], L.c32[2], L.c32[3], L.c32[4], L.c32[5]};
}

// coefficient of row (i, j, k) towards direction d (0..5 = +x -x +y -y +z -z)
template <typename T>
__device__ __forceinline__ T cdir(const C6<T> &c, unsigned d, int i, int j, int k) {
  switch (d) {
    case 0: return __ldg(c.E + i);
    case 1: return __ldg(c.W + i);
    case 2: return __ldg(c.N + j);
    case 3: return __ldg(c.S + j);
    case 4: return __ldg(c.T_ + k);
    default: return __ldg(c.B + k);
  }
}


// Skeleton CTAs of a launch: edge scratch rows (a, b, c, r, zA, zB), each
// `stride` values long.
template <typename T>
struct SkelArgs {
  const WSkel3 *skel;
  T *scr;
  size_t stride;
  int nskel;
};

__device__ __forceinline__ void unpack3(uint32_t v, int &i, int &j, int &k) {
  i = (int)(v & 1023u); j = (int)((v >> 10) & 1023u); k = (int)(v >> 20);
}

// One wireframe edge skeleton per CTA (Sec. 7; the wireframe extension of
// the Thomas algorithm): every edge is a tridiagonal chain between two
// corners, eliminated by Thomas with three right-hand sides (the data, and
// the responses to unit values at its two corners); the eight corner rows
// then form an 8 x 8 system, solved by elimination (an M-matrix: no
// pivoting); the edges are recombined from the corner values.
__device__ __forceinline__ long long step3(unsigned d, int nx1, long long plane) {
  const long long m = d < 2 ? 1 : (d < 4 ? (long long)nx1 : plane);
  return (d & 1u) ? -m : m;
}

template <typename T>
__device__ __forceinline__ void skel_cta(const WSkel3 *__restrict__ S, T *__restrict__ scr, size_t stride,
                                      const T *__restrict__ cW, const T *__restrict__ cE, const T *__restrict__ cS,
                                      const T *__restrict__ cN, const T *__restrict__ cB, const T *__restrict__ cT,
                                      int nx1, int ny1, T *__restrict__ u, const T *__restrict__ f) {
  __shared__ T M[8][9];
  __shared__ T X[8];
  const C6<T> cp{cW, cE, cS, cN, cB, cT};
  const int t = threadIdx.x, nt = blockDim.x;
  const long long plane = (long long)nx1 * ny1;
  const int e0 = (int)S->eoff[0], e12 = (int)S->eoff[12];
  T *rA = scr, *rB = rA + stride, *rC = rB + stride, *rR = rC + stride, *rZA = rR + stride, *rZB = rZA + stride;
  pdl_wait();
  // 1. staging: the chain rows of every edge node
  for (int q = e0 + t; q < e12; q += nt) {
    int e = 0;
    while ((int)S->eoff[e + 1] <= q) ++e;
    const int sidx = q - (int)S->eoff[e];
    const unsigned d = S->ed[e];
    int i, j, k;
    unpack3(S->cijk[S->ea[e]], i, j, k);
    const long long p = (long long)k * plane + (long long)j * nx1 + i + (long long)(sidx + 1) * step3(d, nx1, plane);
    const int pi = (int)(p % nx1), pj = (int)((p / nx1) % ny1), pk = (int)(p / plane);
    T bb = T(0), r = __ldg(f + p), aa = T(0), cc = T(0);
#pragma unroll
    for (unsigned dd = 0; dd < 6; ++dd) {
      const T cd = cdir(cp, dd, pi, pj, pk);
      bb -= cd;
      if (dd == (d ^ 1u)) aa = cd;
      else if (dd == d) cc = cd;
      else r -= cd * u[p + step3(dd, nx1, plane)];
    }
    rA[q] = aa; rB[q] = bb; rC[q] = cc; rR[q] = r;
  }
  __syncthreads();
  // 2. Thomas per edge (thread e): columns y (data), zA, zB (unit corner
  // values); the rows are read SB at a time ahead of the recurrence
  if (t < 12) {
    constexpr int SB = 8;
    const int o = (int)S->eoff[t], m = (int)S->eoff[t + 1] - o;
    T cpv = T(0), y = T(0), za = T(0), cl = T(0), inv = T(0);
    for (int s0 = 0; s0 < m; s0 += SB) {
      T a8[SB], b8[SB], c8[SB], r8[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q)
        if (s0 + q < m) { a8[q] = rA[o + s0 + q]; b8[q] = rB[o + s0 + q]; c8[q] = rC[o + s0 + q]; r8[q] = rR[o + s0 + q]; }
#pragma unroll
      for (int q = 0; q < SB; ++q)
        if (s0 + q < m) {
          const int s = s0 + q;
          inv = T(1) / (b8[q] - a8[q] * cpv);
          cl = c8[q];
          cpv = cl * inv;
          y = (r8[q] - a8[q] * y) * inv;
          za = ((s == 0 ? -a8[q] : T(0)) - a8[q] * za) * inv;
          rC[o + s] = cpv; rR[o + s] = y; rZA[o + s] = za;
        }
    }
    T zb = -cl * inv;  // the last row's coupling to corner eb
    if (m > 0) rZB[o + m - 1] = zb;
    for (int s1 = m - 2; s1 >= 0; s1 -= SB) {  // rows s1, s1 - 1, ... down to 0
      T c8[SB], y8[SB], z8[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q)
        if (s1 - q >= 0) { c8[q] = rC[o + s1 - q]; y8[q] = rR[o + s1 - q]; z8[q] = rZA[o + s1 - q]; }
#pragma unroll
      for (int q = 0; q < SB; ++q)
        if (s1 - q >= 0) {
          const int s = s1 - q;
          y = y8[q] - c8[q] * y;
          za = z8[q] - c8[q] * za;
          zb = -c8[q] * zb;
          rR[o + s] = y; rZA[o + s] = za; rZB[o + s] = zb;
        }
    }
  }
  __syncthreads();
  // 3. corner rows (thread q), then elimination (thread 0)
  if (t < 8) {
    int i, j, k;
    unpack3(S->cijk[t], i, j, k);
    const long long p = (long long)k * plane + (long long)j * nx1 + i;
    for (int c = 0; c < 8; ++c) M[t][c] = T(0);
    unsigned inblk = 0;
    T diag = T(0), rhs = __ldg(f + p);
    for (int e = 0; e < 12; ++e) {
      const int o = (int)S->eoff[e], m = (int)S->eoff[e + 1] - o;
      if (S->ea[e] == t) {  // the edge's first node is next to this corner
        const unsigned d = S->ed[e];
        inblk |= 1u << d;
        const T kc = cdir(cp, d, i, j, k);
        M[t][t] += kc * rZA[o];
        M[t][S->eb[e]] += kc * rZB[o];
        rhs -= kc * rR[o];
      } else if (S->eb[e] == t) {
        const unsigned d = S->ed[e] ^ 1u;
        inblk |= 1u << d;
        const T kc = cdir(cp, d, i, j, k);
        M[t][S->ea[e]] += kc * rZA[o + m - 1];
        M[t][t] += kc * rZB[o + m - 1];
        rhs -= kc * rR[o + m - 1];
      }
    }
    for (unsigned d = 0; d < 6; ++d) {
      const T cd = cdir(cp, d, i, j, k);
      diag -= cd;
      if (!(inblk & (1u << d))) rhs -= cd * u[p + step3(d, nx1, plane)];
    }
    M[t][t] += diag;
    M[t][8] = rhs;
  }
  __syncthreads();
  if (t == 0) {
    for (int c = 0; c < 8; ++c) {
      const T ip = T(1) / M[c][c];
      for (int r = c + 1; r < 8; ++r) {
        const T l = M[r][c] * ip;
        for (int q = c; q < 9; ++q) M[r][q] -= l * M[c][q];
      }
    }
    for (int c = 7; c >= 0; --c) {
      T v = M[c][8];
      for (int q = c + 1; q < 8; ++q) v -= M[c][q] * X[q];
      X[c] = v / M[c][c];
    }
  }
  __syncthreads();
  // 4. write back
  if (t < 8) {
    int i, j, k;
    unpack3(S->cijk[t], i, j, k);
    u[(long long)k * plane + (long long)j * nx1 + i] = X[t];
  }
  for (int q = e0 + t; q < e12; q += nt) {
    int e = 0;
    while ((int)S->eoff[e + 1] <= q) ++e;
    const int sidx = q - (int)S->eoff[e];
    int i, j, k;
    unpack3(S->cijk[S->ea[e]], i, j, k);
    const long long p = (long long)k * plane + (long long)j * nx1 + i + (long long)(sidx + 1) * step3(S->ed[e], nx1, plane);
    u[p] = rR[q] + X[S->ea[e]] * rZA[q] + X[S->eb[e]] * rZB[q];
  }
}

// ------------------------------------------------------------ the kernels --
// One sequence of 32*W*K slots per CTA of W warps (the warp path of
// warp_line.cu, seq_line_kernel, with six directions).  Tweed lists: at most
// one junction per sequence, juncs[CTA] (natt = 0: none).
template <typename T, int K, int W>
__global__ void __launch_bounds__(32 * W) seq3_single_kernel(const WNode3 *__restrict__ nodes,
                                                             const WJunc3 *__restrict__ juncs, C6<T> cp, int nx1,
                                                             int ny1, int nz1, T *__restrict__ u,
                                                             const T *__restrict__ f) {
  constexpr int NT = 32 * W, N = NT * K;
  extern __shared__ __align__(16) unsigned char sm3[];
  T *sa = reinterpret_cast<T *>(sm3);
  T *sb = sa + N, *sc = sb + N, *sd = sc + N, *sz = sd + N;
  T *rep = sz + N;
  T *red = rep + 4 * NT;
  T *xjs = red + 8 * NT;
  int *sp = reinterpret_cast<int *>(xjs + 2);
  const int t = threadIdx.x, lane = t & 31;
  const size_t plane = (size_t)nx1 * ny1;
  const uint2 *nd = reinterpret_cast<const uint2 *>(nodes) + (size_t)blockIdx.x * N;
  pdl_trigger();
  // the junction: coefficient towards attached node e (thread e < natt)
  const WJunc3 *jbp = juncs + blockIdx.x;
  struct {
    uint32_t ijk, adirs;
  } jb;
  jb.ijk = jbp->ijk;
  jb.adirs = jbp->adirs;
  int natt = jbp->natt;
  // checked builds: the junction must be interior with at most 6 legs (else
  // the sequence has none)
  if (natt != 0 && !MG_OK_IF(natt <= 6 && (jb.ijk & 1023u) >= 1u && (int)(jb.ijk & 1023u) <= nx1 - 2 &&
                             ((jb.ijk >> 10) & 1023u) >= 1u && (int)((jb.ijk >> 10) & 1023u) <= ny1 - 2 &&
                             (jb.ijk >> 20) >= 1u && (int)(jb.ijk >> 20) <= nz1 - 2))
    natt = 0;
  const bool has_j = natt != 0;
  T kp = T(0), cJ = T(1);
  int ji = 0, jj = 0, jk = 0;
  unsigned att = 0;
  if (has_j) {
    ji = (int)(jb.ijk & 1023u); jj = (int)((jb.ijk >> 10) & 1023u); jk = (int)(jb.ijk >> 20);
    for (int e = 0; e < natt; ++e) att |= 1u << ((jb.adirs >> (3 * e)) & 7u);
    if (t < natt) kp = cdir(cp, (jb.adirs >> (3 * t)) & 7u, ji, jj, jk);
    cJ = T(0);
    for (unsigned d = 0; d < 6; ++d) cJ -= cdir(cp, d, ji, jj, jk);
  }
  pdl_wait();  // u and f from here on
  // ---- 1. staging (thread t: nodes NT*q + t)
#pragma unroll
  for (int q = 0; q < K; ++q) {
    uint2 dsc = __ldg(nd + NT * q + t);
    // checked builds: a node must be an interior node (else its slot is unused)
    if ((dsc.y & WN3_VALID) && !MG_OK_IF((dsc.x & 1023u) >= 1u && (int)(dsc.x & 1023u) <= nx1 - 2 &&
                                          ((dsc.x >> 10) & 1023u) >= 1u && (int)((dsc.x >> 10) & 1023u) <= ny1 - 2 &&
                                          (dsc.x >> 20) >= 1u && (int)(dsc.x >> 20) <= nz1 - 2))
      dsc = make_uint2(0u, 0u);
    const unsigned fl = dsc.y;
    const bool valid = (fl & WN3_VALID) != 0u;
    const int i = (int)(dsc.x & 1023u), j = (int)((dsc.x >> 10) & 1023u), k = (int)(dsc.x >> 20);
    const unsigned pd = (fl & WN3_PRED) ? (fl & 7u) : 7u, sd_ = (fl & WN3_SUCC) ? ((fl >> 4) & 7u) : 7u,
                   jd = (fl & WN3_JUNC) ? ((fl >> 8) & 7u) : 7u;
    const size_t p = (size_t)k * plane + (size_t)j * nx1 + i;
    const size_t off[6] = {1, (size_t)0 - 1, (size_t)nx1, (size_t)0 - nx1, plane, (size_t)0 - plane};
    T a = T(0), c = T(0), z = T(0), b = T(0), r = valid ? __ldg(f + p) : T(0);
#pragma unroll
    for (unsigned d = 0; d < 6; ++d) {
      const T cd = cdir(cp, d, i, j, k);
      b -= cd;
      const bool outside = valid && d != pd && d != sd_ && d != jd;
      if (outside) r -= cd * u[p + off[d]];
      if (d == pd) a = cd;
      if (d == sd_) c = cd;
      if (d == jd) z = -cd;
    }
    const int s = NT * q + t, sl = wslot(s);
    sa[sl] = a;
    sc[sl] = c;
    sz[sl] = z;
    sb[sl] = valid ? b : T(1);
    sd[sl] = r;
    sp[s] = valid ? (int)p : -1;
  }
  T rJ = T(0);
  size_t pJ = 0;
  if (has_j && t == 0) {
    pJ = (size_t)jk * plane + (size_t)jj * nx1 + ji;
    rJ = __ldg(f + pJ);
    const size_t off[6] = {1, (size_t)-1, (size_t)nx1, (size_t)0 - nx1, plane, (size_t)0 - plane};
#pragma unroll
    for (unsigned d = 0; d < 6; ++d)
      if (!(att & (1u << d))) rJ -= cdir(cp, d, ji, jj, jk) * u[pJ + off[d]];
  }
  __syncthreads();

  // ---- 2. forward sweep per thread
  const int base = t * K;
  Sweep<T, K> sw;
  sw.run(base, sa, sb, sc, sd, sz);
  rep[t] = sw.Y0; rep[NT + t] = sw.Z0; rep[2 * NT + t] = sw.W0; rep[3 * NT + t] = sw.V0;
  __syncthreads();

  // ---- 3. separator rows, cyclic reduction through shared memory
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

  // ---- 5. junction value (warp 0; up to six attached nodes), write back
  T xJ = T(0);
  if (has_j) {
    if (t < 32) {
      T sy = T(0), szz = T(0);
      if (lane < natt) {
        const int s = jbp->as[lane];
        sy = kp * sa[wslot(s)];
        szz = kp * sb[wslot(s)];
      }
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) {
        sy += __shfl_xor_sync(0xFFFFFFFFu, sy, o);
        szz += __shfl_xor_sync(0xFFFFFFFFu, szz, o);
      }
      if (t == 0) {
        const T x = (rJ - sy) / (cJ + szz);
        xjs[0] = x;
        u[pJ] = x;
      }
    }
    __syncthreads();
    xJ = xjs[0];
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int s = NT * q + t;
    const int p = sp[s];
    if (p >= 0) {
      const int sl = wslot(s);
      u[p] = sa[sl] + xJ * sb[sl];
    }
  }
}

// Wireframe lists: the same sequences with up to WJ3_MAX junctions each (the
// nodes that close rings; sequence w owns juncs[jofs[w] .. jofs[w + 1])),
// and the first sk.nskel CTAs of a launch each solve an edge skeleton.
template <typename T, int K, int W>
__global__ void __launch_bounds__(32 * W, sizeof(T) == 4 ? 32 / W : 1) seq3_multi_kernel(const WNode3 *__restrict__ nodes,
                                                      const WJunc3 *__restrict__ juncs, const int *__restrict__ jofs,
                                                      C6<T> cp, int nx1, int ny1, int nz1, T *__restrict__ u,
                                                      const T *__restrict__ f, const SkelArgs<T> sk) {
  pdl_trigger();
  if ((int)blockIdx.x < sk.nskel) {
    skel_cta<T>(sk.skel + blockIdx.x, sk.scr, sk.stride, cp.W, cp.E, cp.S, cp.N, cp.B, cp.T_, nx1, ny1, u, f);
    return;
  }
  constexpr int NT = 32 * W, N = NT * K;
  extern __shared__ __align__(16) unsigned char sm3[];
  T *sa = reinterpret_cast<T *>(sm3);
  T *sb = sa + N, *sc = sb + N, *sd = sc + N, *sz = sd + N;
  T *rep = sz + N;
  T *red = rep + 4 * NT;
  T *xjs = red + 8 * NT;             // junction values, then their rows' diagonal and rhs
  T *jcs = xjs + WJ3_MAX, *jrs = jcs + WJ3_MAX;
  int *sp = reinterpret_cast<int *>(jrs + WJ3_MAX);
  unsigned char *sj = reinterpret_cast<unsigned char *>(sp + N);  // junction of each slot's block
  const int t = threadIdx.x, lane = t & 31, cta = (int)blockIdx.x - sk.nskel;
  const size_t plane = (size_t)nx1 * ny1;
  const uint2 *nd = reinterpret_cast<const uint2 *>(nodes) + (size_t)cta * N;
  const int j0 = __ldg(jofs + cta), nj_list = __ldg(jofs + cta + 1) - j0;
  // checked builds: at most WJ3_MAX junctions per sequence (else none)
  const int nj = MG_OK_IF(nj_list >= 0 && nj_list <= WJ3_MAX) ? nj_list : 0;
  pdl_wait();  // u and f from here on
  // ---- 1. staging (thread t: nodes NT*q + t)
#pragma unroll
  for (int q = 0; q < K; ++q) {
    uint2 dsc = __ldg(nd + NT * q + t);
    // checked builds: a node must be an interior node (else its slot is unused)
    if ((dsc.y & WN3_VALID) && !MG_OK_IF((dsc.x & 1023u) >= 1u && (int)(dsc.x & 1023u) <= nx1 - 2 &&
                                          ((dsc.x >> 10) & 1023u) >= 1u && (int)((dsc.x >> 10) & 1023u) <= ny1 - 2 &&
                                          (dsc.x >> 20) >= 1u && (int)(dsc.x >> 20) <= nz1 - 2))
      dsc = make_uint2(0u, 0u);
    const unsigned fl = dsc.y;
    const bool valid = (fl & WN3_VALID) != 0u;
    const int i = (int)(dsc.x & 1023u), j = (int)((dsc.x >> 10) & 1023u), k = (int)(dsc.x >> 20);
    const unsigned pd = (fl & WN3_PRED) ? (fl & 7u) : 7u, sd_ = (fl & WN3_SUCC) ? ((fl >> 4) & 7u) : 7u,
                   jd = (fl & WN3_JUNC) ? ((fl >> 8) & 7u) : 7u;
    const size_t p = (size_t)k * plane + (size_t)j * nx1 + i;
    const size_t off[6] = {1, (size_t)0 - 1, (size_t)nx1, (size_t)0 - nx1, plane, (size_t)0 - plane};
    T a = T(0), c = T(0), z = T(0), b = T(0), r = valid ? __ldg(f + p) : T(0);
#pragma unroll
    for (unsigned d = 0; d < 6; ++d) {
      const T cd = cdir(cp, d, i, j, k);
      b -= cd;
      const bool outside = valid && d != pd && d != sd_ && d != jd;
      if (outside) r -= cd * u[p + off[d]];
      if (d == pd) a = cd;
      if (d == sd_) c = cd;
      if (d == jd) z = -cd;
    }
    const int s = NT * q + t, sl = wslot(s);
    sa[sl] = a;
    sc[sl] = c;
    sz[sl] = z;
    sb[sl] = valid ? b : T(1);
    sd[sl] = r;
    sp[s] = valid ? (int)p : -1;
    sj[s] = (unsigned char)((fl >> WN3_JSHIFT) & 31u);
  }
  // junction rows (thread e: junction e): diagonal and right-hand side
  if (t < nj) {
    const uint32_t Jijk = __ldg(&juncs[j0 + t].ijk), Jadirs = __ldg(&juncs[j0 + t].adirs);
    const int Jnatt = juncs[j0 + t].natt;
    int ji, jj, jk;
    unpack3(Jijk, ji, jj, jk);
    unsigned att = 0;
    for (int e = 0; e < Jnatt; ++e) att |= 1u << ((Jadirs >> (3 * e)) & 7u);
    const size_t pJ = (size_t)jk * plane + (size_t)jj * nx1 + ji;
    T rJ = __ldg(f + pJ), cJ = T(0);
    const size_t off[6] = {1, (size_t)0 - 1, (size_t)nx1, (size_t)0 - nx1, plane, (size_t)0 - plane};
#pragma unroll
    for (unsigned d = 0; d < 6; ++d) {
      const T cd = cdir(cp, d, ji, jj, jk);
      cJ -= cd;
      if (!(att & (1u << d))) rJ -= cd * u[pJ + off[d]];
    }
    jcs[t] = cJ;
    jrs[t] = rJ;
  }
  __syncthreads();

  // ---- 2. forward sweep per thread
  const int base = t * K;
  Sweep<T, K> sw;
  sw.run(base, sa, sb, sc, sd, sz);
  rep[t] = sw.Y0; rep[NT + t] = sw.Z0; rep[2 * NT + t] = sw.W0; rep[3 * NT + t] = sw.V0;
  __syncthreads();

  // ---- 3. separator rows, cyclic reduction through shared memory
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

  // ---- 5. junction values (lane e of warp 0: junction e), write back
  if (nj > 0) {
    if (t < 32) {
      T x = T(0);
      if (t < nj) {
        const uint32_t Jijk = __ldg(&juncs[j0 + t].ijk), Jadirs = __ldg(&juncs[j0 + t].adirs);
        const int Jnatt = juncs[j0 + t].natt;
        int ji, jj, jk;
        unpack3(Jijk, ji, jj, jk);
        T sy = T(0), szz = T(0);
        for (int e = 0; e < Jnatt; ++e) {
          const T kp = cdir(cp, (Jadirs >> (3 * e)) & 7u, ji, jj, jk);
          const int sl = wslot(juncs[j0 + t].as[e]);
          sy += kp * sa[sl];
          szz += kp * sb[sl];
        }
        x = (jrs[t] - sy) / (jcs[t] + szz);
        u[(size_t)jk * plane + (size_t)jj * nx1 + ji] = x;
      }
      xjs[lane] = x;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < K; ++q) {
    const int s = NT * q + t;
    const int p = sp[s];
    if (p >= 0) {
      const int sl = wslot(s);
      u[p] = nj > 0 ? sa[sl] + xjs[sj[s]] * sb[sl] : sa[sl];
    }
  }
}

template <typename T, int K, int W, bool MULTI>
constexpr size_t seq3_smem() {
  return MULTI ? (size_t)32 * W * K * (5 * sizeof(T) + sizeof(int) + 1) + sizeof(T) * (12 * 32 * W + 3 * WJ3_MAX)
               : (size_t)32 * W * K * (5 * sizeof(T) + sizeof(int)) + sizeof(T) * (12 * 32 * W + 2);
}

template <typename T, int K, int W, bool MULTI>
cudaError_t launch3_kw(const Grid3 &G, const Level3 &L, const WarpList3 &w, T *u, const T *f, cudaStream_t s) {
  count_launch(1);
  if constexpr (MULTI) {
    const SkelArgs<T> sk{w.skel, reinterpret_cast<T *>(G.skel_scr), G.skel_len, w.nskel};
    return launch_pdl(seq3_multi_kernel<T, K, W>, dim3(w.nskel + w.nwarp), dim3(32 * W),
                      seq3_smem<T, K, W, true>(), s, (const WNode3 *)w.node, (const WJunc3 *)w.junc,
                      (const int *)w.jofs, coefs3<T>(L), L.nx + 1, L.ny + 1, L.nz + 1, u, f, sk);
  } else {
    return launch_pdl(seq3_single_kernel<T, K, W>, dim3(w.nwarp), dim3(32 * W), seq3_smem<T, K, W, false>(), s,
                      (const WNode3 *)w.node, (const WJunc3 *)w.junc, coefs3<T>(L), L.nx + 1, L.ny + 1, L.nz + 1, u,
                      f);
  }
}
template <typename T, int K, bool MULTI>
cudaError_t launch3_k(const Grid3 &G, const Level3 &L, const WarpList3 &w, T *u, const T *f, cudaStream_t s) {
  switch (w.W) {
    case 1: return launch3_kw<T, K, 1, MULTI>(G, L, w, u, f, s);
    case 2: return launch3_kw<T, K, 2, MULTI>(G, L, w, u, f, s);
    case 4: return launch3_kw<T, K, 4, MULTI>(G, L, w, u, f, s);
    case 8: return launch3_kw<T, K, 8, MULTI>(G, L, w, u, f, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T, bool MULTI>
cudaError_t launch_warp3_t(const Grid3 &G, const Level3 &L, const WarpList3 &w, T *u, const T *f, cudaStream_t s) {
  if (w.nwarp + w.nskel == 0) return cudaSuccess;
  switch (w.K) {
    case 1: return launch3_k<T, 1, MULTI>(G, L, w, u, f, s);
    case 2: return launch3_k<T, 2, MULTI>(G, L, w, u, f, s);
    case 4: return launch3_k<T, 4, MULTI>(G, L, w, u, f, s);
    case 8: return launch3_k<T, 8, MULTI>(G, L, w, u, f, s);
    default: return cudaErrorInvalidValue;
  }
}
template <typename T, int K, int W, bool MULTI>
cudaError_t opt_in3_kw() {
  if constexpr (MULTI)
    return cudaFuncSetAttribute(seq3_multi_kernel<T, K, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)seq3_smem<T, K, W, true>());
  else
    return cudaFuncSetAttribute(seq3_single_kernel<T, K, W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)seq3_smem<T, K, W, false>());
}
template <typename T, int K, bool MULTI>
cudaError_t opt_in3() {
  cudaError_t e = opt_in3_kw<T, K, 1, MULTI>();
  if (e == cudaSuccess) e = opt_in3_kw<T, K, 2, MULTI>();
  if (e == cudaSuccess) e = opt_in3_kw<T, K, 4, MULTI>();
  if (e == cudaSuccess) e = opt_in3_kw<T, K, 8, MULTI>();
  return e;
}
template <bool MULTI>
cudaError_t prepare3_t() {
  cudaError_t e = opt_in3<float, 1, MULTI>();
  if (e == cudaSuccess) e = opt_in3<float, 2, MULTI>();
  if (e == cudaSuccess) e = opt_in3<float, 4, MULTI>();
  if (e == cudaSuccess) e = opt_in3<float, 8, MULTI>();
  if (e == cudaSuccess) e = opt_in3<double, 1, MULTI>();
  if (e == cudaSuccess) e = opt_in3<double, 2, MULTI>();
  if (e == cudaSuccess) e = opt_in3<double, 4, MULTI>();
  if (e == cudaSuccess) e = opt_in3<double, 8, MULTI>();
  return e;
}

}  // namespace

// the wireframe instances live in their own translation unit (grid3d_wf.cu)
template <typename T>
cudaError_t launch_seq3_multi(const Grid3 &G, const Level3 &L, const WarpList3 &w, T *u, const T *f, cudaStream_t s);
cudaError_t prepare_seq3_multi();

}  // namespace tmg
