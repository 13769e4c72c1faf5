// tiles3.cu -- the 3D tiled tweed path of tweedmg (sm_103a): one colour pass
// of 3D tweed relaxation (Sec. 7) as three kernels, the 2D tiled path's
// organisation (tiles.cu) on the blocks of a 3D level (layout: Tile3List in
// mg_internal.h, built by tile3_host.h).
//
// Each block is solved exactly by the m-legged Thomas algorithm (Eq.
// mLThomas), in three levels:
//   tile3_reduce  one lane per 32-node chunk of a leg: the chunk's right-hand
//                 side (f minus the four neighbours across the run, and the
//                 known node before the leg or after a free end) and its two
//                 reduced rows (partition method, tile_math.cuh);
//   tile3_couple  per leg (up to six), its chunks found through the leg's
//                 slot list: Thomas on those rows towards the junction; the
//                 junction row with its six neighbours fixes the junction
//                 value; back-substitution gives every chunk's end values
//                 (FP32: tile3_couple_pc, with the pivots from setup, after
//                 a tile3_reduce that forms only the rows' right-hand sides);
//   tile3_expand  one lane per chunk: the interior by Thomas between the
//                 known ends, written to u.
// Lanes of a tile are chunks of parallel legs over the same 32 positions, so
// the along-run coefficients are shared (staged once per warp).  Runs along
// y and z read and write u with the lanes' x coordinates adjacent (coalesced
// where the layout could put consecutive blocks side by side); runs along x
// go through a per-warp shared-memory transpose, one lane's run per step.
#include <algorithm>

#include "tile3_host.h"
#include "tile_math.cuh"

namespace tmg {

namespace {

template <typename T>
constexpr int TW3 = sizeof(T) == 8 ? 2 : 4;  // warps (tiles) per CTA in reduce / expand

template <typename T>
struct Coef3T {
  const T *c[6];  // W, E, S, N, B, T
};
template <typename T>
Coef3T<T> coef3t(const Level3 &L);
template <>
Coef3T<double> coef3t<double>(const Level3 &L) {
  return {{L.c64[0], L.c64[1], L.c64[2], L.c64[3], L.c64[4], L.c64[5]}};
}
template <>
Coef3T<float> coef3t<float>(const Level3 &L) {
  return {{L.c32[0], L.c32[1], L.c32[2], L.c32[3], L.c32[4], L.c32[5]}};
}

// Per tile: run axis (0 x, 1 y, 2 z), step, the along-run coefficient arrays
// on the predecessor and successor side, and the level's strides.
template <typename T>
struct Geo3 {
  int base, step, vmax, axis;
  long long nx1, plane, sv;  // sv: offset of the next node along the run
  const T *lo_arr, *hi_arr;
  __device__ __forceinline__ Geo3(const Tile3Desc &td, const Coef3T<T> &cp, int nx, int ny, int nz) {
    axis = td.dir >> 1;
    step = (td.dir & 1) ? -1 : 1;
    base = td.base;
    vmax = axis == 0 ? nx : axis == 1 ? ny : nz;
    nx1 = nx + 1;
    plane = nx1 * (ny + 1);
    sv = (axis == 0 ? 1 : axis == 1 ? nx1 : plane) * step;
    // coupling to the lower / upper neighbour (constant indices: a runtime
    // index into the parameter array would put it in local memory)
    const T *neg = axis == 0 ? cp.c[0] : axis == 1 ? cp.c[2] : cp.c[4];
    const T *pos = axis == 0 ? cp.c[1] : axis == 1 ? cp.c[3] : cp.c[5];
    lo_arr = step > 0 ? neg : pos;
    hi_arr = step > 0 ? pos : neg;
  }
  __device__ __forceinline__ int v(int q) const { return base + q * step; }
  // node of slot q of the run with fixed coordinates (c1, c2)
  __device__ __forceinline__ long long node(int q, int c1, int c2) const {
    const long long w = v(q);
    return axis == 0 ? c2 * plane + c1 * nx1 + w : axis == 1 ? c2 * plane + w * nx1 + c1 : w * plane + c2 * nx1 + c1;
  }
  // the four neighbours across the run: offsets and coefficients
  __device__ __forceinline__ void across(const Coef3T<T> &cp, int c1, int c2, long long &sa, long long &sb, T &am,
                                         T &ap, T &bm, T &bp) const {
    if (axis == 0) {  // y (c1 = j) and z (c2 = k)
      sa = nx1; sb = plane;
      am = __ldg(cp.c[2] + c1); ap = __ldg(cp.c[3] + c1); bm = __ldg(cp.c[4] + c2); bp = __ldg(cp.c[5] + c2);
    } else if (axis == 1) {  // x (c1 = i) and z (c2 = k)
      sa = 1; sb = plane;
      am = __ldg(cp.c[0] + c1); ap = __ldg(cp.c[1] + c1); bm = __ldg(cp.c[4] + c2); bp = __ldg(cp.c[5] + c2);
    } else {  // x (c1 = i) and y (c2 = j)
      sa = 1; sb = nx1;
      am = __ldg(cp.c[0] + c1); ap = __ldg(cp.c[1] + c1); bm = __ldg(cp.c[2] + c2); bp = __ldg(cp.c[3] + c2);
    }
  }
  // the lane's run stays inside the level (checked builds)
  __device__ __forceinline__ bool inside(int m, int c1, int c2, int nx, int ny, int nz) const {
    const int m1 = axis == 0 ? ny : nx, m2 = axis == 2 ? ny : nz;
    return m <= CMAX && c1 >= 1 && c1 <= m1 - 1 && c2 >= 1 && c2 <= m2 - 1 && v(0) >= 1 && v(0) <= vmax - 1 &&
           v(m - 1) >= 1 && v(m - 1) <= vmax - 1;
  }
};

template <typename T>
__device__ __forceinline__ void stage_coefs3(const Geo3<T> &g, int lane, T (&co)[2][32]) {
  const int v = min(max(g.v(lane), 0), g.vmax);
  co[0][lane] = __ldg(g.lo_arr + v);
  co[1][lane] = __ldg(g.hi_arr + v);
  __syncwarp();
}

// YONLY (FP32 lists whose couple takes setup-time pivots): the rows'
// couplings are not formed; only (y_lo, y_hi) of each lane slot is written,
// as a 2-vector at tile * 32 + lane of `rows`.
template <typename T, bool YONLY = false>
__global__ void __launch_bounds__(32 * TW3<T>) tile3_reduce(const Tile3Desc *__restrict__ tiles,
                                                        const Tile3Lane *__restrict__ lanes, int ntile,
                                                        Coef3T<T> cp, int nx, int ny, int nz,
                                                        const T *__restrict__ u, const T *__restrict__ f,
                                                        TRow<T> *__restrict__ rows, T *__restrict__ dscr) {
  constexpr int TW = TW3<T>;
  __shared__ T tr[TW][32][33];
  __shared__ T cos[TW][2][32];
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * TW + warp;
  if (t >= ntile) return;
  const Tile3Desc td = tiles[t];
  const Tile3Lane ln = lanes[(size_t)t * 32 + lane];
  const Geo3<T> g(td, cp, nx, ny, nz);
  const int fl = ln.flags;
  // checked builds: a lane's run must lie inside the level (else it is skipped)
  const int m = (ln.q1 == 0 || MG_OK_IF(td.dir < 6 && g.inside(ln.q1, ln.c1, ln.c2, nx, ny, nz))) ? ln.q1 : 0;
  T d[CMAX];
  stage_coefs3(g, lane, cos[warp]);
  const T(&co)[2][32] = cos[warp];
  pdl_wait();  // u and f from here on
  const int mq = m > 0 ? m - 1 : 0;
  // unused lanes read a valid node and write nothing
  const int c1 = m > 0 ? ln.c1 : 1, c2 = m > 0 ? ln.c2 : 1;
  long long sa, sb;
  T am, ap, bm, bp;
  g.across(cp, c1, c2, sa, sb, am, ap, bm, bp);
  if (g.axis != 0) {
    // runs along y or z: each lane reads its own run, the lanes side by side
    // in x; slots past the lane's chunk load nothing (the layout packs ragged
    // chunks side by side, so clamped loads would touch other rows)
    const long long p0 = g.node(0, c1, c2), pm = g.node(mq, c1, c2);
    const T wfirst = (fl & TL_FIRST) ? co[0][0] * u[p0 - g.sv] : T(0);
    const T wlast = (fl & TL_LAST_W) ? co[1][mq] * u[pm + g.sv] : T(0);
#pragma unroll
    for (int q = 0; q < CMAX; ++q) {
      T r = T(0);
      if (q < m) {
        const long long p = g.node(q, c1, c2);
        r = f[p] - am * u[p - sa] - ap * u[p + sa] - bm * u[p - sb] - bp * u[p + sb];
        if (q == 0) r -= wfirst;
        if (q == mq) r -= wlast;
      }
      d[q] = r;
    }
  } else {
    // runs along x: for each lane's run in turn, all lanes read along it
    // (coalesced) and the values are transposed through shared memory; the
    // run's row offset and its four coefficients across (S, N of its y, B,
    // T of its z: the lane's own am, ap, bm, bp) come from its lane by
    // shuffle, and slots past its chunk load nothing
    const int q = lane;
    const long long rb = (long long)c2 * g.plane + (long long)c1 * g.nx1;
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      const long long rbc = __shfl_sync(0xffffffffu, rb, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      const int fc = __shfl_sync(0xffffffffu, fl, c);
      const T amc = __shfl_sync(0xffffffffu, am, c), apc = __shfl_sync(0xffffffffu, ap, c);
      const T bmc = __shfl_sync(0xffffffffu, bm, c), bpc = __shfl_sync(0xffffffffu, bp, c);
      T r = T(0);
      if (q < mc) {
        const long long p = rbc + g.v(q);
        r = f[p] - amc * u[p - g.nx1] - apc * u[p + g.nx1] - bmc * u[p - g.plane] - bpc * u[p + g.plane];
        if (q == 0 && (fc & TL_FIRST)) r -= co[0][0] * u[p - g.sv];
        if (q == mc - 1 && (fc & TL_LAST_W)) r -= co[1][q] * u[p + g.sv];
      }
      tr[warp][c][q] = r;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < CMAX; ++k) d[k] = tr[warp][lane][k];
  }
  if (m == 0) return;
  const T cross = (am + ap) + (bm + bp);
  TRow<T> rlo, rhi;
  reduce_rows<T, false, !YONLY>(co, m, fl, cross, d, rlo, rhi);
  if constexpr (YONLY) {
    static_assert(sizeof(T) == 4, "the y-only rows are FP32");
    reinterpret_cast<float2 *>(rows)[(size_t)t * 32 + lane] = make_float2(rlo.y, rhi.y);
  } else {
    rows[((size_t)t * 32 + lane) * 2] = rlo;
    rows[((size_t)t * 32 + lane) * 2 + 1] = rhi;
  }
#pragma unroll
  for (int q = 0; q < CMAX; ++q)
    if (q < m) dscr[((size_t)t * 32 + q) * 32 + lane] = d[q];
}

// One CTA of two warps per group: lane b is block b, and warp w takes legs
// w, w + 2, w + 4 of it in turn (most blocks have two legs; the stars'
// groups take longer but run beside the others, in the same launch).  Per
// leg: Thomas on its reduced rows from its first chunk towards the junction
// (normalised rows, so the pivot of row k is 1 - a_k c'_{k-1}); then the
// block's junction row with the substitutions x_last = d' - c' x_junction
// of its legs; then back-substitution to every chunk's end values.
template <typename T>
__global__ void __launch_bounds__(64) tile3_couple(const Block3Desc *__restrict__ blocks,
                                                   const uint32_t *__restrict__ slots, int nslot, int ntile,
                                                   Coef3T<T> cp, int nx, int ny, int nz,
                                                   const TRow<T> *__restrict__ rows, T *cdp, T *__restrict__ xscr,
                                                   T *__restrict__ u, const T *__restrict__ f) {
  __shared__ T s_cp[6][32], s_dp[6][32], s_xj[32];
  pdl_trigger();
  const int w = threadIdx.x >> 5, b = threadIdx.x & 31;
  // the record's fields are read where they lie (a copy indexed by the
  // leg would live in local memory)
  const Block3Desc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  int nleg = bp->nleg, junc = bp->junc;
  const unsigned jdirs = bp->jdirs;
  const int ji = bp->ji, jj = bp->jj, jk = bp->jk;
  // checked builds: a block's chunk slots must lie in the lists and its
  // junction inside the level (else the block is skipped)
  if (nleg > 0 || junc) {
    bool ok = nleg <= 6 && (!junc || (ji >= 1 && ji <= nx - 1 && jj >= 1 && jj <= ny - 1 && jk >= 1 && jk <= nz - 1));
    for (int e = 0; e < nleg && ok; ++e) {
      const int nc = (bp->leg_len[e] + CMAX - 1) / CMAX;
      ok = (size_t)bp->leg_slot0[e] + nc <= (size_t)nslot;
      for (int r = 0; r < nc && ok; ++r) ok = slots[bp->leg_slot0[e] + r] < 32u * ntile;
    }
    if (!MG_OK_IF(ok)) { nleg = 0; junc = 0; }
  }
  pdl_wait();  // the reduced rows, u and f from here on
  constexpr int B = 4;  // chunks whose rows are loaded together (legs of at most a few chunks)
  for (int l = w; l < nleg; l += 2) {
    const int len = bp->leg_len[l];
    const int nch = (len + CMAX - 1) / CMAX;
    const uint32_t *sl = slots + bp->leg_slot0[l];
    T cpv = T(0), dpv = T(0);
    for (int r0 = 0; r0 < nch; r0 += B) {
      TRow<T> lo[B], hi[B];
#pragma unroll
      for (int k = 0; k < B; ++k)
        if (r0 + k < nch) {
          const size_t idx = (size_t)__ldg(sl + r0 + k) * 2;
          lo[k] = rows[idx];
          hi[k] = rows[idx + 1];
        }
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int r = r0 + k;
        if (r < nch) {
          const size_t idx = (size_t)__ldg(sl + r) * 2;
          const int mlen = min(CMAX, len - CMAX * r);
          T den = rcp_t(T(1) - lo[k].a * cpv);
          cpv = lo[k].c * den;
          dpv = (lo[k].y - lo[k].a * dpv) * den;
          cdp[2 * idx] = cpv; cdp[2 * idx + 1] = dpv;
          if (mlen >= 2) {
            den = rcp_t(T(1) - hi[k].a * cpv);
            cpv = hi[k].c * den;
            dpv = (hi[k].y - hi[k].a * dpv) * den;
            cdp[2 * idx + 2] = cpv; cdp[2 * idx + 3] = dpv;
          }
        }
      }
    }
    s_cp[l][b] = cpv;
    s_dp[l][b] = dpv;
  }
  __syncthreads();
  if (w == 0 && junc) {
    const long long nx1 = nx + 1, plane = nx1 * (ny + 1);
    const long long p = jk * plane + jj * nx1 + ji;
    unsigned att = 0;
    for (int e = 0; e < nleg; ++e) att |= 1u << ((jdirs >> (3 * e)) & 7u);
    const T cw = __ldg(cp.c[0] + ji), ce = __ldg(cp.c[1] + ji), cs = __ldg(cp.c[2] + jj), cn = __ldg(cp.c[3] + jj),
            cb = __ldg(cp.c[4] + jk), ct = __ldg(cp.c[5] + jk);
    T num = f[p];
    if (!(att & 1u)) num -= ce * u[p + 1];
    if (!(att & 2u)) num -= cw * u[p - 1];
    if (!(att & 4u)) num -= cn * u[p + nx1];
    if (!(att & 8u)) num -= cs * u[p - nx1];
    if (!(att & 16u)) num -= ct * u[p + plane];
    if (!(att & 32u)) num -= cb * u[p - plane];
    T den = -(((cw + ce) + (cs + cn)) + (cb + ct));
    for (int e = 0; e < nleg; ++e) {
      const unsigned d = (jdirs >> (3 * e)) & 7u;
      const T kc = d == 0 ? ce : d == 1 ? cw : d == 2 ? cn : d == 3 ? cs : d == 4 ? ct : cb;
      num -= kc * s_dp[e][b];
      den -= kc * s_cp[e][b];
    }
    const T x = num / den;
    u[p] = x;
    s_xj[b] = x;
  }
  __syncthreads();
  for (int l = w; l < nleg; l += 2) {
    const int len = bp->leg_len[l];
    const int nch = (len + CMAX - 1) / CMAX;
    const uint32_t *sl = slots + bp->leg_slot0[l];
    T xn = junc ? s_xj[b] : T(0);
    for (int r = nch - 1; r >= 0; --r) {
      const size_t idx = (size_t)__ldg(sl + r) * 2;
      const int mlen = min(CMAX, len - CMAX * r);
      T xhi = T(0);
      if (mlen >= 2) {
        xhi = cdp[2 * idx + 3] - cdp[2 * idx + 2] * xn;
        xn = xhi;
      }
      const T xlo = cdp[2 * idx + 1] - cdp[2 * idx] * xn;
      xn = xlo;
      if (mlen < 2) xhi = xlo;
      xscr[idx] = xlo;
      xscr[idx + 1] = xhi;
    }
  }
}

// ---- FP32 couple with setup-time pivots, as tiles.cu's tile_couple_pc:
// the pivots p = 1 / (1 - a c'_prev), a p and c' of every reduced row depend
// only on the coefficients, so couple3_consts_kernel forms them once from the
// rows tile3_reduce gives for any right-hand side; per pass the forward sweep
// is d' = y p - (a p) d'_prev on the rows' right-hand sides alone.
__global__ void __launch_bounds__(64) couple3_consts_kernel(const Block3Desc *__restrict__ blocks,
                                                            const uint32_t *__restrict__ slots,
                                                            const TRow<float> *__restrict__ rows,
                                                            float4 *__restrict__ ca, float2 *__restrict__ cb) {
  const int w = threadIdx.x >> 5, b = threadIdx.x & 31;
  const Block3Desc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  const int nleg = min((int)bp->nleg, 6);
  for (int l = w; l < nleg; l += 2) {
    const int len = bp->leg_len[l];
    const int nch = (len + CMAX - 1) / CMAX;
    const uint32_t *sl = slots + bp->leg_slot0[l];
    float cpv = 0.f;
    for (int r = 0; r < nch; ++r) {
      const size_t i = sl[r];
      const TRow<float> lo = rows[2 * i], hi = rows[2 * i + 1];
      float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
      float2 B;
      float p = rcp_t(1.f - lo.a * cpv);
      cpv = lo.c * p;
      A.x = p; A.y = lo.a * p; B.x = cpv; B.y = cpv;
      if (min(CMAX, len - CMAX * r) >= 2) {
        p = rcp_t(1.f - hi.a * cpv);
        cpv = hi.c * p;
        A.z = p; A.w = hi.a * p; B.y = cpv;
      }
      ca[i] = A;
      cb[i] = B;
    }
  }
}

__global__ void __launch_bounds__(64) tile3_couple_pc(const Block3Desc *__restrict__ blocks,
                                                      const uint32_t *__restrict__ slots, int nslot, int ntile,
                                                      Coef3T<float> cp, int nx, int ny, int nz,
                                                      const float2 *__restrict__ ys, const float4 *__restrict__ ca,
                                                      const float2 *__restrict__ cb, float *cdp,
                                                      float *__restrict__ xscr, float *__restrict__ u,
                                                      const float *__restrict__ f) {
  __shared__ float s_cp[6][32], s_dp[6][32], s_xj[32];
  pdl_trigger();
  const int w = threadIdx.x >> 5, b = threadIdx.x & 31;
  const Block3Desc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  int nleg = bp->nleg, junc = bp->junc;
  const unsigned jdirs = bp->jdirs;
  const int ji = bp->ji, jj = bp->jj, jk = bp->jk;
  // checked builds: a block's chunk slots must lie in the lists and its
  // junction inside the level (else the block is skipped)
  if (nleg > 0 || junc) {
    bool ok = nleg <= 6 && (!junc || (ji >= 1 && ji <= nx - 1 && jj >= 1 && jj <= ny - 1 && jk >= 1 && jk <= nz - 1));
    for (int e = 0; e < nleg && ok; ++e) {
      const int nc = (bp->leg_len[e] + CMAX - 1) / CMAX;
      ok = (size_t)bp->leg_slot0[e] + nc <= (size_t)nslot;
      for (int r = 0; r < nc && ok; ++r) ok = slots[bp->leg_slot0[e] + r] < 32u * ntile;
    }
    if (!MG_OK_IF(ok)) { nleg = 0; junc = 0; }
  }
  pdl_wait();  // the rows' right-hand sides, u and f from here on
  constexpr int B = 4;  // chunks whose loads are issued together (legs of at most a few chunks)
  for (int l = w; l < nleg; l += 2) {
    const int len = bp->leg_len[l];
    const int nch = (len + CMAX - 1) / CMAX;
    const uint32_t *sl = slots + bp->leg_slot0[l];
    float cpv = 0.f, dpv = 0.f;
    for (int r0 = 0; r0 < nch; r0 += B) {
      float2 y[B], c2[B];
      float4 A[B];
#pragma unroll
      for (int k = 0; k < B; ++k)
        if (r0 + k < nch) {
          const size_t i = __ldg(sl + r0 + k);
          y[k] = ys[i];
          A[k] = ca[i];
          c2[k] = cb[i];
        }
#pragma unroll
      for (int k = 0; k < B; ++k) {
        const int r = r0 + k;
        if (r < nch) {
          const size_t idx = (size_t)__ldg(sl + r) * 2;
          const int mlen = min(CMAX, len - CMAX * r);
          dpv = fmaf(-A[k].y, dpv, y[k].x * A[k].x);
          cpv = c2[k].x;
          cdp[2 * idx] = cpv; cdp[2 * idx + 1] = dpv;
          if (mlen >= 2) {
            dpv = fmaf(-A[k].w, dpv, y[k].y * A[k].z);
            cpv = c2[k].y;
            cdp[2 * idx + 2] = cpv; cdp[2 * idx + 3] = dpv;
          }
        }
      }
    }
    s_cp[l][b] = cpv;
    s_dp[l][b] = dpv;
  }
  __syncthreads();
  if (w == 0 && junc) {
    const long long nx1 = nx + 1, plane = nx1 * (ny + 1);
    const long long p = jk * plane + jj * nx1 + ji;
    unsigned att = 0;
    for (int e = 0; e < nleg; ++e) att |= 1u << ((jdirs >> (3 * e)) & 7u);
    const float cw = __ldg(cp.c[0] + ji), ce = __ldg(cp.c[1] + ji), cs = __ldg(cp.c[2] + jj),
                cn = __ldg(cp.c[3] + jj), cbo = __ldg(cp.c[4] + jk), ct = __ldg(cp.c[5] + jk);
    float num = f[p];
    if (!(att & 1u)) num -= ce * u[p + 1];
    if (!(att & 2u)) num -= cw * u[p - 1];
    if (!(att & 4u)) num -= cn * u[p + nx1];
    if (!(att & 8u)) num -= cs * u[p - nx1];
    if (!(att & 16u)) num -= ct * u[p + plane];
    if (!(att & 32u)) num -= cbo * u[p - plane];
    float den = -(((cw + ce) + (cs + cn)) + (cbo + ct));
    for (int e = 0; e < nleg; ++e) {
      const unsigned d = (jdirs >> (3 * e)) & 7u;
      const float kc = d == 0 ? ce : d == 1 ? cw : d == 2 ? cn : d == 3 ? cs : d == 4 ? ct : cbo;
      num -= kc * s_dp[e][b];
      den -= kc * s_cp[e][b];
    }
    const float x = num / den;
    u[p] = x;
    s_xj[b] = x;
  }
  __syncthreads();
  for (int l = w; l < nleg; l += 2) {
    const int len = bp->leg_len[l];
    const int nch = (len + CMAX - 1) / CMAX;
    const uint32_t *sl = slots + bp->leg_slot0[l];
    float xn = junc ? s_xj[b] : 0.f;
    for (int r = nch - 1; r >= 0; --r) {
      const size_t idx = (size_t)__ldg(sl + r) * 2;
      const int mlen = min(CMAX, len - CMAX * r);
      float xhi = 0.f;
      if (mlen >= 2) {
        xhi = cdp[2 * idx + 3] - cdp[2 * idx + 2] * xn;
        xn = xhi;
      }
      const float xlo = cdp[2 * idx + 1] - cdp[2 * idx] * xn;
      xn = xlo;
      if (mlen < 2) xhi = xlo;
      xscr[idx] = xlo;
      xscr[idx + 1] = xhi;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * TW3<T>) tile3_expand(const Tile3Desc *__restrict__ tiles,
                                                        const Tile3Lane *__restrict__ lanes, int ntile,
                                                        Coef3T<T> cp, int nx, int ny, int nz,
                                                        const T *__restrict__ dscr, const T *__restrict__ xscr,
                                                        T *__restrict__ u) {
  constexpr int TW = TW3<T>;
  __shared__ T tr[TW][32][33];
  __shared__ T cs[TW][32][33];
  __shared__ T cos[TW][2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tiles in the reverse order of tile3_reduce (the u it read last is the
  // likeliest to be in L2)
  pdl_trigger();
  const int t = ntile - 1 - (blockIdx.x * TW + warp);
  if (t < 0) return;
  const Tile3Desc td = tiles[t];
  const Tile3Lane ln = lanes[(size_t)t * 32 + lane];
  const Geo3<T> g(td, cp, nx, ny, nz);
  const int fl = ln.flags;
  const int m = (ln.q1 == 0 || MG_OK_IF(td.dir < 6 && g.inside(ln.q1, ln.c1, ln.c2, nx, ny, nz))) ? ln.q1 : 0;
  stage_coefs3(g, lane, cos[warp]);
  const T(&co)[2][32] = cos[warp];
  pdl_wait();  // the scratch and u from here on
  T *x = tr[warp][lane], *cpv = cs[warp][lane];
  const int c1 = m > 0 ? ln.c1 : 1, c2 = m > 0 ? ln.c2 : 1;
  if (m > 0) {
    long long sa, sb;
    T am, ap, bm, bp;
    g.across(cp, c1, c2, sa, sb, am, ap, bm, bp);
    const T cross = (am + ap) + (bm + bp);
    const T xlo = xscr[((size_t)t * 32 + lane) * 2], xhi = xscr[((size_t)t * 32 + lane) * 2 + 1];
    const T *dl = dscr + (size_t)t * 32 * 32 + lane;  // d of slot q at dl[32 q]
    T dv[CMAX];
#pragma unroll
    for (int q = 0; q < CMAX; ++q) dv[q] = q < m ? dl[32 * q] : T(0);
    if (sizeof(T) == 4 && m == CMAX) expand_rows<T, true>(co, m, fl, cross, dv, xlo, xhi, x, cpv);
    else expand_rows<T, false>(co, m, fl, cross, dv, xlo, xhi, x, cpv);
  }
  __syncwarp();
  if (g.axis != 0) {
#pragma unroll 8
    for (int q = 0; q < CMAX; ++q)
      if (q < m) u[g.node(q, c1, c2)] = x[q];
  } else {
    const int q = lane;
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      const int jc = __shfl_sync(0xffffffffu, c1, c);
      const int kc = __shfl_sync(0xffffffffu, c2, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      if (q < mc) u[g.node(q, jc, kc)] = tr[warp][c][q];
    }
  }
}

}  // namespace

mg_status build_tiles3(Grid &g, Level3 &L, const std::vector<HBlock3> &tweed_blocks, bool *ok) {
  *ok = false;
  tile3::Tile3Host th[2];
  for (int c = 0; c < 2; ++c)
    if (!tile3::layout(L, tweed_blocks, c, th[c])) return MG_OK;
  for (int c = 0; c < 2; ++c) {
    Tile3List &T = L.t3[c];
    const size_t s0 = th[c].tiles.size() * sizeof(Tile3Desc), s1 = th[c].lanes.size() * sizeof(Tile3Lane),
                 s2 = th[c].blocks.size() * sizeof(Block3Desc), s3 = th[c].slots.size() * sizeof(uint32_t);
    const size_t o1 = (s0 + 255) / 256 * 256, o2 = o1 + (s1 + 255) / 256 * 256, o3 = o2 + (s2 + 255) / 256 * 256;
    const size_t o4 = o3 + (s3 + 255) / 256 * 256;
    const size_t s4 = (g.prec_mask & 2) ? th[c].tiles.size() * 32 * (16 + 8) : 0;  // couple constants
    char *mem = nullptr;
    if (cudaMalloc(&mem, o4 + s4 + 16) != cudaSuccess) return MG_ERR_ALLOC;
    T.mem = mem;
    T.cconst = s4 ? mem + o4 : nullptr;
    T.tile = reinterpret_cast<Tile3Desc *>(mem);
    T.lane = reinterpret_cast<Tile3Lane *>(mem + o1);
    T.block = reinterpret_cast<Block3Desc *>(mem + o2);
    T.slot = reinterpret_cast<uint32_t *>(mem + o3);
    if ((s0 && cudaMemcpy(T.tile, th[c].tiles.data(), s0, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (s1 && cudaMemcpy(T.lane, th[c].lanes.data(), s1, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (s2 && cudaMemcpy(T.block, th[c].blocks.data(), s2, cudaMemcpyHostToDevice) != cudaSuccess) ||
        (s3 && cudaMemcpy(T.slot, th[c].slots.data(), s3, cudaMemcpyHostToDevice) != cudaSuccess))
      return MG_ERR_CUDA;
    T.ntile = (int)th[c].tiles.size();
    T.nblock = (int)th[c].blocks.size();
    T.nslot = (int)th[c].slots.size();
    T.ngroup = th[c].ngroup;
    T.max_leg_chunks = th[c].max_chunks;
    g.tile_cap = std::max(g.tile_cap, (size_t)T.ntile);
  }
  *ok = true;
  return MG_OK;
}

// the two constant arrays of a 3D tile list (Tile3List.cconst)
static float4 *couple3_ca(const Tile3List &tl) { return static_cast<float4 *>(tl.cconst); }
static float2 *couple3_cb(const Tile3List &tl) {
  return reinterpret_cast<float2 *>(static_cast<char *>(tl.cconst) + (size_t)tl.ntile * 32 * sizeof(float4));
}

cudaError_t setup_couple_consts3(Grid &g) {
  // the rows' couplings do not depend on u and f: reduce zero arrays
  float *z = static_cast<float *>(g.e32);
  cudaError_t e = cudaMemset(z, 0, g.g3->lev[0].nn * sizeof(float));
  TRow<float> *rows = static_cast<TRow<float> *>(g.tile_rows);
  float *dscr = static_cast<float *>(g.tile_d);
  for (Level3 &L : g.g3->lev)
    for (int c = 0; c < 2 && e == cudaSuccess && L.t3_ok; ++c) {
      const Tile3List &tl = L.t3[c];
      if (!tl.cconst || tl.ntile == 0) continue;
      constexpr int TW = TW3<float>;
      tile3_reduce<float><<<(tl.ntile + TW - 1) / TW, 32 * TW>>>(tl.tile, tl.lane, tl.ntile, coef3t<float>(L), L.nx,
                                                                 L.ny, L.nz, z, z, rows, dscr);
      if (tl.ngroup > 0)
        couple3_consts_kernel<<<tl.ngroup, 64>>>(tl.block, tl.slot, rows, couple3_ca(tl), couple3_cb(tl));
      count_launch(tl.ngroup > 0 ? 2 : 1);
      e = cudaGetLastError();
    }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

template <typename T>
cudaError_t launch_tile3_pass(const Grid &g, const Level3 &L, const Tile3List &tl, T *u, const T *f,
                              cudaStream_t s) {
  if (tl.ntile == 0 && tl.nblock == 0) return cudaSuccess;
  TRow<T> *rows = static_cast<TRow<T> *>(g.tile_rows);
  T *cdp = reinterpret_cast<T *>(static_cast<char *>(g.tile_rows) + g.tile_cap * 32 * 2 * sizeof(TRow<double>));
  T *dscr = static_cast<T *>(g.tile_d), *xscr = static_cast<T *>(g.tile_x);
  const Coef3T<T> cp = coef3t<T>(L);
  constexpr int TW = TW3<T>;
  const int ctas = (tl.ntile + TW - 1) / TW;
  cudaError_t e = cudaSuccess;
  const bool pc = sizeof(T) == 4 && tl.cconst;  // FP32 with setup-time pivots
  if (tl.ntile > 0) {
    if (pc)
      e = launch_pdl(tile3_reduce<float, true>, dim3(ctas), dim3(32 * TW), 0, s, (const Tile3Desc *)tl.tile,
                     (const Tile3Lane *)tl.lane, tl.ntile, coef3t<float>(L), L.nx, L.ny, L.nz, (const float *)u,
                     (const float *)f, (TRow<float> *)rows, (float *)dscr);
    else
      e = launch_pdl(tile3_reduce<T>, dim3(ctas), dim3(32 * TW), 0, s, (const Tile3Desc *)tl.tile,
                     (const Tile3Lane *)tl.lane, tl.ntile, cp, L.nx, L.ny, L.nz, (const T *)u, f, rows, dscr);
  }
  if (e == cudaSuccess && tl.ngroup > 0) {
    if (pc)
      e = launch_pdl(tile3_couple_pc, dim3(tl.ngroup), dim3(64), 0, s, (const Block3Desc *)tl.block,
                     (const uint32_t *)tl.slot, tl.nslot, tl.ntile, coef3t<float>(L), L.nx, L.ny, L.nz,
                     (const float2 *)rows, couple3_ca(tl), couple3_cb(tl), (float *)cdp, (float *)xscr, (float *)u,
                     (const float *)f);
    else
      e = launch_pdl(tile3_couple<T>, dim3(tl.ngroup), dim3(64), 0, s, (const Block3Desc *)tl.block,
                     (const uint32_t *)tl.slot, tl.nslot, tl.ntile, cp, L.nx, L.ny, L.nz, (const TRow<T> *)rows,
                     cdp, xscr, u, f);
  }
  if (e == cudaSuccess && tl.ntile > 0)
    e = launch_pdl(tile3_expand<T>, dim3(ctas), dim3(32 * TW), 0, s, (const Tile3Desc *)tl.tile,
                   (const Tile3Lane *)tl.lane, tl.ntile, cp, L.nx, L.ny, L.nz, (const T *)dscr, (const T *)xscr, u);
  count_launch((tl.ntile > 0 ? 2 : 0) + (tl.ngroup > 0 ? 1 : 0));
  return e;
}
template cudaError_t launch_tile3_pass<double>(const Grid &, const Level3 &, const Tile3List &, double *,
                                               const double *, cudaStream_t);
template cudaError_t launch_tile3_pass<float>(const Grid &, const Level3 &, const Tile3List &, float *, const float *,
                                              cudaStream_t);

}  // namespace tmg
