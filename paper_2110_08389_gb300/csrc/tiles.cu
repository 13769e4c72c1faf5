// tiles.cu -- the tiled line path of tweedmg (sm_103a): one colour pass of
// tweed or zebra relaxation on a large level, as three kernels (see TileList
// in mg_internal.h for the data layout).
//
// Each block (Sec. 3) is solved exactly.  The solve is the paper's m-legged
// Thomas algorithm (Eq. mLThomas) organised in three levels:
//   tile_reduce  one lane per 32-node chunk of a leg: the chunk's right-hand
//                side (f minus the neighbours outside the block) and, by
//                eliminating its interior (partition method), two rows
//                coupling its first and last node to the neighbouring chunks;
//   tile_couple  one thread per leg: Thomas on those rows from the wall
//                towards the junction; the junction row fixes the junction
//                value; back-substitution gives every chunk's end values
//                (FP32 levels whose legs have at most 64 chunks: the
//                pivots of that Thomas come from setup, tile_couple_pc);
//   tile_expand  one lane per chunk: the interior by Thomas between the known
//                ends, written to u.
// Lanes of a tile are parallel legs at the same stretch of 32 positions, so
// the along-direction coefficients are the same for all lanes (broadcast
// loads); vertical tiles read and write u coalesced across lanes, horizontal
// tiles go through a per-warp shared-memory transpose.
#include <algorithm>

#include "device_util.cuh"
#include "tile_math.cuh"

namespace tmg {

namespace {

// warps (tiles) per CTA in tile_reduce / tile_expand (static shared memory
// per CTA stays below 48 KB)
template <typename T>
constexpr int TWv = sizeof(T) == 8 ? 2 : 4;

template <typename T>
struct CoefT {
  const T *W, *E, *S, *N;
};
template <typename T>
CoefT<T> coefs(const Level &L);
template <>
CoefT<double> coefs<double>(const Level &L) { return {L.W64, L.E64, L.S64, L.N64}; }
template <>
CoefT<float> coefs<float>(const Level &L) { return {L.W32, L.E32, L.S32, L.N32}; }

// Per-tile constants: run direction, step, which coefficient array is the
// predecessor / successor coupling along the run, and the lane's
// perpendicular coefficient sum.
template <typename T>
struct TileGeom {
  int base, step, vmax;
  bool xrun;
  const T *lo_arr, *hi_arr;
  __device__ __forceinline__ TileGeom(const TileDesc &td, const CoefT<T> &cp, int nx, int ny) {
    const int dir = td.dir;
    xrun = dir < 2;
    step = (dir == DIR_PX || dir == DIR_PY) ? 1 : -1;
    base = td.base;
    vmax = xrun ? nx : ny;
    if (xrun) { lo_arr = step > 0 ? cp.W : cp.E; hi_arr = step > 0 ? cp.E : cp.W; }
    else { lo_arr = step > 0 ? cp.S : cp.N; hi_arr = step > 0 ? cp.N : cp.S; }
  }
  __device__ __forceinline__ int v(int q) const { return base + q * step; }
};

// Positions of unused slots past the end of the axis (ragged last tiles of
// lines from wall to wall) are clamped into the coefficient arrays.
template <typename T>
__device__ __forceinline__ void stage_coefs(const TileGeom<T> &g, int lane, T (&co)[2][32]) {
  const int v = min(max(g.v(lane), 0), g.vmax);
  co[0][lane] = __ldg(g.lo_arr + v);
  co[1][lane] = __ldg(g.hi_arr + v);
  __syncwarp();
}

// YONLY (FP32 levels whose couple takes precomputed pivots): the rows'
// couplings are not formed, and only the pair (y_lo, y_hi) of each lane's
// chunk is written, as a 2-vector at tile * 32 + lane of `rows`.
template <typename T, bool YONLY = false>
__global__ void __launch_bounds__(32 * TWv<T>) tile_reduce(const TileDesc *__restrict__ tiles,
                                                       const TileLane *__restrict__ lanes, int ntile, CoefT<T> cp,
                                                       int nx, int ny, const T *__restrict__ u,
                                                       const T *__restrict__ f, TRow<T> *__restrict__ rows,
                                                       T *__restrict__ dscr) {
  const int nx1 = nx + 1;
  constexpr int TW = TWv<T>;
  __shared__ T tr[TW][32][33];
  __shared__ T cos[TW][2][32];
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int t = blockIdx.x * TW + warp;
  if (t >= ntile) return;
  const TileDesc td = tiles[t];
  const TileLane ln = lanes[(size_t)t * 32 + lane];
  const TileGeom<T> g(td, cp, nx, ny);
  const int fl = ln.flags;
  // checked builds: a lane's run must lie inside the level (else it is skipped)
  const int m = (ln.q1 == 0 || MG_OK_IF(ln.q1 <= CMAX && td.dir < 4 && ln.line >= 1 &&
                                        ln.line <= (g.xrun ? ny : nx) - 1 && g.v(0) >= 1 && g.v(0) <= g.vmax - 1 &&
                                        g.v(ln.q1 - 1) >= 1 && g.v(ln.q1 - 1) <= g.vmax - 1))
                    ? ln.q1
                    : 0;
  T d[CMAX];
  stage_coefs(g, lane, cos[warp]);
  const T(&co)[2][32] = cos[warp];
  pdl_wait();  // u, f and the scratch from here on

  // ---- right-hand sides.  Loads are unconditional (indices clamped into the
  // lane's run) so that all of them can be in flight at once; the wall terms
  // of a leg's first / last node are loaded before the loop.
  const int mq = m > 0 ? m - 1 : 0;  // last valid slot (clamp)
  if (!g.xrun) {
    // vertical tile: lane = column, slots = rows; coalesced across lanes
    const int i = m > 0 ? ln.line : 1;
    const T cw = __ldg(cp.W + i), ce = __ldg(cp.E + i);
    const int sv = g.step * nx1;
    const size_t p0 = (size_t)g.v(0) * nx1 + i, pm = (size_t)g.v(mq) * nx1 + i;
    const T wfirst = (fl & TL_FIRST) ? co[0][0] * u[p0 - sv] : T(0);
    const T wlast = (fl & TL_LAST_W) ? co[1][mq] * u[pm + sv] : T(0);
#pragma unroll
    for (int q = 0; q < CMAX; ++q) {
      const int qq = q < m ? q : mq;
      const size_t p = (size_t)g.v(qq) * nx1 + i;
      T r = f[p] - cw * u[p - 1] - ce * u[p + 1];
      if (q == 0) r -= wfirst;
      if (q == mq) r -= wlast;
      d[q] = r;
    }
  } else {
    // horizontal tile: for each lane's row in turn, all lanes load along it
    // (coalesced) and the values are transposed through shared memory
    const int q = lane;
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      const int jc = __shfl_sync(0xffffffffu, (int)ln.line, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      const int fc = __shfl_sync(0xffffffffu, fl, c);
      const int jj = mc > 0 ? jc : 1;
      const int qq = q < mc ? q : (mc > 0 ? mc - 1 : 0);
      const int i = g.v(qq);
      const size_t p = (size_t)jj * nx1 + i;
      T r = f[p] - __ldg(cp.S + jj) * u[p - nx1] - __ldg(cp.N + jj) * u[p + nx1];
      if (q == 0 && (fc & TL_FIRST)) r -= co[0][0] * u[p - g.step];
      if (q == mc - 1 && (fc & TL_LAST_W)) r -= co[1][q] * u[p + g.step];
      tr[warp][c][q] = r;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < CMAX; ++k) d[k] = tr[warp][lane][k];
  }
  if (m == 0) return;
  const T cross = g.xrun ? __ldg(cp.S + ln.line) + __ldg(cp.N + ln.line) : __ldg(cp.W + ln.line) + __ldg(cp.E + ln.line);

  // ---- the chunk's two reduced rows.  (A guard-free copy for full chunks,
  // as tile_expand has, doubled the registers here to 150 and was slower on
  // GB300: 79 vs 50 us per pass at 4097^2.)
  TRow<T> rlo, rhi;
  reduce_rows<T, false, !YONLY>(co, m, fl, cross, d, rlo, rhi);
  if constexpr (YONLY) {
    static_assert(sizeof(T) == 4, "the y-only rows are FP32");
    reinterpret_cast<float2 *>(rows)[(size_t)t * 32 + lane] = make_float2(rlo.y, rhi.y);
  } else {
    rows[((size_t)t * 32 + lane) * 2] = rlo;
    rows[((size_t)t * 32 + lane) * 2 + 1] = rhi;
  }
  if (m == CMAX) {
#pragma unroll
    for (int q = 0; q < CMAX; ++q) dscr[((size_t)t * 32 + q) * 32 + lane] = d[q];
  } else {
#pragma unroll
    for (int q = 0; q < CMAX; ++q)
      if (q < m) dscr[((size_t)t * 32 + q) * 32 + lane] = d[q];
  }
}

// One CTA per group: thread (leg l, lane b).  Thomas on the leg's reduced
// rows from the wall to the junction (normalised rows, so the pivot of row k
// is 1 - a_k c'_{k-1}); the block's junction row; back-substitution.  The
// forward sweep writes (c', d') to a separate array so that the row loads of
// later chunks do not wait for those stores.
template <typename T>
__global__ void __launch_bounds__(128) tile_couple(const BlockDesc *__restrict__ blocks, int ntile, size_t nn,
                                                   CoefT<T> cp, int nx1,
                                                   const TRow<T> *__restrict__ rows, T *cdp,
                                                   T *__restrict__ xscr, T *__restrict__ u, const T *__restrict__ f) {
  __shared__ T s_cp[4][32], s_dp[4][32], s_xj[32];
  pdl_trigger();
  const int l = threadIdx.x >> 5, b = threadIdx.x & 31;
  // the record's fields are read where they lie (a copy indexed by the
  // thread's leg would live in local memory)
  const BlockDesc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  int nleg = bp->nleg, junc = bp->junc;
  const int lane = bp->lane, ji = bp->ji, jj = bp->jj;
  const unsigned jdirs = bp->jdirs;
  // checked builds: a block's legs must lie in the tile list and its junction
  // inside the level (else the block is skipped)
  if (nleg > 0 || junc) {
    bool ok = nleg <= 4 && lane == b && (!junc || (ji >= 1 && ji <= nx1 - 2 && jj >= 1 && (size_t)(jj + 1) * nx1 < nn));
    for (int e = 0; e < nleg && ok; ++e)
      ok = (size_t)bp->leg_tile0[e] + (bp->leg_len[e] + CMAX - 1) / CMAX <= (size_t)ntile;
    if (!MG_OK_IF(ok)) { nleg = 0; junc = 0; }
  }
  const bool active = l < nleg;
  const int len = active ? bp->leg_len[l] : 0;
  const int nch = (len + CMAX - 1) / CMAX;
  const size_t t0 = active ? bp->leg_tile0[l] : 0;
  pdl_wait();  // the reduced rows, u and f from here on
  T cpv = T(0), dpv = T(0);
  constexpr int B = 16;  // chunks whose rows are loaded together
  for (int r0 = 0; r0 < nch; r0 += B) {
    TRow<T> lo[B], hi[B];
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (r0 + k < nch) {
        const size_t idx = ((t0 + r0 + k) * 32 + lane) * 2;
        lo[k] = rows[idx];
        hi[k] = rows[idx + 1];
      }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int r = r0 + k;
      if (r < nch) {
        const size_t idx = ((t0 + r) * 32 + lane) * 2;
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
  __syncthreads();
  if (l == 0 && junc) {
    const int i = ji, j = jj;
    const size_t p = (size_t)j * nx1 + i;
    unsigned att = 0;
    for (int e = 0; e < nleg; ++e) att |= 1u << ((jdirs >> (2 * e)) & 3);
    const T w = __ldg(cp.W + i), e_ = __ldg(cp.E + i), s = __ldg(cp.S + j), n = __ldg(cp.N + j);
    T num = f[p];
    if (!(att & 2u)) num -= w * u[p - 1];
    if (!(att & 1u)) num -= e_ * u[p + 1];
    if (!(att & 8u)) num -= s * u[p - nx1];
    if (!(att & 4u)) num -= n * u[p + nx1];
    T den = -((w + e_) + (s + n));
    for (int e = 0; e < nleg; ++e) {
      const int d = (jdirs >> (2 * e)) & 3;
      const T k = d == DIR_PX ? e_ : d == DIR_MX ? w : d == DIR_PY ? n : s;
      num -= k * s_dp[e][b];
      den -= k * s_cp[e][b];
    }
    const T x = num / den;
    u[p] = x;
    s_xj[b] = x;
  }
  __syncthreads();
  if (!active) return;
  T xn = junc ? s_xj[b] : T(0);
  // back-substitution, chunk by chunk towards the wall, B chunks per batch
  for (int r1 = nch - 1; r1 >= 0; r1 -= B) {
    T v[B][4];
#pragma unroll
    for (int k = 0; k < B; ++k)
      if (r1 - k >= 0) {
        const size_t idx = ((t0 + r1 - k) * 32 + lane) * 2;
#pragma unroll
        for (int e = 0; e < 4; ++e) v[k][e] = cdp[2 * idx + e];
      }
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int r = r1 - k;
      if (r >= 0) {
        const int mlen = min(CMAX, len - CMAX * r);
        T xhi = T(0);
        if (mlen >= 2) {
          xhi = v[k][3] - v[k][2] * xn;
          xn = xhi;
        }
        const T xlo = v[k][1] - v[k][0] * xn;
        xn = xlo;
        if (mlen < 2) xhi = xlo;
        xscr[((t0 + r) * 32 + lane) * 2] = xlo;
        xscr[((t0 + r) * 32 + lane) * 2 + 1] = xhi;
      }
    }
  }
}

// ---- FP32 couple with precomputed pivots.  In the forward sweep of
// tile_couple only d' depends on the right-hand sides: the pivots
// p = 1 / (1 - a c'_prev) and c' of every reduced row are fixed by the
// level's coefficients, so couple_consts_kernel computes them once at setup
// (from the rows tile_reduce gives for any right-hand side) and the sweep per
// pass is one dependent FMA per row, d' = y p - (a p) d'_prev.  A group's
// legs are carried by at most 64 threads (two legs per block; a block of
// three or four legs is alone in its group), so every chunk of every leg fits
// in shared memory at once: each thread copies its leg's constants with
// cp.async before waiting for the previous kernel, then the rows' right-hand
// sides in four copy groups, and eliminates each group as it lands; the
// back-substitution reads (c', d') from shared memory; the junction's
// neighbour values are loaded before the sweep.  Legs of at most
// TILE_PC_CHUNKS chunks.
constexpr int CCH = TILE_PC_CHUNKS, CSLOT = 64, CSEG = 4;
static_assert(CCH % CSEG == 0, "whole copy groups");
constexpr size_t COUPLE_PC_SMEM = (size_t)CCH * CSLOT * (16 + 16 + 8);

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Shared-memory slot of thread (leg l, lane b) in tile_couple_pc: legs 0 and
// 1 of the group's blocks, and legs 2 and 3 of a block alone in its group.
__device__ __forceinline__ int couple_slot(int l, int b) { return l < 2 ? l * 32 + b : (l - 2) * 32 + b + 1; }

// One CTA per group, thread (leg l, lane b) as in tile_couple: the forward
// sweep of the leg's reduced rows without right-hand sides.  Per lane and
// chunk: ca = (p_lo, a_lo p_lo, p_hi, a_hi p_hi), cb = (c'_lo, c'_hi).
__global__ void __launch_bounds__(128) couple_consts_kernel(const BlockDesc *__restrict__ blocks, int ntile,
                                                           const TRow<float> *__restrict__ rows,
                                                           float4 *__restrict__ ca, float2 *__restrict__ cb) {
  const int l = threadIdx.x >> 5, b = threadIdx.x & 31;
  const BlockDesc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  const int nleg = bp->nleg;
  if (l >= nleg || l >= 4 || bp->lane != b) return;
  const int len = bp->leg_len[l], nch = (len + CMAX - 1) / CMAX;
  const size_t t0 = bp->leg_tile0[l];
  if (!MG_OK_IF(t0 + nch <= (size_t)ntile)) return;
  float cpv = 0.f;
  for (int r = 0; r < nch; ++r) {
    const size_t i = (t0 + r) * 32 + b;
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

__global__ void __launch_bounds__(128) tile_couple_pc(const BlockDesc *__restrict__ blocks, int ntile, size_t nn,
                                                     CoefT<float> cp, int nx1, const float2 *__restrict__ ys,
                                                     const float4 *__restrict__ ca, const float2 *__restrict__ cb,
                                                     float *__restrict__ xscr, float *__restrict__ u,
                                                     const float *__restrict__ f) {
  extern __shared__ float4 couple_smem[];
  // chunk r of slot s: sA (p_lo, a_lo p_lo, p_hi, a_hi p_hi), sB (c'_lo,
  // c'_hi, d'_lo, d'_hi), sY (y_lo, y_hi) at [r * CSLOT + s]
  float4 *sA = couple_smem, *sB = couple_smem + CCH * CSLOT;
  float2 *sY = reinterpret_cast<float2 *>(couple_smem + 2 * CCH * CSLOT);
  __shared__ float s_cp[4][32], s_dp[4][32], s_xj[32];
  pdl_trigger();
  const int l = threadIdx.x >> 5, b = threadIdx.x & 31;
  const BlockDesc *bp = blocks + (size_t)blockIdx.x * 32 + b;
  int nleg = bp->nleg, junc = bp->junc;
  const int lane = bp->lane, ji = bp->ji, jj = bp->jj;
  const unsigned jdirs = bp->jdirs;
  // checked builds: a block's legs must lie in the tile list, within the
  // chunk cap, a block of more than two legs alone in its group (lane 0), and
  // its junction inside the level (else it is skipped)
  if (nleg > 0 || junc) {
    bool ok = nleg <= 4 && lane == b && (nleg <= 2 || b == 0) &&
              (!junc || (ji >= 1 && ji <= nx1 - 2 && jj >= 1 && (size_t)(jj + 1) * nx1 < nn));
    for (int e = 0; e < nleg && ok; ++e)
      ok = (size_t)bp->leg_tile0[e] + (bp->leg_len[e] + CMAX - 1) / CMAX <= (size_t)ntile &&
           (bp->leg_len[e] + CMAX - 1) / CMAX <= CCH;
    if (!MG_OK_IF(ok)) { nleg = 0; junc = 0; }
  }
  const bool active = l < nleg;
  const int len = active ? bp->leg_len[l] : 0;
  const int nch = (len + CMAX - 1) / CMAX;
  const size_t t0 = active ? bp->leg_tile0[l] : 0;
  const int sl = couple_slot(l, b);
  const size_t i0 = t0 * 32 + lane;  // lane-chunk index of chunk r: i0 + 32 r
  // the constants (setup data) while the previous kernel may still run
  for (int r = 0; r < nch; ++r) {
    cp_async16(&sA[r * CSLOT + sl], ca + i0 + 32 * (size_t)r);
    cp_async8(&sB[r * CSLOT + sl], cb + i0 + 32 * (size_t)r);
  }
  pdl_wait();  // the reduced rows, u and f from here on
  // the junction row's terms outside the block (loaded now, summed in the
  // order tile_couple sums them)
  float jnum = 0.f, jw = 0.f, je = 0.f, js = 0.f, jn = 0.f;
  if (l == 0 && junc) {
    const size_t p = (size_t)jj * nx1 + ji;
    unsigned att = 0;
    for (int e = 0; e < nleg; ++e) att |= 1u << ((jdirs >> (2 * e)) & 3);
    jw = __ldg(cp.W + ji); je = __ldg(cp.E + ji); js = __ldg(cp.S + jj); jn = __ldg(cp.N + jj);
    jnum = f[p];
    if (!(att & 2u)) jnum -= jw * u[p - 1];
    if (!(att & 1u)) jnum -= je * u[p + 1];
    if (!(att & 8u)) jnum -= js * u[p - nx1];
    if (!(att & 4u)) jnum -= jn * u[p + nx1];
  }
  // the rows' right-hand sides (y of the lo and hi row, tile_reduce<float,
  // true>), CSEG copy groups (the first also holds the constants)
#pragma unroll
  for (int g = 0; g < CSEG; ++g) {
    for (int r = g * (CCH / CSEG); r < min(nch, (g + 1) * (CCH / CSEG)); ++r)
      cp_async8(&sY[r * CSLOT + sl], ys + i0 + 32 * (size_t)r);
    cp_async_commit();
  }
  float dpv = 0.f;
#pragma unroll
  for (int g = 0; g < CSEG; ++g) {
    if (g == 0) cp_async_wait<CSEG - 1>();
    else if (g == 1) cp_async_wait<CSEG - 2>();
    else if (g == 2) cp_async_wait<CSEG - 3>();
    else cp_async_wait<0>();
    for (int r = g * (CCH / CSEG); r < min(nch, (g + 1) * (CCH / CSEG)); ++r) {
      const float4 A = sA[r * CSLOT + sl];
      const float2 y = sY[r * CSLOT + sl];
      dpv = fmaf(-A.y, dpv, y.x * A.x);
      const float dlo = dpv;
      if (min(CMAX, len - CMAX * r) >= 2) dpv = fmaf(-A.w, dpv, y.y * A.z);
      *reinterpret_cast<float2 *>(&sB[r * CSLOT + sl].z) = make_float2(dlo, dpv);
    }
  }
  // c' of the leg's last row: c'_hi of its last chunk (= c'_lo for a chunk of one node)
  s_cp[l][b] = nch > 0 ? sB[(nch - 1) * CSLOT + sl].y : 0.f;
  s_dp[l][b] = dpv;
  __syncthreads();
  if (l == 0 && junc) {
    float num = jnum, den = -((jw + je) + (js + jn));
    for (int e = 0; e < nleg; ++e) {
      const int d = (jdirs >> (2 * e)) & 3;
      const float k = d == DIR_PX ? je : d == DIR_MX ? jw : d == DIR_PY ? jn : js;
      num -= k * s_dp[e][b];
      den -= k * s_cp[e][b];
    }
    const float xj = num / den;
    u[(size_t)jj * nx1 + ji] = xj;
    s_xj[b] = xj;
  }
  __syncthreads();
  if (!active) return;
  float xn = junc ? s_xj[b] : 0.f;
  // back-substitution, chunk by chunk towards the wall
  for (int r = nch - 1; r >= 0; --r) {
    const float4 v = sB[r * CSLOT + sl];  // (c'_lo, c'_hi, d'_lo, d'_hi)
    const int mlen = min(CMAX, len - CMAX * r);
    float xhi = 0.f;
    if (mlen >= 2) {
      xhi = v.w - v.y * xn;
      xn = xhi;
    }
    const float xlo = v.z - v.x * xn;
    xn = xlo;
    if (mlen < 2) xhi = xlo;
    xscr[(i0 + 32 * (size_t)r) * 2] = xlo;
    xscr[(i0 + 32 * (size_t)r) * 2 + 1] = xhi;
  }
}

template <typename T>
__global__ void __launch_bounds__(32 * TWv<T>) tile_expand(const TileDesc *__restrict__ tiles,
                                                       const TileLane *__restrict__ lanes, int ntile, CoefT<T> cp,
                                                       int nx, int ny, const T *__restrict__ dscr,
                                                       const T *__restrict__ xscr, T *__restrict__ u) {
  const int nx1 = nx + 1;
  // per lane one row of x (tr) and of the Thomas multipliers c' (cs) in
  // shared memory, stride 33 (conflict-free both per lane and per slot)
  constexpr int TW = TWv<T>;
  __shared__ T tr[TW][32][33];
  __shared__ T cs[TW][32][33];
  __shared__ T cos[TW][2][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // tiles in the reverse order of tile_reduce: the u lines it read last are
  // the likeliest to still be in L2 for these partial-sector writes
  pdl_trigger();
  const int t = ntile - 1 - (blockIdx.x * TW + warp);
  if (t < 0) return;
  const TileDesc td = tiles[t];
  const TileLane ln = lanes[(size_t)t * 32 + lane];
  const TileGeom<T> g(td, cp, nx, ny);
  const int fl = ln.flags;
  // checked builds: a lane's run must lie inside the level (else it is skipped)
  const int m = (ln.q1 == 0 || MG_OK_IF(ln.q1 <= CMAX && td.dir < 4 && ln.line >= 1 &&
                                        ln.line <= (g.xrun ? ny : nx) - 1 && g.v(0) >= 1 && g.v(0) <= g.vmax - 1 &&
                                        g.v(ln.q1 - 1) >= 1 && g.v(ln.q1 - 1) <= g.vmax - 1))
                    ? ln.q1
                    : 0;
  stage_coefs(g, lane, cos[warp]);
  const T(&co)[2][32] = cos[warp];
  pdl_wait();  // the scratch and u from here on
  T *x = tr[warp][lane], *cpv = cs[warp][lane];
  if (m > 0) {
    const T cross = g.xrun ? __ldg(cp.S + ln.line) + __ldg(cp.N + ln.line)
                           : __ldg(cp.W + ln.line) + __ldg(cp.E + ln.line);
    const T xlo = xscr[((size_t)t * 32 + lane) * 2], xhi = xscr[((size_t)t * 32 + lane) * 2 + 1];
    const T *dl = dscr + (size_t)t * 32 * 32 + lane;  // d of slot q at dl[32 q]
    T dv[CMAX];
#pragma unroll
    for (int q = 0; q < CMAX; ++q) dv[q] = dl[32 * (q < m ? q : m - 1)];  // all loads in flight
    // FP32 full chunks (all but a leg's last) without guards: 26 vs 30 us
    // per pass at 4097^2 on GB300, with the same registers (in FP64 the copy
    // raised them from 94 to 151)
    if (sizeof(T) == 4 && m == CMAX) expand_rows<T, true>(co, m, fl, cross, dv, xlo, xhi, x, cpv);
    else expand_rows<T, false>(co, m, fl, cross, dv, xlo, xhi, x, cpv);
  }
  __syncwarp();
  if (!g.xrun) {
    const int i = ln.line;
#pragma unroll 8
    for (int q = 0; q < CMAX; ++q)
      if (q < m) u[(size_t)g.v(q) * nx1 + i] = x[q];
  } else {
    const int q = lane;
    const int i = g.v(q);
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      const int jc = __shfl_sync(0xffffffffu, (int)ln.line, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      if (q < mc) u[(size_t)jc * nx1 + i] = tr[warp][c][q];
    }
  }
}

}  // namespace

// the two constant arrays of a tile list (TileList.cconst)
static float4 *couple_ca(const TileList &tl) { return static_cast<float4 *>(tl.cconst); }
static float2 *couple_cb(const TileList &tl) {
  return reinterpret_cast<float2 *>(static_cast<char *>(tl.cconst) + (size_t)tl.ntile * 32 * sizeof(float4));
}

cudaError_t prepare_tile_kernels() {
  return cudaFuncSetAttribute(tile_couple_pc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)COUPLE_PC_SMEM);
}

cudaError_t setup_couple_consts(Grid &g) {
  // the rows' couplings do not depend on u and f: reduce zero arrays
  float *z = static_cast<float *>(g.e32);
  cudaError_t e = cudaMemset(z, 0, g.lev[0].nn * sizeof(float));
  TRow<float> *rows = static_cast<TRow<float> *>(g.tile_rows);
  float *dscr = static_cast<float *>(g.tile_d);
  for (int l = 0; l < g.nlev && e == cudaSuccess; ++l)
    for (int wl = 0; wl < WL_COUNT && e == cudaSuccess; ++wl)
      for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
        const Level &L = g.lev[l];
        const TileList &tl = L.tl[wl][c];
        if (!tl.cconst) continue;
        constexpr int TW = TWv<float>;
        tile_reduce<float><<<(tl.ntile + TW - 1) / TW, 32 * TW>>>(tl.tile, tl.lane, tl.ntile, coefs<float>(L), L.nx,
                                                                 L.ny, z, z, rows, dscr);
        couple_consts_kernel<<<tl.ngroup, 128>>>(tl.block, tl.ntile, rows, couple_ca(tl), couple_cb(tl));
        count_launch(2);
        e = cudaGetLastError();
      }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

template <typename T>
cudaError_t launch_tile_pass(const Grid &g, const Level &L, const TileList &tl, T *u, const T *f, cudaStream_t s,
                             cudaEvent_t *ev) {
  if (tl.ntile == 0 && tl.nblock == 0) return cudaSuccess;
  TRow<T> *rows = static_cast<TRow<T> *>(g.tile_rows);
  T *cdp = reinterpret_cast<T *>(static_cast<char *>(g.tile_rows) + g.tile_cap * 32 * 2 * sizeof(TRow<double>));
  T *dscr = static_cast<T *>(g.tile_d), *xscr = static_cast<T *>(g.tile_x);
  const CoefT<T> cp = coefs<T>(L);
  const int nx1 = L.nx + 1;
  constexpr int TW = TWv<T>;
  const int ctas = (tl.ntile + TW - 1) / TW;
  if (ev) cudaEventRecord(ev[0], s);
  cudaError_t e = cudaSuccess;
  if (tl.ntile > 0) {
    if constexpr (sizeof(T) == 4) {
      if (tl.cconst)
        e = launch_pdl(tile_reduce<float, true>, dim3(ctas), dim3(32 * TW), 0, s, (const TileDesc *)tl.tile,
                       (const TileLane *)tl.lane, tl.ntile, cp, L.nx, L.ny, u, f, rows, dscr);
      else
        e = launch_pdl(tile_reduce<float, false>, dim3(ctas), dim3(32 * TW), 0, s, (const TileDesc *)tl.tile,
                       (const TileLane *)tl.lane, tl.ntile, cp, L.nx, L.ny, u, f, rows, dscr);
    } else {
      e = launch_pdl(tile_reduce<T>, dim3(ctas), dim3(32 * TW), 0, s, (const TileDesc *)tl.tile,
                     (const TileLane *)tl.lane, tl.ntile, cp, L.nx, L.ny, u, f, rows, dscr);
    }
  }
  if (ev) cudaEventRecord(ev[1], s);
  if (e == cudaSuccess) {
    if (sizeof(T) == 4 && tl.cconst)
      e = launch_pdl(tile_couple_pc, dim3(tl.ngroup), dim3(128), COUPLE_PC_SMEM, s, (const BlockDesc *)tl.block,
                     tl.ntile, L.nn, coefs<float>(L), nx1, (const float2 *)rows, couple_ca(tl), couple_cb(tl),
                     (float *)xscr, (float *)u, (const float *)f);
    else
      e = launch_pdl(tile_couple<T>, dim3(tl.ngroup), dim3(128), 0, s, (const BlockDesc *)tl.block, tl.ntile, L.nn,
                     cp, nx1, (const TRow<T> *)rows, cdp, xscr, u, f);
  }
  if (ev) cudaEventRecord(ev[2], s);
  if (e == cudaSuccess && tl.ntile > 0)
    e = launch_ex(true, tile_expand<T>, dim3(ctas), dim3(32 * TW), 0, s, (const TileDesc *)tl.tile,
                   (const TileLane *)tl.lane, tl.ntile, cp, L.nx, L.ny, (const T *)dscr, (const T *)xscr, u);
  if (ev) cudaEventRecord(ev[3], s);
  count_launch(tl.ntile > 0 ? 3 : 1);
  return e;
}
template cudaError_t launch_tile_pass<double>(const Grid &, const Level &, const TileList &, double *, const double *,
                                              cudaStream_t, cudaEvent_t *);
template cudaError_t launch_tile_pass<float>(const Grid &, const Level &, const TileList &, float *, const float *,
                                             cudaStream_t, cudaEvent_t *);

}  // namespace tmg
