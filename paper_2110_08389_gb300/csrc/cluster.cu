// cluster.cu -- the cluster pass of tweedmg (sm_103a): one FP32 colour pass
// of tweed or zebra relaxation on a large level in ONE kernel, each group of
// blocks on the CTAs of a thread-block cluster, every intermediate in shared
// memory (see ClusterPlan in mg_internal.h for the layout and the phases).
//
// Each block (Sec. 3) is solved exactly by the m-legged Thomas algorithm
// (Eq. mLThomas) in the arrangement of the tiled path: every 32-node chunk
// of a leg is reduced to two rows (partition method, cluster_math.h), each
// leg is eliminated on those rows from the wall to the junction, the junction
// row gives the junction value, back-substitution gives the chunks' end
// values, and each chunk's interior follows by Thomas between them.  The
// rows and end values stay in the shared memory of the CTA that holds the
// chunk; the CTA that solves a leg reads and writes them there through
// distributed shared memory.  Global memory sees only the reads of u and f
// and the writes of u: no scratch.
//
// Synchronisation: __syncthreads inside a CTA and two cluster barriers
// (arrive.release / wait.acquire), both reached by every thread of every CTA
// (no early exit, no spin-wait): the first makes every CTA's rows visible to
// the cluster, the second the chunk end values; no CTA touches another's
// shared memory after the second, so each may then finish and exit.
#include <cooperative_groups.h>

#include "cluster_math.h"
#include "device_util.cuh"

namespace tmg {

namespace {

namespace cg = cooperative_groups;
using clmath::Row;

constexpr int NT = CL_WARPS * 32;
constexpr int SLOTS = CL_TILES * 32;
constexpr int DP = 33;  // pitch of a slot row of D: conflict-free by lane and by slot
constexpr int LEG_BATCH = 16;  // rows of a leg loaded together in the leg solve

struct Smem {
  float D[CL_TILES][32][DP];  // per tile, [slot q][lane]: right-hand sides, then the solution
  float4 row[SLOTS][2];       // per chunk: its lo and hi rows (a, c, y)
  float2 cd[CL_LEGROWS];      // (c', d') of every row of the legs this CTA solves
  float2 chx[SLOTS];          // per chunk: values of its first and last node
  float co[CL_TILES][2][32];  // regular tiles: coefficients to the predecessor / successor of each slot
  float lcp[4][32], ldp[4][32], xj[32];
  uint8_t mlen[SLOTS];        // nodes of each chunk (0: unused lane)
};

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;" ::: "memory"); }

// Run geometry of a tile.
struct Geo {
  bool xrun;
  int step, vmax;
  const float *lo_arr, *hi_arr;
  __device__ __forceinline__ Geo(int dir, const Coefs<float> &cp, int nx, int ny) {
    xrun = dir < 2;
    step = (dir == DIR_PX || dir == DIR_PY) ? 1 : -1;
    vmax = xrun ? nx : ny;
    if (xrun) { lo_arr = step > 0 ? cp.W : cp.E; hi_arr = step > 0 ? cp.E : cp.W; }
    else { lo_arr = step > 0 ? cp.S : cp.N; hi_arr = step > 0 ? cp.N : cp.S; }
  }
  __device__ __forceinline__ int clampv(int v) const { return min(max(v, 0), vmax); }
};

// Coefficients of a chunk's slots: staged in shared memory (regular tiles,
// the same 32 positions for every lane) or read per lane (compact tiles).
struct CoSm {
  const float *lo_, *hi_;
  __device__ __forceinline__ float lo(int q) const { return lo_[q]; }
  __device__ __forceinline__ float hi(int q) const { return hi_[q]; }
};
struct CoGl {
  const Geo *g;
  int base;
  __device__ __forceinline__ float lo(int q) const { return __ldg(g->lo_arr + g->clampv(base + q * g->step)); }
  __device__ __forceinline__ float hi(int q) const { return __ldg(g->hi_arr + g->clampv(base + q * g->step)); }
};
struct DReg {
  const float *d;
  __device__ __forceinline__ float operator()(int q) const { return d[q]; }
};
struct XReg {
  float *x;
  __device__ __forceinline__ float get(int q) const { return x[q]; }
  __device__ __forceinline__ void set(int q, float v) { x[q] = v; }
};
struct Args {
  const CTile *tile;
  const CLane *lane;
  const CCta *cta;
  const CSeg *seg;
  const CBlock *block;
  const CChain *chain;
  Coefs<float> cp;
  int nx, ny;
  float *u;
  const float *f;
};

// Phase 1 for one tile (one warp): right-hand sides into D, reduced rows.
template <bool COMPACT>
__device__ __forceinline__ void tile_rows(Smem &sm, const Args &a, int t, const CTile &td, const CLane &ln,
                                          int lane) {
  const int nx1 = a.nx + 1;
  const Geo g(td.dir, a.cp, a.nx, a.ny);
  const int fl = ln.flags;
  // checked builds: a lane's run must lie inside the level (else it is skipped)
  const int base = COMPACT ? (int)ln.cbase : (int)td.base;
  const int m = (ln.q1 == 0 || MG_OK_IF(ln.q1 <= 32 && ln.line >= 1 && ln.line <= (g.xrun ? a.ny : a.nx) - 1 &&
                                        base >= 1 && base <= g.vmax - 1 && base + (ln.q1 - 1) * g.step >= 1 &&
                                        base + (ln.q1 - 1) * g.step <= g.vmax - 1))
                    ? ln.q1
                    : 0;
  if (!COMPACT) {
    const int v = g.clampv(base + lane * g.step);
    sm.co[t][0][lane] = __ldg(g.lo_arr + v);
    sm.co[t][1][lane] = __ldg(g.hi_arr + v);
    __syncwarp();
  }
  const float *u = a.u, *f = a.f;
  float d[32];
  const int mq = m > 0 ? m - 1 : 0;
  if (!g.xrun) {
    // runs along y: lane = column; regular tiles read rows coalesced across lanes
    const int i = m > 0 ? ln.line : 1;
    const float cw = __ldg(a.cp.W + i), ce = __ldg(a.cp.E + i);
    const int sv = g.step * nx1;
    const size_t p0 = (size_t)g.clampv(base) * nx1 + i, pm = (size_t)g.clampv(base + mq * g.step) * nx1 + i;
    float wfirst = 0.0f, wlast = 0.0f;
    if (fl & TL_FIRST) {
      const float lo0 = COMPACT ? __ldg(g.lo_arr + g.clampv(base)) : sm.co[t][0][0];
      wfirst = lo0 * __ldg(u + p0 - sv);
    }
    if (fl & TL_LAST_W) {
      const float hiq = COMPACT ? __ldg(g.hi_arr + g.clampv(base + mq * g.step)) : sm.co[t][1][mq];
      wlast = hiq * __ldg(u + pm + sv);
    }
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      const int qq = q < m ? q : mq;
      const size_t p = (size_t)g.clampv(base + qq * g.step) * nx1 + i;
      float r = __ldg(f + p) - cw * __ldg(u + p - 1) - ce * __ldg(u + p + 1);
      if (q == 0) r -= wfirst;
      if (q == mq) r -= wlast;
      d[q] = r;
      sm.D[t][q][lane] = r;
    }
  } else {
    // runs along x: for each lane's row in turn all lanes read along it
    // (coalesced) and store transposed into D
    const int q = lane;
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      const int jc = __shfl_sync(0xffffffffu, (int)ln.line, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      const int fc = __shfl_sync(0xffffffffu, fl, c);
      const int bc = COMPACT ? __shfl_sync(0xffffffffu, base, c) : base;
      const int jj = mc > 0 ? jc : 1;
      const int qq = q < mc ? q : (mc > 0 ? mc - 1 : 0);
      const int i = g.clampv(bc + qq * g.step);
      const size_t p = (size_t)jj * nx1 + i;
      float r = __ldg(f + p) - __ldg(a.cp.S + jj) * __ldg(u + p - nx1) - __ldg(a.cp.N + jj) * __ldg(u + p + nx1);
      if (q == 0 && (fc & TL_FIRST)) {
        const float lo0 = COMPACT ? __ldg(g.lo_arr + g.clampv(bc)) : sm.co[t][0][0];
        r -= lo0 * __ldg(u + p - g.step);
      }
      if (q == mc - 1 && (fc & TL_LAST_W)) {
        const float hiq = COMPACT ? __ldg(g.hi_arr + i) : sm.co[t][1][q];
        r -= hiq * __ldg(u + p + g.step);
      }
      sm.D[t][q][c] = r;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) d[k] = sm.D[t][k][lane];
  }
  const int slot = t * 32 + lane;
  sm.mlen[slot] = (uint8_t)m;
  if (m == 0) return;
  const float cross = g.xrun ? __ldg(a.cp.S + ln.line) + __ldg(a.cp.N + ln.line)
                             : __ldg(a.cp.W + ln.line) + __ldg(a.cp.E + ln.line);
  Row<float> rlo, rhi;
  const bool first = fl & TL_FIRST, last_w = fl & TL_LAST_W;
  if (COMPACT) clmath::chunk_reduce<float>(CoGl{&g, base}, m, first, last_w, cross, DReg{d}, rlo, rhi);
  else clmath::chunk_reduce<float>(CoSm{sm.co[t][0], sm.co[t][1]}, m, first, last_w, cross, DReg{d}, rlo, rhi);
  sm.row[slot][0] = make_float4(rlo.a, rlo.c, rlo.y, 0.0f);
  sm.row[slot][1] = make_float4(rhi.a, rhi.c, rhi.y, 0.0f);
}

// Phase 3 for one tile (one warp): chunk interiors from D and the chunk end
// values, written back to u.
template <bool COMPACT>
__device__ __forceinline__ void tile_expand(Smem &sm, const Args &a, int t, const CTile &td, const CLane &ln,
                                            int lane) {
  const int nx1 = a.nx + 1;
  const Geo g(td.dir, a.cp, a.nx, a.ny);
  const int fl = ln.flags;
  // checked builds: a lane's run must lie inside the level (else it is skipped)
  const int base = COMPACT ? (int)ln.cbase : (int)td.base;
  const int m = (ln.q1 == 0 || MG_OK_IF(ln.q1 <= 32 && ln.line >= 1 && ln.line <= (g.xrun ? a.ny : a.nx) - 1 &&
                                        base >= 1 && base <= g.vmax - 1 && base + (ln.q1 - 1) * g.step >= 1 &&
                                        base + (ln.q1 - 1) * g.step <= g.vmax - 1))
                    ? ln.q1
                    : 0;
  const int slot = t * 32 + lane;
  if (m > 0) {
    float d[32], x[32], cpv[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) d[q] = sm.D[t][q][lane];
    const float cross = g.xrun ? __ldg(a.cp.S + ln.line) + __ldg(a.cp.N + ln.line)
                               : __ldg(a.cp.W + ln.line) + __ldg(a.cp.E + ln.line);
    const float2 ends = sm.chx[slot];
    const bool first = fl & TL_FIRST, last_w = fl & TL_LAST_W;
    XReg xs{x};
    if (COMPACT)
      clmath::chunk_expand<float>(CoGl{&g, base}, m, first, last_w, cross, DReg{d}, ends.x, ends.y, xs, cpv);
    else
      clmath::chunk_expand<float>(CoSm{sm.co[t][0], sm.co[t][1]}, m, first, last_w, cross, DReg{d}, ends.x, ends.y,
                                  xs, cpv);
#pragma unroll
    for (int q = 0; q < 32; ++q)
      if (q < m) sm.D[t][q][lane] = x[q];
  }
  __syncwarp();
  float *u = a.u;
  if (!g.xrun) {
    const int i = ln.line;
#pragma unroll 8
    for (int q = 0; q < 32; ++q)
      if (q < m) u[(size_t)(base + q * g.step) * nx1 + i] = sm.D[t][q][lane];
  } else {
    const int q = lane;
#pragma unroll 4
    for (int c = 0; c < 32; ++c) {
      const int jc = __shfl_sync(0xffffffffu, (int)ln.line, c);
      const int mc = __shfl_sync(0xffffffffu, m, c);
      const int bc = COMPACT ? __shfl_sync(0xffffffffu, base, c) : base;
      if (q < mc) u[(size_t)jc * nx1 + bc + q * g.step] = sm.D[t][q][c];
    }
  }
}

__global__ void __launch_bounds__(NT, 2) cluster_pass_kernel(const Args a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rank = (int)cluster.block_rank();
  const CCta cd = a.cta[blockIdx.x];

  // ---- phase 1: chunk right-hand sides and reduced rows
  for (int t = warp; t < cd.ntile; t += CL_WARPS) {
    const CTile td = a.tile[cd.tile0 + t];
    const CLane ln = a.lane[(size_t)(cd.tile0 + t) * 32 + lane];
    if (td.kind == CT_COMPACT) tile_rows<true>(sm, a, t, td, ln, lane);
    else tile_rows<false>(sm, a, t, td, ln, lane);
  }
  __syncthreads();
  cluster_arrive();
  cluster_wait();
  // ---- phase 2: this CTA's blocks of the group (b = grank, grank + ngr, ...):
  // thread (l, bi) eliminates leg l of block bi * ngr + grank on its chunk
  // rows, wherever in the cluster they lie
  if (cd.group >= 0) {
    __shared__ const float4 (*prow[CL_CTAS])[2];
    __shared__ float2 *pchx[CL_CTAS];
    __shared__ int pseg0[CL_CTAS];
    if (tid < CL_CTAS) {
      prow[tid] = cluster.map_shared_rank(sm.row, tid);
      pchx[tid] = cluster.map_shared_rank(sm.chx, tid);
      pseg0[tid] = a.cta[blockIdx.x - rank + tid].seg0;
    }
    __syncthreads();
    const int l = tid >> 5, bi = tid & 31, b = bi * cd.ngr + cd.grank;
    CBlock bd;
    bd.nleg = 0; bd.junc = 0;
    if (b < 32) bd = a.block[(size_t)cd.group * 32 + b];
    const bool act = l < 4 && l < bd.nleg;
    CChain ch;
    ch.nseg = 0;
    if (act) {
      ch = a.chain[(size_t)cd.group * 128 + l * 32 + b];
      // checked builds: the leg's segments must be CTAs of this cluster and
      // its rows must fit the (c', d') store (else the leg is skipped)
      bool ok = ch.nseg <= CL_MAXSEG && (int)ch.roff + ch.nrow <= CL_LEGROWS;
      for (int s = 0; s < CL_MAXSEG && ok; ++s) ok = s >= ch.nseg || ch.rank[s] < CL_CTAS;
      if (!MG_OK_IF(ok)) ch.nseg = 0;
    }
    // forward: normalised rows, pivot 1 - a c'_prev.  The rows are read where
    // they lie (remote loads only); (c', d') go to this CTA's own store.
    float cpv = 0.0f, dpv = 0.0f;
    int kr = ch.roff;
    for (int s = 0; s < ch.nseg; ++s) {
      const int rk = ch.rank[s];
      CSeg sg = a.seg[pseg0[rk] + ch.slot[s]];
      // checked builds: the segment's chunks must be slots of its CTA
      if (!MG_OK_IF(sg.nchunk >= 1 && sg.slot0 + (sg.nchunk - 1) * sg.stride < SLOTS && sg.one <= 1)) sg.nchunk = 0;
      const int R = 2 * sg.nchunk - sg.one;
      const float4(*rows)[2] = prow[rk];
      for (int k0 = 0; k0 < R; k0 += LEG_BATCH) {
        float4 v[LEG_BATCH];
#pragma unroll
        for (int e = 0; e < LEG_BATCH; ++e)
          if (k0 + e < R) v[e] = rows[sg.slot0 + ((k0 + e) >> 1) * sg.stride][(k0 + e) & 1];
#pragma unroll
        for (int e = 0; e < LEG_BATCH; ++e)
          if (k0 + e < R) {
            const float den = clmath::rcp(1.0f - v[e].x * cpv);
            cpv = v[e].y * den;
            dpv = (v[e].z - v[e].x * dpv) * den;
            sm.cd[kr + k0 + e] = make_float2(cpv, dpv);
          }
      }
      kr += R;
    }
    if (act) {
      sm.lcp[l][bi] = cpv;
      sm.ldp[l][bi] = dpv;
    }
    __syncthreads();
    // the junction row of Eq. mLThomas with each leg's last unknown
    // x_last = d' - c' x_junction substituted (checked builds: the junction
    // must lie inside the level, else the block's junction is skipped)
    if (l == 0 && bd.junc && MG_OK_IF(bd.ji >= 1 && bd.ji <= a.nx - 1 && bd.jj >= 1 && bd.jj <= a.ny - 1)) {
      const int nx1 = a.nx + 1, i = bd.ji, j = bd.jj;
      const size_t p = (size_t)j * nx1 + i;
      unsigned att = 0;
      for (int e = 0; e < bd.nleg; ++e) att |= 1u << ((bd.jdirs >> (2 * e)) & 3);
      const float w = __ldg(a.cp.W + i), e_ = __ldg(a.cp.E + i), sc = __ldg(a.cp.S + j), n = __ldg(a.cp.N + j);
      float num = __ldg(a.f + p);
      if (!(att & 2u)) num -= w * __ldg(a.u + p - 1);
      if (!(att & 1u)) num -= e_ * __ldg(a.u + p + 1);
      if (!(att & 8u)) num -= sc * __ldg(a.u + p - nx1);
      if (!(att & 4u)) num -= n * __ldg(a.u + p + nx1);
      float den = -((w + e_) + (sc + n));
      for (int e = 0; e < bd.nleg; ++e) {
        const int d = (bd.jdirs >> (2 * e)) & 3;
        const float k = d == DIR_PX ? e_ : d == DIR_MX ? w : d == DIR_PY ? n : sc;
        num -= k * sm.ldp[e][bi];
        den -= k * sm.lcp[e][bi];
      }
      const float x = num / den;
      sm.xj[bi] = x;
      a.u[p] = x;
    }
    __syncthreads();
    // back-substitution from the junction (0: a leg that ends at a wall) to
    // the wall; each row's value is its chunk's first (lo) or last (hi)
    // value, stored where the chunk lies (remote stores only)
    float xn = (act && bd.junc) ? sm.xj[bi] : 0.0f;
    kr = ch.roff + ch.nrow;
    for (int s = ch.nseg - 1; s >= 0; --s) {
      const int rk = ch.rank[s];
      CSeg sg = a.seg[pseg0[rk] + ch.slot[s]];
      // checked builds: the segment's chunks must be slots of its CTA
      if (!MG_OK_IF(sg.nchunk >= 1 && sg.slot0 + (sg.nchunk - 1) * sg.stride < SLOTS && sg.one <= 1)) sg.nchunk = 0;
      const int R = 2 * sg.nchunk - sg.one;
      float2 *chx = pchx[rk];
      kr -= R;
      for (int k = R - 1; k >= 0; --k) {
        const float2 v = sm.cd[kr + k];
        xn = v.y - v.x * xn;
        float2 &dst = chx[sg.slot0 + (k >> 1) * sg.stride];
        if (k & 1) dst.y = xn;
        else dst.x = xn;
        if (k == R - 1 && sg.one) dst.y = xn;  // a one-node chunk: first = last
      }
    }
  }
  __syncthreads();
  cluster_arrive();
  cluster_wait();
  // ---- phase 3: chunk interiors, written to u
  for (int t = warp; t < cd.ntile; t += CL_WARPS) {
    const CTile td = a.tile[cd.tile0 + t];
    const CLane ln = a.lane[(size_t)(cd.tile0 + t) * 32 + lane];
    if (td.kind == CT_COMPACT) tile_expand<true>(sm, a, t, td, ln, lane);
    else tile_expand<false>(sm, a, t, td, ln, lane);
  }
}

}  // namespace

cudaError_t prepare_cluster_kernel() {
  return cudaFuncSetAttribute(cluster_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
}

cudaError_t launch_cluster_pass(const Level &L, const ClusterPlan &cp, float *u, const float *f, cudaStream_t s,
                                cudaEvent_t *ev) {
  if (ev) cudaEventRecord(ev[0], s);
  Args a;
  a.tile = cp.tile; a.lane = cp.lane; a.cta = cp.cta; a.seg = cp.seg; a.block = cp.block; a.chain = cp.chain;
  a.cp = level_coefs<float>(L);
  a.nx = L.nx; a.ny = L.ny;
  a.u = u; a.f = f;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cp.ncta);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(Smem);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL_CTAS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, cluster_pass_kernel, a);
  if (ev) for (int k = 1; k < 4; ++k) cudaEventRecord(ev[k], s);
  count_launch(1);
  return e;
}

// Clusters of CL_CTAS CTAs of this kernel that the current device can hold
// at once (0: the cluster pass cannot run).
int cluster_pass_capacity() {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL_CTAS);
  cfg.blockDim = dim3(NT);
  cfg.dynamicSmemBytes = sizeof(Smem);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = CL_CTAS;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, cluster_pass_kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

}  // namespace tmg
