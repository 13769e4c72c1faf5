// smooth.cu -- relaxation kernels of tweedmg for sm_103a.
//
// line_pass_kernel: one colour pass of a line smoother (tweed, wireframe,
// zebra) on levels below the tiled path whose largest block is too long for
// the warp path of warp_line.cu (more than 1024 nodes in FP32 or 512 in FP64:
// wireframe rings from 512^2 up, in FP64 from 256^2 up; the FP64 tweed cross
// at 512^2).  Every block of the colour is solved exactly (Sec. 3: the
// equation is solved on all nodes of the block at once, the other colour held
// fixed).
// A CTA owns whole blocks.  Each block is a set of chains (open tridiagonal
// systems along straight runs that may turn corners) plus at most one
// junction node:
//   - tweed L-block (the paper's m = 2 case): one chain, no junction;
//   - tweed cross / T (m = 4 / 3, Eq. mLThomas): one chain per leg, all legs
//     coupled to the branch point, which is the junction;
//   - wireframe ring (Eq. CircTri): the ring is opened at one corner node,
//     which becomes the junction coupled to both ends of the remaining chain;
//   - zebra lines, straight tweed lines, the wireframe centre line: one chain;
//   - corner / centre points: a junction with no chain.
//
// The exact block solve is reorganised for parallelism, not approximated:
//   phase 0  all threads: right-hand side of every chain node (f minus the
//            neighbours outside the block) into shared memory;
//   phase 1  one thread per chunk (<= CMAX consecutive nodes of a run):
//            two eliminations across the chunk give the two reduced rows that
//            couple the chunk's first / last node to the neighbouring chunks
//            (partition method);
//   phase 2  parallel cyclic reduction (pointer jumping) on the reduced
//            system of all chunks, for two right-hand sides: the actual one
//            (y) and the response to a unit junction value (z);
//   phase 2b one thread per junction: its own row fixes the junction value
//            (x_J = (r_J - sum k y)/(C_J + sum k z)), the m-legged / periodic
//            Thomas step of the paper;
//   phase 3  one thread per chunk: chunk ends X = y + x_J z, interior by
//            Thomas with those ends;
//   phase 4  all threads: write the block back to u.
//
// checker_kernel: one colour of red-black point Gauss-Seidel (Sec. 2).
#include <cstdio>

#include "device_util.cuh"

namespace tmg {

template <typename T>
using CoefP = Coefs<T>;

__device__ __forceinline__ int di_of(int d) { return d == DIR_PX ? 1 : (d == DIR_MX ? -1 : 0); }
__device__ __forceinline__ int dj_of(int d) { return d == DIR_PY ? 1 : (d == DIR_MY ? -1 : 0); }

// Coefficient of row (i,j) for the neighbour one step in direction d.
template <typename T>
__device__ __forceinline__ T cf(const CoefP<T> &c, int i, int j, int d) {
  return d == DIR_PX ? __ldg(c.E + i) : d == DIR_MX ? __ldg(c.W + i) : d == DIR_PY ? __ldg(c.N + j) : __ldg(c.S + j);
}
// C_ij = -(W_i + E_i + S_j + N_j).
template <typename T>
__device__ __forceinline__ T centre(const CoefP<T> &c, int i, int j) {
  return -((__ldg(c.W + i) + __ldg(c.E + i)) + (__ldg(c.S + j) + __ldg(c.N + j)));
}


// Geometry of one chunk: a straight run of m nodes in direction dir.  Along
// the run only the two "along" coefficients vary (W/E for x-runs, S/N for
// y-runs); the two perpendicular ones are constant and enter the diagonal
// C = -(W + E + S + N) as the sum `cross`.
template <typename T>
struct ChunkGeom {
  int i0, j0, m, dir, nd, fl, var0, step;
  const T *lo_arr, *hi_arr;   // coefficient towards the predecessor / successor
  T cross, clast, cnd;        // perpendicular sum; successor coefficient of the last node;
                              // coefficient of the last node towards nextdir
  __device__ __forceinline__ void init(const ChunkDesc &cd, const CoefP<T> &cp) {
    i0 = cd.i0; j0 = cd.j0; m = cd.len; fl = cd.flags; dir = fl & 3; nd = (fl >> 2) & 3;
    const bool xrun = dir < 2;
    step = (dir == DIR_PX || dir == DIR_PY) ? 1 : -1;
    var0 = xrun ? i0 : j0;
    if (xrun) {
      lo_arr = dir == DIR_PX ? cp.W : cp.E;
      hi_arr = dir == DIR_PX ? cp.E : cp.W;
      cross = __ldg(cp.S + j0) + __ldg(cp.N + j0);
    } else {
      lo_arr = dir == DIR_PY ? cp.S : cp.N;
      hi_arr = dir == DIR_PY ? cp.N : cp.S;
      cross = __ldg(cp.W + i0) + __ldg(cp.E + i0);
    }
    const int il = i0 + (m - 1) * di_of(dir), jl = j0 + (m - 1) * dj_of(dir);
    cnd = cf(cp, il, jl, nd);
    clast = (fl & F_LN) ? cnd : T(0);
  }
  __device__ __forceinline__ T lo_at(int q) const { return __ldg(lo_arr + var0 + (q < m ? q : m - 1) * step); }
  __device__ __forceinline__ T hi_at(int q) const { return __ldg(hi_arr + var0 + (q < m ? q : m - 1) * step); }
  __device__ __forceinline__ T b_of(T lo, T hi) const { return -(cross + (lo + hi)); }
};

// Shared-memory slot of node q of chunk c (XOR swizzle, see ChunkDesc).
__device__ __forceinline__ int slot_of(int c, int q) { return 32 * c + (q ^ (c & 31)); }

// One reduced row  a x_L + x + c x_U = (y, z), stored as a vector.
template <typename T>
struct __align__(4 * sizeof(T)) Row {
  T a, c, y, z;
};

// Shared memory of one CTA: reduced rows, the slot arrays (right-hand side;
// with SC also the two along coefficients of every node, written by the load
// phase so that the eliminations read no global memory), junction values,
// reduced-row links, and copies of the CTA's chunk and vertical-group
// descriptors.
template <typename T, int NT, bool SC>
struct LineSmem {
  static constexpr size_t rows = sizeof(Row<T>) * 2 * NT;
  static constexpr size_t nodes = sizeof(T) * 32 * NT * (SC ? 3 : 1);
  static constexpr size_t junc = sizeof(T) * NT;
  static constexpr size_t links = sizeof(short2) * 2 * NT;
  static constexpr size_t descs = sizeof(ChunkDesc) * NT;
  static constexpr size_t groups = sizeof(VGroup) * (NT / 2);
  static constexpr size_t bytes = rows + nodes + junc + links + descs + groups;
};

// Per-chunk constants of the load / store phases: run direction and the
// neighbour mask of interior nodes (the two perpendicular directions) and of
// the first and last node.
struct RunMask {
  int dir, di, dj;
  unsigned mid, first, last;
  __device__ __forceinline__ RunMask(const ChunkDesc &cd) {
    dir = cd.flags & 3;
    const int nd = (cd.flags >> 2) & 3;
    di = di_of(dir);
    dj = dj_of(dir);
    const unsigned prev = 1u << (dir ^ 1), next = 1u << dir;
    const unsigned ex_prev = (cd.flags & (F_LP | F_FJ)) ? prev : 0u;   // predecessor in the chain / junction
    const unsigned ex_next = (cd.flags & (F_LN | F_LJ)) ? (1u << nd) : 0u;
    mid = 0xFu & ~prev & ~next;
    first = 0xFu & ~next & ~ex_prev;
    last = 0xFu & ~prev & ~ex_next;
    if (cd.len == 1) first = last = 0xFu & ~ex_prev & ~ex_next;
  }
  __device__ __forceinline__ unsigned at(int q, int len) const {
    return q == 0 ? first : (q == len - 1 ? last : mid);
  }
};

// Right-hand sides of U nodes (all loads issued before any is used).  Node k:
// slot sl[k] (or < 0 for none), coordinates (ik, jk), neighbour mask inc[k]
// (bits 0-3) and run direction dk[k].  With SC the two along coefficients of
// each node are stored as well.
template <typename T, bool SC, int U>
__device__ __forceinline__ void rhs_batch(const int (&sl)[U], const int (&ik)[U], const int (&jk)[U],
                                          const unsigned (&inc)[U], const int (&dk)[U], const CoefP<T> &cp,
                                          int nx1, const T *__restrict__ u, const T *__restrict__ f, T *node,
                                          T *clo, T *chi) {
  T fv[U], uw[U], ue[U], us[U], un[U], cw[U], ce[U], cs[U], cn[U];
#pragma unroll
  for (int k = 0; k < U; ++k) {
    const size_t p = (size_t)jk[k] * nx1 + ik[k];
    const bool ok = sl[k] >= 0;
    fv[k] = ok ? f[p] : T(0);
    uw[k] = (inc[k] & 2u) ? u[p - 1] : T(0);
    ue[k] = (inc[k] & 1u) ? u[p + 1] : T(0);
    us[k] = (inc[k] & 8u) ? u[p - nx1] : T(0);
    un[k] = (inc[k] & 4u) ? u[p + nx1] : T(0);
    cw[k] = __ldg(cp.W + ik[k]);
    ce[k] = __ldg(cp.E + ik[k]);
    cs[k] = __ldg(cp.S + jk[k]);
    cn[k] = __ldg(cp.N + jk[k]);
  }
#pragma unroll
  for (int k = 0; k < U; ++k) {
    if (sl[k] >= 0) {
      node[sl[k]] = fv[k] - cw[k] * uw[k] - ce[k] * ue[k] - cs[k] * us[k] - cn[k] * un[k];
      if constexpr (SC) {
        const bool x = dk[k] < 2, plus = (dk[k] & 1) == 0;
        const T a = x ? cw[k] : cs[k], b = x ? ce[k] : cn[k];
        clo[sl[k]] = plus ? a : b;
        chi[sl[k]] = plus ? b : a;
      }
    }
  }
}

// Phases 1 and 3 of one chunk with m nodes (m == CMAX when FULL, so that all
// guards are resolved at compile time).
template <typename T, bool SC, bool FULL>
struct ChunkSolver {
  const ChunkGeom<T> &g;
  const T *node, *clo, *chi;
  int c, m;
  __device__ __forceinline__ int mm() const { return FULL ? CMAX : m; }
  __device__ __forceinline__ int sl(int q) const {
    const int qq = FULL ? q : (q < m ? q : m - 1);
    return slot_of(c, qq);
  }
  __device__ __forceinline__ T LO(int q) const { if constexpr (SC) return clo[sl(q)]; else return g.lo_at(q); }
  __device__ __forceinline__ T HI(int q) const { if constexpr (SC) return chi[sl(q)]; else return g.hi_at(q); }
  __device__ __forceinline__ T DD(int q) const { return node[sl(q)]; }
  __device__ __forceinline__ T A(int q, T lo) const { return (q > 0 || (g.fl & F_LP)) ? lo : T(0); }
  __device__ __forceinline__ T C(int q, T hi) const { return q < mm() - 1 ? hi : g.clast; }

  // reduced rows: lo (in terms of x_{-1}, x_{m-1}) and hi (x_0, x_m)
  __device__ __forceinline__ void reduce(T kf, T kl, Row<T> &rlo, Row<T> &rhi) const {
    const int n = mm();
    const T l0 = LO(0), h0 = HI(0), d0 = DD(0);
    const T a0 = A(0, l0), b0 = g.b_of(l0, h0), c0 = C(0, h0);
    rhi.a = T(0); rhi.c = T(0); rhi.y = T(0); rhi.z = T(0);
    if (!FULL && n <= 2) {
      const T rb = recip(b0);
      rlo.a = a0 * rb; rlo.c = c0 * rb; rlo.y = d0 * rb; rlo.z = -(n == 1 ? kf + kl : kf) * rb;
      if (n == 1) return;
    }
    const T l1 = LO(1), h1 = HI(1);
    T rinv_f = recip(g.b_of(l1, h1));
    T al = A(1, l1) * rinv_f, ga = C(1, h1) * rinv_f, de = DD(1) * rinv_f;
    T ah = T(0), ch = T(0), dh = T(0);
#pragma unroll
    for (int k = 1; k <= CMAX - 2; ++k) {
      const int qf = k + 1;  // forward step
      if (FULL || qf < n) {
        const T lq = LO(qf), hq = HI(qf);
        const T a = A(qf, lq), cc = C(qf, hq);
        const T ri = recip(g.b_of(lq, hq) - a * ga);
        al = -a * al * ri;
        ga = cc * ri;
        de = (DD(qf) - a * de) * ri;
        rinv_f = ri;
      }
      const int qb = CMAX - 1 - k;  // backward step (descending)
      if (FULL || qb <= n - 2) {
        const T lq = LO(qb), hq = HI(qb);
        const T a = A(qb, lq), cc = C(qb, hq);
        if ((FULL && k == 1) || (!FULL && qb == n - 2)) {
          const T ri = recip(g.b_of(lq, hq));
          ah = a * ri; ch = cc * ri; dh = DD(qb) * ri;
        } else {
          const T ri = recip(g.b_of(lq, hq) - cc * ah);
          ah = a * ri;
          ch = -cc * ch * ri;
          dh = (DD(qb) - cc * dh) * ri;
        }
      }
    }
    rhi.a = al; rhi.c = ga; rhi.y = de; rhi.z = -kl * rinv_f;
    if (FULL || n >= 3) {
      const T rd = recip(b0 - c0 * ah);
      rlo.a = a0 * rd; rlo.c = -c0 * ch * rd; rlo.y = (d0 - c0 * dh) * rd; rlo.z = -kf * rd;
    }
  }

  // interior nodes 1..m-2 by Thomas with the known ends, written to the slots
  __device__ __forceinline__ void interior(T xlo, T xhi, T *out) const {
    const int n = mm();
    T cpv[CMAX];
    T dprev = xlo;
#pragma unroll
    for (int q = 1; q < CMAX - 1; ++q) {
      if (FULL || q <= n - 2) {
        const T lq = LO(q), hq = HI(q);
        const T a = A(q, lq), b = g.b_of(lq, hq), cc = C(q, hq);
        T dq = DD(q) - a * dprev;
        if ((FULL && q == CMAX - 2) || (!FULL && q == n - 2)) dq -= cc * xhi;
        const T ri = (q == 1) ? recip(b) : recip(b - a * cpv[q - 1]);
        cpv[q] = cc * ri;
        dprev = dq * ri;
        out[slot_of(c, q)] = dprev;
      }
    }
    T xn = dprev;  // x_{m-2}
#pragma unroll
    for (int q = CMAX - 3; q >= 1; --q) {
      if (FULL || q <= n - 3) {
        xn = out[slot_of(c, q)] - cpv[q] * xn;
        out[slot_of(c, q)] = xn;
      }
    }
  }
};

template <typename T, int NT, bool SC>
__global__ void __launch_bounds__(NT, NT == NT_SMALL ? 2 : 1)
    line_pass_kernel(const CtaWork *__restrict__ works, const ChunkDesc *__restrict__ chunks_all,
                     const JuncDesc *__restrict__ juncs_all, const VGroup *__restrict__ vgs_all, CoefP<T> cp,
                     int nx1, int ny1, T *__restrict__ u, const T *__restrict__ f) {
  using SM = LineSmem<T, NT, SC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Row<T> *rv = reinterpret_cast<Row<T> *>(smem_raw);                        // 2*NT reduced rows
  T *node = reinterpret_cast<T *>(smem_raw + SM::rows);                     // 32*NT slots
  T *clo = node + 32 * NT;                                                  // along coefficients (SC)
  T *chi = clo + 32 * NT;
  T *xj = reinterpret_cast<T *>(smem_raw + SM::rows + SM::nodes);           // junction values
  short2 *lu = reinterpret_cast<short2 *>(smem_raw + SM::rows + SM::nodes + SM::junc);
  ChunkDesc *sc = reinterpret_cast<ChunkDesc *>(smem_raw + SM::rows + SM::nodes + SM::junc + SM::links);
  VGroup *svg = reinterpret_cast<VGroup *>(smem_raw + SM::rows + SM::nodes + SM::junc + SM::links + SM::descs);

  pdl_trigger();
  CtaWork w = works[blockIdx.x];
  // checked builds: the CTA's counts must fit its shared memory (else it
  // does nothing)
  if (!MG_OK_IF(w.nchunk >= 0 && w.nchunk <= NT && w.nvg >= 0 && w.nvg <= NT && w.njunc >= 0 && w.njunc <= NT))
    w.nchunk = w.nvg = w.njunc = 0;
  const JuncDesc *juncs = juncs_all + w.junc0;
  const int tid = threadIdx.x;
  for (int t = tid; t < w.nchunk; t += NT) {
    ChunkDesc cd = chunks_all[w.chunk0 + t];
#ifdef MG_CHECK
    // checked builds: a chunk's run must lie among the interior nodes (else
    // it is emptied)
    const int dir = cd.flags & 3;
    const int di = dir == DIR_PX ? 1 : dir == DIR_MX ? -1 : 0, dj = dir == DIR_PY ? 1 : dir == DIR_MY ? -1 : 0;
    const int ie = cd.i0 + (cd.len - 1) * di, je = cd.j0 + (cd.len - 1) * dj;
    if (cd.len > 0 && !MG_OK_IF(cd.len <= CMAX && cd.i0 >= 1 && cd.i0 <= nx1 - 2 && cd.j0 >= 1 &&
                                cd.j0 <= ny1 - 2 && ie >= 1 && ie <= nx1 - 2 && je >= 1 && je <= ny1 - 2))
      cd.len = 0;
#endif
    sc[t] = cd;
  }
  for (int t = tid; t < w.nvg; t += NT) svg[t] = vgs_all[w.vg0 + t];
  pdl_wait();  // u and f from here on
  __syncthreads();

  // ---- phase 0: right-hand sides of all chain nodes.  Grouped vertical
  // chunks first (lanes over 8 rows x 4 columns), then every other chunk with
  // lanes along its run; several nodes per thread per batch.
  {
    const int warp = tid >> 5, lane = tid & 31;
    for (int vi = warp; vi < w.nvg; vi += NT / 32) {
      const int c = svg[vi].c[lane & 3];
      ChunkDesc cd;
      cd.len = 0; cd.flags = 0; cd.i0 = 1; cd.j0 = 1;
      if (c != 0xFFFF) cd = sc[c];
      const RunMask rm(cd);
      int sl[4], ik[4], jk[4], dk[4];
      unsigned inc[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int q = 8 * r + (lane >> 2);
        const bool ok = q < cd.len;
        sl[r] = ok ? slot_of(c, q) : -1;
        ik[r] = cd.i0 + q * rm.di; jk[r] = cd.j0 + q * rm.dj;
        if (!ok) { ik[r] = 1; jk[r] = 1; }
        inc[r] = ok ? rm.at(q, cd.len) : 0u;
        dk[r] = rm.dir;
      }
      rhs_batch<T, SC, 4>(sl, ik, jk, inc, dk, cp, nx1, u, f, node, clo, chi);
    }
  }
  {
    constexpr int U = 4;
    const int warp = tid >> 5, lane = tid & 31;
    // warp-uniform chunks: lanes are the nodes of one chunk
    for (int c0 = warp; c0 < w.nchunk; c0 += U * (NT / 32)) {
      int sl[U], ik[U], jk[U], dk[U];
      unsigned inc[U];
#pragma unroll
      for (int k = 0; k < U; ++k) {
        const int c = c0 + k * (NT / 32);
        ChunkDesc cd;
        cd.len = 0; cd.flags = 0; cd.i0 = 1; cd.j0 = 1; cd.info = GROUPED;
        if (c < w.nchunk) cd = sc[c];
        const RunMask rm(cd);
        const bool ok = lane < cd.len && !(cd.info & GROUPED);
        sl[k] = ok ? slot_of(c, lane) : -1;
        ik[k] = ok ? cd.i0 + lane * rm.di : 1;
        jk[k] = ok ? cd.j0 + lane * rm.dj : 1;
        inc[k] = ok ? rm.at(lane, cd.len) : 0u;
        dk[k] = rm.dir;
      }
      rhs_batch<T, SC, U>(sl, ik, jk, inc, dk, cp, nx1, u, f, node, clo, chi);
    }
  }
  __syncthreads();

  // ---- phase 1: reduced rows of every chunk (partition method).  Two
  // independent eliminations run interleaved: nodes 1..m-2 towards node m-1
  // (the "hi" row, in terms of x_0 and x_m) and nodes m-2..1 towards node 0
  // (the "lo" row, in terms of x_{-1} and x_{m-1}).
  const int R = 2 * w.nchunk;
  if (tid < w.nchunk) {
    const ChunkDesc cd = sc[tid];
    ChunkGeom<T> g;
    g.init(cd, cp);
    const T kf = (g.fl & F_FJ) ? cf(cp, g.i0, g.j0, g.dir ^ 1) : T(0);
    const T kl = (g.fl & F_LJ) ? g.cnd : T(0);
    Row<T> rlo, rhi;
    if (g.m == CMAX) ChunkSolver<T, SC, true>{g, node, clo, chi, tid, g.m}.reduce(kf, kl, rlo, rhi);
    else ChunkSolver<T, SC, false>{g, node, clo, chi, tid, g.m}.reduce(kf, kl, rlo, rhi);
    const int m = g.m;
    short Llo = -1, Ulo;
    if (g.fl & F_LP) Llo = (short)(sc[tid - 1].len >= 2 ? 2 * (tid - 1) + 1 : 2 * (tid - 1));
    if (m >= 2) Ulo = (short)(2 * tid + 1);
    else Ulo = (g.fl & F_LN) ? (short)(2 * (tid + 1)) : (short)-1;
    rv[2 * tid] = rlo;
    rv[2 * tid + 1] = rhi;
    lu[2 * tid] = make_short2(Llo, Ulo);
    lu[2 * tid + 1] = (m >= 2) ? make_short2((short)(2 * tid), (g.fl & F_LN) ? (short)(2 * (tid + 1)) : (short)-1)
                               : make_short2(-1, -1);
  }
  __syncthreads();

  // ---- phase 2: parallel cyclic reduction (pointer jumping) on the reduced
  // system, two right-hand sides (y: data, z: unit junction value)
  for (int it = 0; it < 24; ++it) {
    Row<T> nr[2];
    short2 nl[2];
    bool upd[2] = {false, false};
    bool more = false;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int r = tid + k * NT;
      if (r < R) {
        const short2 l = lu[r];
        if (l.x >= 0 || l.y >= 0) {
          const Row<T> me = rv[r];
          Row<T> L = {T(0), T(0), T(0), T(0)}, Uu = {T(0), T(0), T(0), T(0)};
          short LL = -1, UU = -1;
          if (l.x >= 0) { L = rv[l.x]; LL = lu[l.x].x; }
          if (l.y >= 0) { Uu = rv[l.y]; UU = lu[l.y].y; }
          const T beta = recip(T(1) - me.a * L.c - me.c * Uu.a);
          nr[k].a = -me.a * L.a * beta;
          nr[k].c = -me.c * Uu.c * beta;
          nr[k].y = (me.y - me.a * L.y - me.c * Uu.y) * beta;
          nr[k].z = (me.z - me.a * L.z - me.c * Uu.z) * beta;
          nl[k] = make_short2(LL, UU);
          upd[k] = true;
          more |= (LL >= 0 || UU >= 0);
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 2; ++k)
      if (upd[k]) { rv[tid + k * NT] = nr[k]; lu[tid + k * NT] = nl[k]; }
    if (!__syncthreads_or(more)) break;
  }

  // ---- phase 2b: junction rows
  if (tid < w.njunc) {
    JuncDesc jd = juncs[tid];
    // checked builds: the junction must be interior with at most 4 chain ends
    bool jok = jd.i >= 1 && jd.i <= nx1 - 2 && jd.j >= 1 && jd.j <= ny1 - 2 && jd.nend <= 4;
    for (int e = 0; e < 4 && jok; ++e) jok = e >= jd.nend || jd.row[e] < 2 * NT;
    if (!MG_OK_IF(jok)) {
      jd.i = 1; jd.j = 1; jd.nend = 0;
    }
    const int i = jd.i, j = jd.j;
    const size_t p = (size_t)j * nx1 + i;
    unsigned att = 0;
    for (int e = 0; e < jd.nend; ++e) att |= 1u << ((jd.dirs >> (2 * e)) & 3);
    T r = f[p];
    if (!(att & 2u)) r -= __ldg(cp.W + i) * u[p - 1];
    if (!(att & 1u)) r -= __ldg(cp.E + i) * u[p + 1];
    if (!(att & 8u)) r -= __ldg(cp.S + j) * u[p - nx1];
    if (!(att & 4u)) r -= __ldg(cp.N + j) * u[p + nx1];
    T num = r, den = centre(cp, i, j);
    for (int e = 0; e < jd.nend; ++e) {
      const T k = cf(cp, i, j, (jd.dirs >> (2 * e)) & 3);
      const Row<T> re = rv[jd.row[e]];
      num -= k * re.y;
      den += k * re.z;
    }
    const T x = num / den;
    u[p] = x;
    xj[tid] = x;
  }
  __syncthreads();

  // ---- phase 3: chunk ends from the reduced solution, interiors by Thomas
  if (tid < w.nchunk) {
    const ChunkDesc cd = sc[tid];
    ChunkGeom<T> g;
    g.init(cd, cp);
    const int m = g.m;
    const int jn = cd.info & 1023;
    const T jx = (jn != JNONE) ? xj[jn] : T(0);
    const Row<T> r0 = rv[2 * tid], r1 = rv[2 * tid + 1];
    const T xlo = r0.y + jx * r0.z;
    const T xhi = (m >= 2) ? r1.y + jx * r1.z : xlo;
    if (m == CMAX) ChunkSolver<T, SC, true>{g, node, clo, chi, tid, m}.interior(xlo, xhi, node);
    else if (m >= 3) ChunkSolver<T, SC, false>{g, node, clo, chi, tid, m}.interior(xlo, xhi, node);
    node[slot_of(tid, 0)] = xlo;
    if (m >= 2) node[slot_of(tid, m - 1)] = xhi;
  }
  __syncthreads();

  // ---- phase 4: write the block back (same two mappings as phase 0)
  {
    const int warp = tid >> 5, lane = tid & 31;
    for (int vi = warp; vi < w.nvg; vi += NT / 32) {
      const int c = svg[vi].c[lane & 3];
      if (c == 0xFFFF) continue;
      const ChunkDesc cd = sc[c];
      const int dj = dj_of(cd.flags & 3);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int q = 8 * r + (lane >> 2);
        if (q < cd.len) u[(size_t)(cd.j0 + q * dj) * nx1 + cd.i0] = node[slot_of(c, q)];
      }
    }
    for (int c = warp; c < w.nchunk; c += NT / 32) {
      const ChunkDesc cd = sc[c];
      if ((cd.info & GROUPED) || lane >= cd.len) continue;
      const int dir = cd.flags & 3;
      u[(size_t)(cd.j0 + lane * dj_of(dir)) * nx1 + cd.i0 + lane * di_of(dir)] = node[slot_of(c, lane)];
    }
  }
}


template <typename T, int NT>
static cudaError_t launch_shape(const Level &L, const WorkList &w, T *u, const T *f, cudaStream_t s) {
  constexpr bool SC = sizeof(T) == 4;  // FP64 keeps the coefficients in L1 (smem is too small)
  constexpr size_t smem = LineSmem<T, NT, SC>::bytes;
  auto kern = line_pass_kernel<T, NT, SC>;
  count_launch(1);
  return launch_pdl(kern, dim3(w.ncta), dim3(NT), smem, s, (const CtaWork *)w.cta, (const ChunkDesc *)w.chunk,
                    (const JuncDesc *)w.junc, (const VGroup *)w.vg, level_coefs<T>(L), L.nx + 1, L.ny + 1, u, f);
}

template <typename T>
cudaError_t launch_line_pass(const Level &L, const WorkList &w, T *u, const T *f, cudaStream_t s) {
  if (w.ncta == 0) return cudaSuccess;
  return w.nt == NT_SMALL ? launch_shape<T, NT_SMALL>(L, w, u, f, s) : launch_shape<T, NT_LARGE>(L, w, u, f, s);
}

// Opt the line kernels into their dynamic shared memory on the current device
// (mg_setup_grid calls this on the grid's device).
template <typename T, int NT>
static cudaError_t prepare_shape() {
  constexpr bool SC = sizeof(T) == 4;
  return cudaFuncSetAttribute(line_pass_kernel<T, NT, SC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)LineSmem<T, NT, SC>::bytes);
}
cudaError_t prepare_line_kernels() {
  cudaError_t e = prepare_shape<double, NT_SMALL>();
  if (e == cudaSuccess) e = prepare_shape<double, NT_LARGE>();
  if (e == cudaSuccess) e = prepare_shape<float, NT_SMALL>();
  if (e == cudaSuccess) e = prepare_shape<float, NT_LARGE>();
  return e;
}

template cudaError_t launch_line_pass<double>(const Level &, const WorkList &, double *, const double *, cudaStream_t);
template cudaError_t launch_line_pass<float>(const Level &, const WorkList &, float *, const float *, cudaStream_t);

// ---------------------------------------------------------------------------
// Red-black point Gauss-Seidel, one colour (red = (i+j) even).  One thread per
// node of the colour; blockIdx.y = interior row.
template <typename T>
__global__ void checker_kernel(CoefP<T> cp, int nx, int colour, T *__restrict__ u, const T *__restrict__ f) {
  pdl_trigger();
  pdl_wait();
  const int j = blockIdx.y + 1;
  const int i0 = ((j + colour) & 1) ? 1 : 2;   // first interior i with (i+j)%2 == colour
  const int i = i0 + 2 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i >= nx) return;
  const int nx1 = nx + 1;
  const size_t p = (size_t)j * nx1 + i;
  const T w = __ldg(cp.W + i), e = __ldg(cp.E + i), s = __ldg(cp.S + j), n = __ldg(cp.N + j);
  const T r = f[p] - w * u[p - 1] - e * u[p + 1] - s * u[p - nx1] - n * u[p + nx1];
  u[p] = r / (-((w + e) + (s + n)));
}

template <typename T>
cudaError_t launch_checker_pass(const Level &L, int colour, T *u, const T *f, cudaStream_t s) {
  const int half = L.nx / 2 + 1;
  dim3 block(128), grid((half + 127) / 128, L.ny - 1);
  count_launch(1);
  return launch_pdl(checker_kernel<T>, grid, block, 0, s, level_coefs<T>(L), L.nx, colour, u, f);
}
template cudaError_t launch_checker_pass<double>(const Level &, int, double *, const double *, cudaStream_t);
template cudaError_t launch_checker_pass<float>(const Level &, int, float *, const float *, cudaStream_t);

}  // namespace tmg
