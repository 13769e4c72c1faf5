// mini.cu -- the coarse end of a multigrid cycle (Sec. 4 steps (1)-(6)) in
// one CTA (sm_103a).
//
// On the coarse levels a colour pass touches a few thousand nodes, and a
// kernel per pass costs more in launch and pipeline latency than in work.
// Here the cycle from level m (the finest level whose whole sub-hierarchy
// fits in shared memory) down to the coarsest and back runs in a single
// kernel: every level's u, f and coefficients live in shared memory, and the
// passes, transfers and the coarsest solve are separated by CTA barriers.
//
// Smoothing (Sec. 3): each block of the colour is solved exactly by one
// thread.  A block is chains of nodes (straight runs that may turn corners)
// plus at most one junction node (the tweed star of Eq. mLThomas, the node
// closing a wireframe ring of Eq. CircTri, a lone point).  With the junction
// value x_J as a parameter, every chain is a tridiagonal system; its solution
// is x = yb + x_J zb, yb the solution for x_J = 0 and zb the response to a
// unit x_J.  zb, the Thomas multipliers c' and the pivot reciprocals depend
// only on the coefficients and are prepared on the host at setup.  On the
// device a chain costs one forward sweep (y', written in place into u: no
// node of the block or of its colour appears on the right-hand side of
// another) and one backward sweep; the junction row then gives
//   x_J = (r_J - sum k yb_end) / (C_J + sum k zb_end),
// and u += x_J zb on the chains.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "blocks.h"
#include "mg_internal.h"

namespace tmg {

namespace {

constexpr int MINI_THREADS = 512;
constexpr size_t MINI_SMEM_MAX = 200 * 1024;
constexpr int BASE_CHECKER = 0, BASE_ZEBRA_X = 1, BASE_ZEBRA_Y = 2, BASE_TWEED = 3, BASE_WIREFRAME = 4, NBASE = 5;

// Precomputed data of one (level, base smoother), both colours: per chain
// node the Thomas multiplier c' and the pivot reciprocal (and, after a
// block's chain nodes, 1 / (C_J + sum k zb_end) in piv for a junction
// block); per chain node of a junction block the unit-junction response zb.
// Staged in shared memory at kernel start: cp at soff, piv at soff + na, zb
// at zoff; the global indices a0 .. a0 + na and z0 .. z0 + nz map to them.
struct PreRange {
  uint32_t a0, na, z0, nz;
  int soff, zoff;
};

template <typename T>
struct MiniArgs {
  int nl;  // levels in the kernel: m .. m + nl - 1 (the last is the coarsest)
  int tl0;  // index of level m in the plan's block table
  int smoother, nu1, nu2, gamma, restriction;
  int nbase, base[2];  // base smoothers of the smoother
  int nx[MINI_MAX_LEV], ny[MINI_MAX_LEV];
  int off_u[MINI_MAX_LEV], off_f[MINI_MAX_LEV], off_c[MINI_MAX_LEV];  // shared-memory offsets (elements of T)
  PreRange pr[MINI_MAX_LEV][2];
  const T *W[MINI_MAX_LEV], *E[MINI_MAX_LEV], *S[MINI_MAX_LEV], *N[MINI_MAX_LEV];
  const MBlock *blocks;
  const T *cp, *piv, *zb;  // global copies of the precomputed data
  const uint2 *tab;        // [(level * NBASE + base) * 2 + colour] = (first block, count)
  const double *cinv;      // coarsest level: dense inverse (FP64)
  int cn;
};

// The staged precomputed data of one (level, base), indexed by global index.
template <typename T>
struct PreView {
  const T *cp, *piv, *zb;  // shared memory
  uint32_t a0, z0;
};

__device__ __forceinline__ int dstep(int d, int nx1) { return d == DIR_PX ? 1 : d == DIR_MX ? -1 : d == DIR_PY ? nx1 : -nx1; }

template <typename T>
struct SmemLevel {
  T *U, *F;
  const T *W, *E, *S, *N;
  int nx, ny, nx1;
  __device__ __forceinline__ T coef(int i, int j, int d) const {
    return d == DIR_PX ? E[i] : d == DIR_MX ? W[i] : d == DIR_PY ? N[j] : S[j];
  }
  __device__ __forceinline__ T centre(int i, int j) const { return -((W[i] + E[i]) + (S[j] + N[j])); }
};

template <typename T>
__device__ SmemLevel<T> level_view(const MiniArgs<T> &a, T *sm, int r) {
  SmemLevel<T> v;
  v.nx = a.nx[r]; v.ny = a.ny[r]; v.nx1 = a.nx[r] + 1;
  v.U = sm + a.off_u[r];
  v.F = sm + a.off_f[r];
  const T *c = sm + a.off_c[r];
  v.W = c; v.E = c + v.nx1; v.S = c + 2 * v.nx1; v.N = c + 2 * v.nx1 + (v.ny + 1);
  return v;
}

constexpr int BATCH = 8;  // nodes whose loads are issued together in a sweep

__device__ __forceinline__ int step_i(int d) { return d == DIR_PX ? 1 : d == DIR_MX ? -1 : 0; }
__device__ __forceinline__ int step_j(int d) { return d == DIR_PY ? 1 : d == DIR_MY ? -1 : 0; }

// Exact solve of one block (see the file comment).  The sweeps go BATCH
// nodes at a time: first every load of the batch (right-hand sides from
// neighbours outside the block, coupling coefficients, precomputed values),
// then the recurrence, so that the loads are in flight together.
template <typename T>
__device__ __forceinline__ void solve_block(const MBlock *__restrict__ Bp, const PreView<T> pv_, const SmemLevel<T> L) {
  const MBlock B = *Bp;
  T yf[4], yl[4];
  uint32_t q = B.pre0;
  const int nx1 = L.nx1;
  for (int e = 0; e < B.nchain; ++e) {
    const MChain &c = B.ch[e];
    const bool fj = c.flags & 1, lj = c.flags & 2;
    const int d0 = c.dir[0];
    int i = c.i0 - step_i(d0), j = c.j0 - step_j(d0);  // one step before the first node
    int k = 0;
    T yprev = T(0);
    // forward sweep: y'_k = (r_k - a_k y'_{k-1}) * pivot_k, stored in u
    for (int s = 0; s < c.nseg; ++s) {
      const int d = c.dir[s], n = c.len[s], di = step_i(d), dj = step_j(d);
      const int nd = s < c.nseg - 1 ? c.dir[s + 1] : (lj ? c.ljdir : -1);
      for (int t0 = 0; t0 < n; t0 += BATCH) {
        T rr[BATCH], aa[BATCH], pv[BATCH];
#pragma unroll
        for (int v = 0; v < BATCH; ++v) {
          const int t = t0 + v, kk = k + v;
          rr[v] = T(0); aa[v] = T(0); pv[v] = T(0);
          if (t < n) {
            const int ii = i + (v + 1) * di, jj = j + (v + 1) * dj, p = jj * nx1 + ii;
            const int pd = kk > 0 ? (d ^ 1) : (fj ? (d0 ^ 1) : -1);
            const int sd = t < n - 1 ? d : nd;
            T r = L.F[p];
#pragma unroll
            for (int dd = 0; dd < 4; ++dd)
              if (dd != pd && dd != sd) r -= L.coef(ii, jj, dd) * L.U[p + dstep(dd, nx1)];
            rr[v] = r;
            if (kk > 0) aa[v] = L.coef(ii, jj, pd);
            pv[v] = pv_.piv[q - pv_.a0 + kk];
          }
        }
#pragma unroll
        for (int v = 0; v < BATCH; ++v)
          if (t0 + v < n) {
            const T y = (rr[v] - aa[v] * yprev) * pv[v];
            L.U[(j + (v + 1) * dj) * nx1 + i + (v + 1) * di] = y;
            yprev = y;
          }
        const int cnt = min(BATCH, n - t0);
        i += cnt * di; j += cnt * dj;
        k += cnt;
      }
    }
    const int n = k;
    // backward sweep (x_J = 0): x_k = y'_k - c'_k x_{k+1}; (i, j) = last node
    T xn = T(0);
    for (int s = c.nseg - 1; s >= 0; --s) {
      const int d = c.dir[s], di = step_i(d), dj = step_j(d);
      for (int t1 = c.len[s]; t1 > 0; t1 -= BATCH) {
        const int cnt = min(BATCH, t1);
        T yv[BATCH], cv[BATCH];
#pragma unroll
        for (int v = 0; v < BATCH; ++v)
          if (v < cnt) {
            yv[v] = L.U[(j - v * dj) * nx1 + i - v * di];
            cv[v] = pv_.cp[q - pv_.a0 + (k - 1 - v)];
          }
#pragma unroll
        for (int v = 0; v < BATCH; ++v)
          if (v < cnt) {
            const T x = yv[v] - cv[v] * xn;  // c'_{n-1} = 0
            L.U[(j - v * dj) * nx1 + i - v * di] = x;
            xn = x;
            if (k - 1 - v == n - 1) yl[e] = x;
          }
        i -= cnt * di; j -= cnt * dj;
        k -= cnt;
      }
    }
    yf[e] = xn;
    q += n;
  }
  if (!B.junc) return;
  // junction row: x_J = (r_J - sum k yb_end) / (C_J + sum k zb_end)
  const int i = B.ji, j = B.jj, p = j * nx1 + i;
  unsigned att = 0;
  for (int e = 0; e < B.nchain; ++e) {
    if (B.ch[e].flags & 1) att |= 1u << B.ch[e].dir[0];
    if (B.ch[e].flags & 2) att |= 1u << (B.ch[e].ljdir ^ 1);
  }
  T num = L.F[p];
#pragma unroll
  for (int dd = 0; dd < 4; ++dd)
    if (!(att & (1u << dd))) num -= L.coef(i, j, dd) * L.U[p + dstep(dd, nx1)];
  for (int e = 0; e < B.nchain; ++e) {
    if (B.ch[e].flags & 1) num -= L.coef(i, j, B.ch[e].dir[0]) * yf[e];
    if (B.ch[e].flags & 2) num -= L.coef(i, j, B.ch[e].ljdir ^ 1) * yl[e];
  }
  const T xj = num * pv_.piv[q - pv_.a0];
  L.U[p] = xj;
  // u += x_J zb on every chain node
  uint32_t q2 = B.zb0 - pv_.z0;
  for (int e = 0; e < B.nchain; ++e) {
    const MChain &c = B.ch[e];
    const int d0 = c.dir[0];
    int ii = c.i0 - step_i(d0), jj = c.j0 - step_j(d0), k = 0;
    for (int s = 0; s < c.nseg; ++s) {
      const int d = c.dir[s], n = c.len[s], di = step_i(d), dj = step_j(d);
      for (int t0 = 0; t0 < n; t0 += BATCH) {
        const int cnt = min(BATCH, n - t0);
        T zv[BATCH];
#pragma unroll
        for (int v = 0; v < BATCH; ++v)
          if (v < cnt) zv[v] = pv_.zb[q2 + k + v];
#pragma unroll
        for (int v = 0; v < BATCH; ++v)
          if (v < cnt) L.U[(jj + (v + 1) * dj) * nx1 + ii + (v + 1) * di] += xj * zv[v];
        ii += cnt * di; jj += cnt * dj;
        k += cnt;
      }
    }
    q2 += k;
  }
}

// One colour pass of a base smoother on level r.
template <typename T>
__device__ void mini_pass(const MiniArgs<T> &a, T *sm, const SmemLevel<T> &L, int r, int base, int colour) {
  if (base == BASE_CHECKER) {
    // red-black point relaxation, red = (i + j) even
    const int w = L.nx - 1, n = w * (L.ny - 1);
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const int i = k % w + 1, j = k / w + 1;
      if (((i + j) & 1) != colour) continue;
      const int p = j * L.nx1 + i;
      const T s = L.coef(i, j, DIR_MX) * L.U[p - 1] + L.coef(i, j, DIR_PX) * L.U[p + 1] +
                  L.coef(i, j, DIR_MY) * L.U[p - L.nx1] + L.coef(i, j, DIR_PY) * L.U[p + L.nx1];
      L.U[p] = (L.F[p] - s) / L.centre(i, j);
    }
  } else {
    const uint2 t = a.tab[((size_t)(a.tl0 + r) * NBASE + base) * 2 + colour];
    const PreRange &R = a.pr[r][base == a.base[0] ? 0 : 1];
    PreView<T> v;
    v.cp = sm + R.soff; v.piv = sm + R.soff + R.na; v.zb = sm + R.zoff;
    v.a0 = R.a0; v.z0 = R.z0;
    for (uint32_t b = threadIdx.x; b < t.y; b += blockDim.x) solve_block(a.blocks + t.x + b, v, L);
  }
  __syncthreads();
}

// One relaxation of the smoother on level r: for each of its base smoothers,
// the red pass then the black pass (alt-zebra: x then y; alt tweed/wireframe:
// tweed then wireframe).
template <typename T>
__device__ void mini_smooth(const MiniArgs<T> &a, T *sm, const SmemLevel<T> &L, int r) {
  const int np = a.nbase > 0 ? 2 * a.nbase : 2;
  for (int k = 0; k < np; ++k) {
    const int base = a.nbase > 0 ? a.base[k >> 1] : BASE_CHECKER;
    mini_pass(a, sm, L, r, base, k & 1);
  }
}

template <typename T>
__device__ __forceinline__ T defect(const SmemLevel<T> &L, int i, int j) {
  const int p = j * L.nx1 + i;
  const T w = L.W[i], e = L.E[i], s = L.S[j], n = L.N[j];
  const T cc = -((w + e) + (s + n));
  return L.F[p] - (w * L.U[p - 1] + e * L.U[p + 1] + s * L.U[p - L.nx1] + n * L.U[p + L.nx1] + cc * L.U[p]);
}

// Defect of level r restricted to level r + 1 (half / full weighting,
// Sec. 4); the coarse correction starts from zero.
template <typename T>
__device__ void mini_restrict(int kind, const SmemLevel<T> &F, const SmemLevel<T> &C) {
  const int nc1 = C.nx1, ncn = nc1 * (C.ny + 1);
  for (int k = threadIdx.x; k < ncn; k += blockDim.x) C.U[k] = T(0);
  const int w = C.nx - 1, n = w * (C.ny - 1);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int I = k % w + 1, J = k / w + 1, i = 2 * I, j = 2 * J;
    const T centre = defect(F, i, j);
    const T edge = (defect(F, i - 1, j) + defect(F, i, j - 1)) + (defect(F, i + 1, j) + defect(F, i, j + 1));
    T v;
    if (kind == MG_RESTRICT_HW) {
      v = T(0.5) * centre + T(0.125) * edge;
    } else {
      const T corner = (defect(F, i - 1, j - 1) + defect(F, i + 1, j - 1)) +
                       (defect(F, i - 1, j + 1) + defect(F, i + 1, j + 1));
      v = T(0.25) * centre + T(0.125) * edge + T(0.0625) * corner;
    }
    C.F[J * nc1 + I] = v;
  }
  __syncthreads();
}

// u_r += bilinear interpolation of u_{r+1} (Sec. 4).
template <typename T>
__device__ void mini_prolong(const SmemLevel<T> &F, const SmemLevel<T> &C) {
  const int w = F.nx - 1, n = w * (F.ny - 1), c1 = C.nx1;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int i = k % w + 1, j = k / w + 1, I = i >> 1, Jc = j >> 1;
    const T *uc = C.U;
    T v;
    if (!(i & 1) && !(j & 1)) v = uc[Jc * c1 + I];
    else if (!(i & 1)) v = T(0.5) * (uc[Jc * c1 + I] + uc[(Jc + 1) * c1 + I]);
    else if (!(j & 1)) v = T(0.5) * (uc[Jc * c1 + I] + uc[Jc * c1 + I + 1]);
    else
      v = T(0.25) * ((uc[Jc * c1 + I] + uc[Jc * c1 + I + 1]) + (uc[(Jc + 1) * c1 + I] + uc[(Jc + 1) * c1 + I + 1]));
    F.U[j * F.nx1 + i] += v;
  }
  __syncthreads();
}

// Coarsest level: u = A^{-1} (f - boundary terms), A^{-1} dense (FP64); one
// warp per row of A^{-1}, lanes over its columns (coalesced), fixed-order
// shuffle reduction.
template <typename T>
__device__ void mini_coarse(const MiniArgs<T> &a, const SmemLevel<T> &L, double *bsm) {
  const int w = L.nx - 1, n = a.cn;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int i = k % w + 1, j = k / w + 1, p = j * L.nx1 + i;
    double b = (double)L.F[p];
    if (i == 1) b -= (double)L.W[i] * (double)L.U[p - 1];
    if (i == L.nx - 1) b -= (double)L.E[i] * (double)L.U[p + 1];
    if (j == 1) b -= (double)L.S[j] * (double)L.U[p - L.nx1];
    if (j == L.ny - 1) b -= (double)L.N[j] * (double)L.U[p + L.nx1];
    bsm[k] = b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = threadIdx.x >> 5; k < n; k += nw) {
    double x = 0.0;
    for (int q = lane; q < n; q += 32) x += __ldg(a.cinv + (size_t)k * n + q) * bsm[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      const int i = k % w + 1, j = k / w + 1;
      L.U[j * L.nx1 + i] = (T)x;
    }
  }
  __syncthreads();
}

// Sec. 4 steps (2)-(6) from level 0 of the plan down, gamma visits of each
// coarser level per visit of its parent (V: 1, W: 2) -- the recursion of the
// host driver, unrolled into a loop over an explicit per-level state so that
// the whole cycle is one inlined kernel body (each step has one call site).
template <typename T>
__device__ void mini_cycle(const MiniArgs<T> &a, T *sm, double *bsm) {
  int visits[MINI_MAX_LEV];
  int r = 0;
  bool down = true;  // entering level r from above (else returning to it from r + 1)
  while (r >= 0) {
    const SmemLevel<T> L = level_view(a, sm, r);
    if (r == a.nl - 1) {
      mini_coarse(a, L, bsm);
      --r;
      down = false;
      continue;
    }
    const SmemLevel<T> C = level_view(a, sm, r + 1);
    int nsm;
    if (down) {
      nsm = a.nu1;
    } else if (++visits[r] < a.gamma) {  // W-cycle: visit level r + 1 again
      ++r;
      down = true;
      continue;
    } else {
      mini_prolong(L, C);
      nsm = a.nu2;
    }
    for (int k = 0; k < nsm; ++k) mini_smooth(a, sm, L, r);
    if (down) {
      mini_restrict(a.restriction, L, C);
      visits[r] = 0;
      ++r;
    } else {
      --r;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(MINI_THREADS) mini_cycle_kernel(MiniArgs<T> a, T *__restrict__ ug,
                                                                  const T *__restrict__ fg) {
  extern __shared__ __align__(16) unsigned char mini_smem[];
  double *bsm = reinterpret_cast<double *>(mini_smem);
  T *sm = reinterpret_cast<T *>(mini_smem + sizeof(double) * ((a.cn + 1) & ~1));
  const int n0 = (a.nx[0] + 1) * (a.ny[0] + 1);
  T *U0 = sm + a.off_u[0], *F0 = sm + a.off_f[0];
  for (int k = threadIdx.x; k < n0; k += blockDim.x) { U0[k] = ug[k]; F0[k] = fg[k]; }
  for (int r = 0; r < a.nl; ++r) {
    const int a1 = a.nx[r] + 1, b1 = a.ny[r] + 1;
    T *c = sm + a.off_c[r];
    for (int k = threadIdx.x; k < a1; k += blockDim.x) { c[k] = a.W[r][k]; c[a1 + k] = a.E[r][k]; }
    for (int k = threadIdx.x; k < b1; k += blockDim.x) { c[2 * a1 + k] = a.S[r][k]; c[2 * a1 + b1 + k] = a.N[r][k]; }
    for (int bi = 0; bi < a.nbase && r < a.nl - 1; ++bi) {
      const PreRange &R = a.pr[r][bi];
      for (uint32_t k = threadIdx.x; k < R.na; k += blockDim.x) {
        sm[R.soff + k] = __ldg(a.cp + R.a0 + k);
        sm[R.soff + R.na + k] = __ldg(a.piv + R.a0 + k);
      }
      for (uint32_t k = threadIdx.x; k < R.nz; k += blockDim.x) sm[R.zoff + k] = __ldg(a.zb + R.z0 + k);
    }
  }
  __syncthreads();
  mini_cycle(a, sm, bsm);
  for (int k = threadIdx.x; k < n0; k += blockDim.x) ug[k] = U0[k];
}

// ---------------------------------------------------------------- host side

int opp(int d) { return d ^ 1; }
double hcoef(const Level &L, int i, int j, int d) {
  return d == DIR_PX ? L.hE[i] : d == DIR_MX ? L.hW[i] : d == DIR_PY ? L.hN[j] : L.hS[j];
}
double hcentre(const Level &L, int i, int j) { return -((L.hW[i] + L.hE[i]) + (L.hS[j] + L.hN[j])); }

struct WalkNode {
  int i, j, pd, sd;  // directions to the in-block predecessor / successor (-1: none)
};
void walk(const HChain &c, std::vector<WalkNode> &out) {
  out.clear();
  int i = c.s[0].i0, j = c.s[0].j0;
  const int ns = (int)c.s.size();
  for (int s = 0; s < ns; ++s) {
    const int d = c.s[s].dir, n = c.s[s].len;
    for (int t = 0; t < n; ++t) {
      if (!out.empty()) { i += d == DIR_PX ? 1 : d == DIR_MX ? -1 : 0; j += d == DIR_PY ? 1 : d == DIR_MY ? -1 : 0; }
      WalkNode w;
      w.i = i; w.j = j;
      w.pd = !out.empty() ? opp(d) : (c.fj ? opp(c.s[0].dir) : -1);
      w.sd = t < n - 1 ? d : (s < ns - 1 ? c.s[s + 1].dir : (c.lj ? c.ljdir : -1));
      out.push_back(w);
    }
  }
}

// Blocks of one base smoother and colour on level L, appended to the plan:
// descriptors, and per chain node c' and the pivot reciprocal (A arrays, plus
// one entry per junction) and, for junction blocks, zb (Z array).
struct PlanData {
  std::vector<MBlock> blocks;
  std::vector<double> cp, piv, zb;
};
void plan_blocks(const Level &L, int base, int colour, PlanData &D) {
  if (base == BASE_CHECKER) return;  // pointwise: no list
  std::vector<HBlock> hb;
  switch (base) {
    case BASE_ZEBRA_X: zebra_blocks(L.nx, L.ny, colour, true, hb); break;
    case BASE_ZEBRA_Y: zebra_blocks(L.nx, L.ny, colour, false, hb); break;
    case BASE_TWEED: tweed_blocks(L.nx, L.ny, colour, hb); break;
    default: wireframe_blocks(L.nx, L.ny, colour, hb); break;
  }
  std::vector<WalkNode> wn;
  for (const HBlock &h : hb) {
    MBlock B;
    std::memset(&B, 0, sizeof(B));
    B.ji = (uint16_t)h.ji; B.jj = (uint16_t)h.jj;
    B.junc = h.junc ? 1 : 0;
    B.nchain = (uint8_t)h.ch.size();
    B.pre0 = (uint32_t)D.cp.size();
    B.zb0 = (uint32_t)D.zb.size();
    double den = h.junc ? hcentre(L, h.ji, h.jj) : 0.0;
    for (size_t e = 0; e < h.ch.size(); ++e) {
      const HChain &c = h.ch[e];
      MChain &m = B.ch[e];
      m.i0 = (uint16_t)c.s[0].i0; m.j0 = (uint16_t)c.s[0].j0;
      m.nseg = (uint8_t)c.s.size();
      m.flags = (uint8_t)((c.fj ? 1 : 0) | (c.lj ? 2 : 0));
      m.ljdir = (uint8_t)c.ljdir;
      for (size_t s = 0; s < c.s.size(); ++s) { m.len[s] = (uint16_t)c.s[s].len; m.dir[s] = (uint8_t)c.s[s].dir; }
      walk(c, wn);
      const int n = (int)wn.size();
      std::vector<double> a(n), b(n), cc(n), cp(n), piv(n), z(n), rhs(n, 0.0);
      for (int k = 0; k < n; ++k) {
        const WalkNode &w = wn[k];
        a[k] = w.pd >= 0 ? hcoef(L, w.i, w.j, w.pd) : 0.0;
        cc[k] = w.sd >= 0 ? hcoef(L, w.i, w.j, w.sd) : 0.0;
        b[k] = hcentre(L, w.i, w.j);
      }
      // Thomas multipliers and pivots of the chain without its junction
      // couplings; response zb to a unit junction value
      if (c.fj) rhs[0] -= a[0];
      if (c.lj) rhs[n - 1] -= cc[n - 1];
      for (int k = 0; k < n; ++k) {
        piv[k] = 1.0 / (k > 0 ? b[k] - a[k] * cp[k - 1] : b[k]);
        cp[k] = k < n - 1 ? cc[k] * piv[k] : 0.0;
        z[k] = (k > 0 ? rhs[k] - a[k] * z[k - 1] : rhs[k]) * piv[k];
      }
      for (int k = n - 2; k >= 0; --k) z[k] -= cp[k] * z[k + 1];
      D.cp.insert(D.cp.end(), cp.begin(), cp.end());
      D.piv.insert(D.piv.end(), piv.begin(), piv.end());
      if (h.junc) D.zb.insert(D.zb.end(), z.begin(), z.end());
      if (c.fj) den += hcoef(L, h.ji, h.jj, c.s[0].dir) * z[0];
      if (c.lj) den += hcoef(L, h.ji, h.jj, opp(c.ljdir)) * z[n - 1];
    }
    if (h.junc) { D.cp.push_back(0.0); D.piv.push_back(1.0 / den); }
    D.blocks.push_back(B);
  }
}

size_t level_elems(const Level &L) { return 2 * L.nn + 2 * (size_t)(L.nx + 1) + 2 * (size_t)(L.ny + 1); }

// Base smoothers relaxed by smoother s (Sec. 2, Sec. 3).
int bases_of(int s, int *b) {
  switch (s) {
    case MG_SMOOTH_CHECKERBOARD: return 0;
    case MG_SMOOTH_ZEBRA_X: b[0] = BASE_ZEBRA_X; return 1;
    case MG_SMOOTH_ZEBRA_Y: b[0] = BASE_ZEBRA_Y; return 1;
    case MG_SMOOTH_ALT_ZEBRA: b[0] = BASE_ZEBRA_X; b[1] = BASE_ZEBRA_Y; return 2;
    case MG_SMOOTH_TWEED: b[0] = BASE_TWEED; return 1;
    case MG_SMOOTH_WIREFRAME: b[0] = BASE_WIREFRAME; return 1;
    default: b[0] = BASE_TWEED; b[1] = BASE_WIREFRAME; return 2;
  }
}

}  // namespace

mg_status build_mini(Grid &g, int prec) {
  MiniPlan &P = g.mini[prec];
  const size_t w = prec == 0 ? sizeof(double) : sizeof(float);
  if (g.nlev < 2) return MG_OK;
  const size_t head = sizeof(double) * ((g.cn + 1) & ~1);
  // candidate levels: at most MINI_MAX_LEV levels down to the coarsest whose
  // arrays alone fit in shared memory
  int l0 = -1;
  for (int l = g.nlev - 2; l >= 0 && g.nlev - l <= MINI_MAX_LEV; --l) {
    size_t e = 0;
    for (int k = l; k < g.nlev; ++k) e += level_elems(g.lev[k]);
    if (head + w * e > MINI_SMEM_MAX) break;
    l0 = l;
  }
  if (l0 < 0) return MG_OK;
  PlanData D;
  std::vector<uint2> tab;
  P.ranges.assign((size_t)(g.nlev - l0) * NBASE, {});
  for (int l = l0; l < g.nlev; ++l)
    for (int base = 0; base < NBASE; ++base) {
      MiniPlan::Range &R = P.ranges[(size_t)(l - l0) * NBASE + base];
      R.a0 = (uint32_t)D.cp.size(); R.z0 = (uint32_t)D.zb.size();
      for (int colour = 0; colour < 2; ++colour) {
        const uint32_t b0 = (uint32_t)D.blocks.size();
        if (l < g.nlev - 1) plan_blocks(g.lev[l], base, colour, D);
        tab.push_back(make_uint2(b0, (uint32_t)D.blocks.size() - b0));
      }
      R.na = (uint32_t)D.cp.size() - R.a0; R.nz = (uint32_t)D.zb.size() - R.z0;
    }
  if (D.cp.size() >= (size_t)UINT32_MAX) return MG_ERR_SIZE;
  P.level0 = l0;
  // per smoother: the finest level whose arrays and staged data fit
  size_t most = 0;
  for (int s = 0; s <= MG_SMOOTH_ALT_TW; ++s) {
    int b[2];
    const int nb = bases_of(s, b);
    P.level_for[s] = -1;
    for (int l = g.nlev - 2; l >= l0; --l) {
      size_t e = 0;
      for (int k = l; k < g.nlev; ++k) {
        e += level_elems(g.lev[k]);
        for (int q = 0; q < nb; ++q) {
          const MiniPlan::Range &R = P.ranges[(size_t)(k - l0) * NBASE + b[q]];
          e += 2 * (size_t)R.na + R.nz;
        }
      }
      const size_t bytes = head + w * e;
      if (bytes > MINI_SMEM_MAX) break;
      P.level_for[s] = l;
      P.smem_for[s] = bytes;
    }
    if (P.level_for[s] >= 0) most = std::max(most, P.smem_for[s]);
  }
  const size_t np = D.cp.size(), nz = D.zb.size();
  const size_t sb = sizeof(MBlock) * std::max<size_t>(D.blocks.size(), 1), st = sizeof(uint2) * tab.size();
  const size_t sa = (w * std::max<size_t>(np, 1) + 255) & ~size_t(255), sz = w * std::max<size_t>(nz, 1);
  const size_t o1 = (sb + 255) & ~size_t(255), o2 = (o1 + st + 255) & ~size_t(255);
  char *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, o2 + 2 * sa + sz);
  if (e != cudaSuccess) { set_error("cudaMalloc(coarse-cycle plan)", e); return MG_ERR_ALLOC; }
  P.mem = mem;
  P.blocks = reinterpret_cast<MBlock *>(mem);
  P.tab = reinterpret_cast<uint2 *>(mem + o1);
  P.pre[0] = mem + o2; P.pre[1] = mem + o2 + sa; P.pre[2] = mem + o2 + 2 * sa;
  if (!D.blocks.empty())
    e = cudaMemcpy(P.blocks, D.blocks.data(), sizeof(MBlock) * D.blocks.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P.tab, tab.data(), st, cudaMemcpyHostToDevice);
  const std::vector<double> *src[3] = {&D.cp, &D.piv, &D.zb};
  for (int v = 0; v < 3 && e == cudaSuccess; ++v) {
    if (src[v]->empty()) continue;
    if (prec == 0) {
      e = cudaMemcpy(P.pre[v], src[v]->data(), w * src[v]->size(), cudaMemcpyHostToDevice);
    } else {
      std::vector<float> pf(src[v]->begin(), src[v]->end());
      e = cudaMemcpy(P.pre[v], pf.data(), w * pf.size(), cudaMemcpyHostToDevice);
    }
  }
  if (e != cudaSuccess) { set_error("cudaMemcpy(coarse-cycle plan)", e); return MG_ERR_CUDA; }
  if (most > 0) {
    e = prec == 0
            ? cudaFuncSetAttribute(mini_cycle_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most)
            : cudaFuncSetAttribute(mini_cycle_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    if (e != cudaSuccess) { set_error("coarse-cycle kernel attributes", e); return MG_ERR_CUDA; }
  }
  return MG_OK;
}

template <typename T>
cudaError_t launch_mini_cycle(const Grid &g, const mg_params &p, T *u, const T *f, cudaStream_t s) {
  const MiniPlan &P = g.mini[sizeof(T) == 8 ? 0 : 1];
  const int m = P.level_for[p.smoother];
  MiniArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.nl = g.nlev - m;
  a.tl0 = m - P.level0;
  a.smoother = p.smoother; a.nu1 = p.nu1; a.nu2 = p.nu2; a.gamma = p.cycle; a.restriction = p.restriction;
  a.nbase = bases_of(p.smoother, a.base);
  size_t off = 0;  // elements of T after the coarse-solve buffer
  for (int r = 0; r < a.nl; ++r) {
    const Level &L = g.lev[m + r];
    a.nx[r] = L.nx; a.ny[r] = L.ny;
    a.off_u[r] = (int)off; off += L.nn;
    a.off_f[r] = (int)off; off += L.nn;
    a.off_c[r] = (int)off; off += 2 * (size_t)(L.nx + 1) + 2 * (size_t)(L.ny + 1);
    if (sizeof(T) == 8) {
      a.W[r] = (const T *)L.W64; a.E[r] = (const T *)L.E64; a.S[r] = (const T *)L.S64; a.N[r] = (const T *)L.N64;
    } else {
      a.W[r] = (const T *)L.W32; a.E[r] = (const T *)L.E32; a.S[r] = (const T *)L.S32; a.N[r] = (const T *)L.N32;
    }
  }
  for (int r = 0; r < a.nl - 1; ++r)
    for (int q = 0; q < a.nbase; ++q) {
      const MiniPlan::Range &R = P.ranges[(size_t)(m + r - P.level0) * NBASE + a.base[q]];
      PreRange &D = a.pr[r][q];
      D.a0 = R.a0; D.na = R.na; D.z0 = R.z0; D.nz = R.nz;
      D.soff = (int)off; off += 2 * (size_t)R.na;
      D.zoff = (int)off; off += R.nz;
    }
  a.blocks = P.blocks;
  a.cp = static_cast<const T *>(P.pre[0]);
  a.piv = static_cast<const T *>(P.pre[1]);
  a.zb = static_cast<const T *>(P.pre[2]);
  a.tab = P.tab;
  a.cinv = g.cinv;
  a.cn = g.cn;
  mini_cycle_kernel<T><<<1, MINI_THREADS, P.smem_for[p.smoother], s>>>(a, u, f);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_mini_cycle<double>(const Grid &, const mg_params &, double *, const double *,
                                               cudaStream_t);
template cudaError_t launch_mini_cycle<float>(const Grid &, const mg_params &, float *, const float *, cudaStream_t);

}  // namespace tmg
