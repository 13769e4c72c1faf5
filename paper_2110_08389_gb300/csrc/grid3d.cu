// grid3d.cu -- 3D grids (Sec. 7): the level hierarchy, the 3D tweed and
// wireframe blocks, their colour passes on the warp path (kernels in
// seq3.cuh), the 7-point defect with full-weighting restriction, trilinear
// prolongation, the coarsest direct solve, the FP64 norms and refinement
// steps, and the cycle of Sec. 4 on them.
//
// With the index distances to the nearer wall d_x = min(i, nx-i), d_y, d_z
// sorted as d1 <= d2 <= d3:
//   3D tweed (Sec. 7): lines run perpendicular to the nearest wall, starting
//     from the eight corner points.  A block is a connected set of interior
//     nodes with equal (d2, d3): a point, a line turning at most at its ends,
//     or a star of m = 3, 4 or 6 legs around one branch node (m = 6 at the
//     centre of a cube).  Red (relaxed first) when d2 + d3 is even, so the
//     corner points are red.
//   3D wireframe (Sec. 7): blocks cover the faces of concentric cuboids.  A
//     block is a connected set of interior nodes with equal (d1, d2): for
//     d1 < d2 a ring around the centre of a cuboid face (a line or a point
//     where the face's rings close), for d1 = d2 the twelve edges of the
//     cuboid with its eight corners (the wireframe itself).  Red when d1 + d2
//     is even, so the outermost skeleton is red.
// Adjacent nodes either share the key or differ by one in its sum (all sides
// even), so blocks of one colour never touch.  Transfers are the tensor
// products of the 1D factors of the 2D rules of Sec. 4: full weighting
// (1/4, 1/2, 1/4) per axis, trilinear prolongation.  Each block is solved
// exactly: lines, stars and rings on the warp path (a ring as the line left
// when one node is taken out, that node then a junction with two attached
// ends), skeletons by one CTA each (Thomas per edge, then the corners).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <functional>
#include <numeric>
#include <thread>
#include <vector>

#include "fp_bits.h"
#include "pack3_host.h"
#include "seq3.cuh"

namespace tmg {

namespace {

// ----------------------------------------------------------- transfers --
constexpr int T3 = 128;  // threads per CTA of the grid kernels (x along i)

// d = f - L u at the interior nodes of a level (boundary of d not written)
template <typename T>
__global__ void __launch_bounds__(T3) defect3_kernel(C6<T> c, int nx, int ny, int nz, const T *__restrict__ u,
                                                     const T *__restrict__ f, T *__restrict__ d) {
  pdl_trigger();
  const int i = 1 + blockIdx.x * T3 + threadIdx.x, j = 1 + blockIdx.y, k = 1 + blockIdx.z;
  const T ci = i < nx ? __ldg(c.W + i) : T(0), ce = i < nx ? __ldg(c.E + i) : T(0);
  const T cs = __ldg(c.S + j), cn = __ldg(c.N + j), cb = __ldg(c.B + k), ct = __ldg(c.T_ + k);
  pdl_wait();
  if (i >= nx) return;
  const int nx1 = nx + 1;
  const size_t plane = (size_t)nx1 * (ny + 1), p = (size_t)k * plane + (size_t)j * nx1 + i;
  const T cc = -((ci + ce) + (cs + cn) + (cb + ct));
  d[p] = f[p] - (ci * u[p - 1] + ce * u[p + 1] + cs * u[p - nx1] + cn * u[p + nx1] + cb * u[p - plane] +
                 ct * u[p + plane] + cc * u[p]);
}

// full weighting of the fine defect onto the coarse interior (tensor
// product of 1/4, 1/2, 1/4); the coarse correction uc is zeroed
template <typename T>
__global__ void __launch_bounds__(T3) restrict3_kernel(int nx, int ny, int nxc, int nyc, int nzc,
                                                       const T *__restrict__ d, T *__restrict__ fc,
                                                       T *__restrict__ uc) {
  pdl_trigger();
  pdl_wait();
  const int I = 1 + blockIdx.x * T3 + threadIdx.x, J = 1 + blockIdx.y, K = 1 + blockIdx.z;
  if (I >= nxc) return;
  const int nx1 = nx + 1;
  const size_t plane = (size_t)nx1 * (ny + 1);
  const T w[3] = {T(0.25), T(0.5), T(0.25)};
  T v = T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const T *row = d + (size_t)(2 * K + c - 1) * plane + (size_t)(2 * J + b - 1) * nx1 + 2 * I - 1;
      v += w[c] * w[b] * ((w[0] * row[0] + w[1] * row[1]) + w[2] * row[2]);
    }
  const size_t q = ((size_t)K * (nyc + 1) + J) * (nxc + 1) + I;
  fc[q] = v;
  if (uc) uc[q] = T(0);
}

// trilinear prolongation of the coarse correction, added to the fine interior
template <typename T>
__global__ void __launch_bounds__(T3) prolong3_kernel(int nx, int ny, int nxc, int nyc, const T *__restrict__ uc,
                                                      T *__restrict__ u) {
  pdl_trigger();
  pdl_wait();
  const int i = 1 + blockIdx.x * T3 + threadIdx.x, j = 1 + blockIdx.y, k = 1 + blockIdx.z;
  if (i >= nx) return;
  const int c1 = nxc + 1;
  const size_t cplane = (size_t)c1 * (nyc + 1);
  const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1, k1 = (k + 1) >> 1;
  const T wi = (i & 1) ? T(0.5) : T(1), wj = (j & 1) ? T(0.5) : T(1), wk = (k & 1) ? T(0.5) : T(1);
  // odd index: both coarse neighbours (weight 1/2 each); even: the coarse
  // node itself (i0 == i1, counted once)
  auto at = [&](int a, int b, int c) { return uc[(size_t)c * cplane + (size_t)b * c1 + a]; };
  T v = at(i0, j0, k0);
  if (i & 1) v += at(i1, j0, k0);
  if (j & 1) { v += at(i0, j1, k0); if (i & 1) v += at(i1, j1, k0); }
  if (k & 1) {
    T w2 = at(i0, j0, k1);
    if (i & 1) w2 += at(i1, j0, k1);
    if (j & 1) { w2 += at(i0, j1, k1); if (i & 1) w2 += at(i1, j1, k1); }
    v += w2;
  }
  u[((size_t)k * (ny + 1) + j) * (nx + 1) + i] += wi * wj * wk * v;
}

// coarsest level: x = A^{-1} b in FP64, b = f - boundary neighbours
constexpr int CS3_THREADS = 1024;
template <typename T>
__global__ void __launch_bounds__(CS3_THREADS) coarse3_kernel(C6<double> c, int nx, int ny, int nz,
                                                              const double *__restrict__ inv, T *__restrict__ u,
                                                              const T *__restrict__ f) {
  extern __shared__ double cb3[];
  pdl_trigger();
  pdl_wait();
  const int mx = nx - 1, my = ny - 1, n = mx * my * (nz - 1), nx1 = nx + 1;
  const size_t plane = (size_t)nx1 * (ny + 1);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int i = r % mx + 1, j = (r / mx) % my + 1, k = r / (mx * my) + 1;
    const size_t p = (size_t)k * plane + (size_t)j * nx1 + i;
    double b = (double)f[p];
    if (i == 1) b -= c.W[i] * (double)u[p - 1];
    if (i == nx - 1) b -= c.E[i] * (double)u[p + 1];
    if (j == 1) b -= c.S[j] * (double)u[p - nx1];
    if (j == ny - 1) b -= c.N[j] * (double)u[p + nx1];
    if (k == 1) b -= c.B[k] * (double)u[p - plane];
    if (k == nz - 1) b -= c.T_[k] * (double)u[p + plane];
    cb3[r] = b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int r = threadIdx.x >> 5; r < n; r += nw) {
    double x = 0.0;
    for (int q = lane; q < n; q += 32) x += inv[(size_t)r * n + q] * cb3[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      const int i = r % mx + 1, j = (r / mx) % my + 1, k = r / (mx * my) + 1;
      u[(size_t)k * plane + (size_t)j * nx1 + i] = (T)x;
    }
  }
}

// ------------------------------------------------------- FP64 norms etc --
constexpr int N3_THREADS = 256;

__device__ __forceinline__ double block_sum3(double s) {
  __shared__ double ss[N3_THREADS];
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int h = N3_THREADS / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) ss[threadIdx.x] += ss[threadIdx.x + h];
    __syncthreads();
  }
  return ss[0];
}

// Sum of squares of r = f - L u over the interior (bnd_only: r = f - B u_b,
// the boundary neighbours alone).  CTA b takes interior rows (j, k) with
// row index b, b + gridDim.x, ...; each thread its columns in order, so the
// sum does not depend on timing.  With r32: stores float(r), zeroes e32.
__global__ void __launch_bounds__(N3_THREADS) norm3_stage1(C6<double> c, int nx, int ny, int nz,
                                                           const double *__restrict__ u, const double *__restrict__ f,
                                                           int bnd_only, float *__restrict__ r32,
                                                           float *__restrict__ e32, double *__restrict__ part) {
  const int nx1 = nx + 1, rows = (ny - 1) * (nz - 1);
  const size_t plane = (size_t)nx1 * (ny + 1);
  double s = 0.0;
  for (int row = blockIdx.x; row < rows; row += gridDim.x) {
    const int j = 1 + row % (ny - 1), k = 1 + row / (ny - 1);
    const double cs = __ldg(c.S + j), cn = __ldg(c.N + j), cb = __ldg(c.B + k), ct = __ldg(c.T_ + k);
    const size_t base = (size_t)k * plane + (size_t)j * nx1;
    for (int i = 1 + threadIdx.x; i < nx; i += N3_THREADS) {
      const size_t p = base + i;
      double r = f[p];
      const double cw = __ldg(c.W + i), ce = __ldg(c.E + i);
      if (bnd_only) {
        if (i == 1) r -= cw * u[p - 1];
        if (i == nx - 1) r -= ce * u[p + 1];
        if (j == 1) r -= cs * u[p - nx1];
        if (j == ny - 1) r -= cn * u[p + nx1];
        if (k == 1) r -= cb * u[p - plane];
        if (k == nz - 1) r -= ct * u[p + plane];
      } else {
        const double cc = (cw + ce) + (cs + cn) + (cb + ct);
        r -= cw * u[p - 1] + ce * u[p + 1] + cs * u[p - nx1] + cn * u[p + nx1] + cb * u[p - plane] +
             ct * u[p + plane] - cc * u[p];
      }
      if (r32) { r32[p] = narrow_rne(r); e32[p] = 0.0f; }
      s = fma(r, r, s);
    }
  }
  s = block_sum3(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(N3_THREADS) norm3_stage2(const double *__restrict__ part, int npart,
                                                           double *__restrict__ out) {
  double s = 0.0;
  for (int k = threadIdx.x; k < npart; k += N3_THREADS) s += part[k];
  s = block_sum3(s);
  if (threadIdx.x == 0) out[0] = s;
}

// u64 += e32 (update = 1) or u64 := 0 (update = 0) at interior nodes
__global__ void __launch_bounds__(T3) interior3_kernel(int nx, int ny, double *__restrict__ u,
                                                       const float *__restrict__ e, int update) {
  const int i = 1 + blockIdx.x * T3 + threadIdx.x, j = 1 + blockIdx.y, k = 1 + blockIdx.z;
  if (i >= nx) return;
  const size_t p = ((size_t)k * (ny + 1) + j) * (nx + 1) + i;
  u[p] = update ? u[p] + widen_exact(e[p]) : 0.0;
}

dim3 interior_grid(const Level3 &L) { return dim3((L.nx - 1 + T3 - 1) / T3, L.ny - 1, L.nz - 1); }

// ------------------------------------------------------------ host setup --
// The warp lists of one colour on the device (pack3_host.h lays them out).
mg_status warp_list3(const Level3 &L, const std::vector<HBlock3> &all, int colour, bool multi, WarpList3 &Wl) {
  Pack3 pk;
  const mg_status st = pack3(L, all, colour, multi, pk);
  if (st != MG_OK) return st;
  if (pk.nwarp == 0 && pk.skel.empty()) return MG_OK;
  const std::vector<WNode3> &nodes = pk.nodes;
  const std::vector<WJunc3> &jn = pk.jn;
  const std::vector<int> &jofs = pk.jofs;
  const std::vector<WSkel3> &skel = pk.skel;
  auto al = [](size_t v) { return (v + 15) & ~size_t(15); };
  const size_t b_nodes = al(sizeof(WNode3) * nodes.size()), b_jn = al(sizeof(WJunc3) * jn.size()),
               b_jofs = al(sizeof(int) * jofs.size()), b_sk = al(sizeof(WSkel3) * skel.size());
  char *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, b_nodes + b_jn + b_jofs + b_sk);
  if (e != cudaSuccess) { set_error("cudaMalloc(3D warp list)", e); return MG_ERR_ALLOC; }
  Wl.mem = mem;
  Wl.node = reinterpret_cast<WNode3 *>(mem);
  Wl.junc = reinterpret_cast<WJunc3 *>(mem + b_nodes);
  Wl.jofs = reinterpret_cast<int *>(mem + b_nodes + b_jn);
  Wl.skel = reinterpret_cast<WSkel3 *>(mem + b_nodes + b_jn + b_jofs);
  if (!nodes.empty()) e = cudaMemcpy(Wl.node, nodes.data(), sizeof(WNode3) * nodes.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !jn.empty()) e = cudaMemcpy(Wl.junc, jn.data(), sizeof(WJunc3) * jn.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(Wl.jofs, jofs.data(), sizeof(int) * jofs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !skel.empty()) e = cudaMemcpy(Wl.skel, skel.data(), sizeof(WSkel3) * skel.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { set_error("cudaMemcpy(3D warp list)", e); return MG_ERR_CUDA; }
  Wl.nwarp = pk.nwarp;
  Wl.K = pk.K;
  Wl.W = pk.W;
  Wl.total_nodes = pk.total_nodes;
  Wl.nskel = (int)skel.size();
  Wl.skel_nodes = pk.skel_nodes;
  Wl.multi = multi;
  return MG_OK;
}

template <typename T>
T *lev_u(Grid &g, int l);
template <>
double *lev_u<double>(Grid &g, int l) { return g.g3->lev[l].u64; }
template <>
float *lev_u<float>(Grid &g, int l) { return g.g3->lev[l].u32; }
template <typename T>
T *lev_f(Grid &g, int l);
template <>
double *lev_f<double>(Grid &g, int l) { return g.g3->lev[l].f64; }
template <>
float *lev_f<float>(Grid &g, int l) { return g.g3->lev[l].f32; }
template <typename T>
T *defect_scratch(Grid &g);
template <>
double *defect_scratch<double>(Grid &g) { return g.g3->d64; }
template <>
float *defect_scratch<float>(Grid &g) { return g.g3->d32; }

}  // namespace

// --------------------------------------------------------------- entries --

mg_status setup3(Grid &g, const int64_t *n, const double *const *coords) {
  g.dim = 3;
  g.g3 = new (std::nothrow) Grid3;
  if (!g.g3) return MG_ERR_ALLOC;
  Grid3 &G = *g.g3;
  int cx = (int)n[0], cy = (int)n[1], cz = (int)n[2];
  std::vector<double> xs(coords[0], coords[0] + cx + 1), ys(coords[1], coords[1] + cy + 1),
      zs(coords[2], coords[2] + cz + 1);
  while (true) {
    Level3 L;
    L.nx = cx; L.ny = cy; L.nz = cz;
    L.nn = (size_t)(cx + 1) * (cy + 1) * (cz + 1);
    L.hx = xs; L.hy = ys; L.hz = zs;
    axis_coefficients(xs, L.hc[0], L.hc[1]);
    axis_coefficients(ys, L.hc[2], L.hc[3]);
    axis_coefficients(zs, L.hc[4], L.hc[5]);
    G.lev.push_back(std::move(L));
    if (cx % 2 || cy % 2 || cz % 2 || cx / 2 < 2 || cy / 2 < 2 || cz / 2 < 2 || std::max(cx, std::max(cy, cz)) <= 8)
      break;
    std::vector<double> xn(cx / 2 + 1), yn(cy / 2 + 1), zn(cz / 2 + 1);
    for (int i = 0; i <= cx / 2; ++i) xn[i] = xs[2 * i];
    for (int j = 0; j <= cy / 2; ++j) yn[j] = ys[2 * j];
    for (int k = 0; k <= cz / 2; ++k) zn[k] = zs[2 * k];
    xs.swap(xn); ys.swap(yn); zs.swap(zn);
    cx /= 2; cy /= 2; cz /= 2;
  }
  g.nlev = (int)G.lev.size();
  TRY_CUDA("3D kernel attributes", prepare3_t<false>());
  TRY_CUDA("3D kernel attributes", prepare_seq3_multi());
  const bool want64 = g.prec_mask & 1, want32 = g.prec_mask & 2;
  for (int l = 0; l < g.nlev; ++l) {
    Level3 &L = G.lev[l];
    const size_t len[6] = {(size_t)L.nx + 1, (size_t)L.nx + 1, (size_t)L.ny + 1, (size_t)L.ny + 1,
                           (size_t)L.nz + 1, (size_t)L.nz + 1};
    size_t tot = 0;
    for (int a = 0; a < 6; ++a) tot += len[a];
    TRY_CUDA("cudaMalloc(3D coefficients)", cudaMalloc(&L.dev_block, tot * (sizeof(double) + sizeof(float)) + 16));
    double *dp = static_cast<double *>(L.dev_block);
    float *fp = reinterpret_cast<float *>(dp + tot);
    std::vector<double> hd;
    std::vector<float> hf;
    for (int a = 0; a < 6; ++a) {
      L.c64[a] = dp + hd.size();
      L.c32[a] = fp + hf.size();
      for (double v : L.hc[a]) { hd.push_back(v); hf.push_back((float)v); }
    }
    TRY_CUDA("cudaMemcpy(3D coefficients)", cudaMemcpy(dp, hd.data(), sizeof(double) * tot, cudaMemcpyHostToDevice));
    TRY_CUDA("cudaMemcpy(3D coefficients)", cudaMemcpy(fp, hf.data(), sizeof(float) * tot, cudaMemcpyHostToDevice));
    if (l > 0) {
      if (want64) {
        TRY_CUDA("cudaMalloc(3D level)", cudaMalloc(&L.u64, sizeof(double) * L.nn));
        TRY_CUDA("cudaMalloc(3D level)", cudaMalloc(&L.f64, sizeof(double) * L.nn));
        TRY_CUDA("cudaMemset(3D level)", cudaMemset(L.u64, 0, sizeof(double) * L.nn));
        TRY_CUDA("cudaMemset(3D level)", cudaMemset(L.f64, 0, sizeof(double) * L.nn));
      }
      if (want32) {
        TRY_CUDA("cudaMalloc(3D level)", cudaMalloc(&L.u32, sizeof(float) * L.nn));
        TRY_CUDA("cudaMalloc(3D level)", cudaMalloc(&L.f32, sizeof(float) * L.nn));
        TRY_CUDA("cudaMemset(3D level)", cudaMemset(L.u32, 0, sizeof(float) * L.nn));
        TRY_CUDA("cudaMemset(3D level)", cudaMemset(L.f32, 0, sizeof(float) * L.nn));
      }
    }
    // tweed and wireframe blocks of the smoothed levels
    if (l + 1 < g.nlev) {
      // the two builds are independent host work: the wireframe one runs on
      // a second thread
      std::vector<HBlock3> blocks, wblocks;
      bool wf_ok = false;
      std::thread wf([&] { wf_ok = blocks3(L, SM3_WIREFRAME, wblocks); });
      const bool tw_ok = blocks3(L, SM3_TWEED, blocks);
      wf.join();
      if (!tw_ok) {
        set_error_text("3D tweed: a side with an odd number of intervals on a smoothed level");
        return MG_ERR_UNSUPPORTED;
      }
      for (int c = 0; c < 2; ++c) TRY(warp_list3(L, blocks, c, false, L.wp[SM3_TWEED][c]));
      if (std::min(L.nx, std::min(L.ny, L.nz)) >= T3_MIN_SIDE) TRY(build_tiles3(g, L, blocks, &L.t3_ok));
      L.wf_ok = wf_ok;
      if (L.wf_ok)
        for (int c = 0; c < 2; ++c) {
          TRY(warp_list3(L, wblocks, c, true, L.wp[SM3_WIREFRAME][c]));
          G.skel_len = std::max(G.skel_len, (size_t)L.wp[SM3_WIREFRAME][c].skel_nodes);
        }
    }
  }
  // coarsest level: dense inverse of the interior operator
  {
    const Level3 &L = G.lev[g.nlev - 1];
    const int mx = L.nx - 1, my = L.ny - 1, mz = L.nz - 1, m = mx * my * mz;
    if (m > 1024) return MG_ERR_SIZE;
    G.cn = m;
    std::vector<double> A((size_t)m * m, 0.0), inv;
    for (int k = 1; k < L.nz; ++k)
      for (int j = 1; j < L.ny; ++j)
        for (int i = 1; i < L.nx; ++i) {
          const int r = ((k - 1) * my + (j - 1)) * mx + (i - 1);
          A[(size_t)r * m + r] = -(L.hc[0][i] + L.hc[1][i] + L.hc[2][j] + L.hc[3][j] + L.hc[4][k] + L.hc[5][k]);
          if (i > 1) A[(size_t)r * m + r - 1] = L.hc[0][i];
          if (i < L.nx - 1) A[(size_t)r * m + r + 1] = L.hc[1][i];
          if (j > 1) A[(size_t)r * m + r - mx] = L.hc[2][j];
          if (j < L.ny - 1) A[(size_t)r * m + r + mx] = L.hc[3][j];
          if (k > 1) A[(size_t)r * m + r - mx * my] = L.hc[4][k];
          if (k < L.nz - 1) A[(size_t)r * m + r + mx * my] = L.hc[5][k];
        }
    if (!invert(m, A, inv)) return MG_ERR_SIZE;
    TRY_CUDA("cudaMalloc(3D coarse)", cudaMalloc(&G.cinv, sizeof(double) * inv.size()));
    TRY_CUDA("cudaMemcpy(3D coarse)", cudaMemcpy(G.cinv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice));
  }
  const size_t nn0 = G.lev[0].nn;
  if (g.tile_cap > 0) {
    // scratch of the 3D tiled path, laid out as the 2D one's (api.cu), FP64 sized
    TRY_CUDA("cudaMalloc(tile rows)", cudaMalloc(&g.tile_rows, g.tile_cap * 32 * 2 * 6 * sizeof(double)));
    TRY_CUDA("cudaMalloc(tile rhs)", cudaMalloc(&g.tile_d, g.tile_cap * 32 * 32 * sizeof(double)));
    TRY_CUDA("cudaMalloc(tile ends)", cudaMalloc(&g.tile_x, g.tile_cap * 32 * 2 * sizeof(double)));
  }
  if (G.skel_len > 0)
    TRY_CUDA("cudaMalloc(3D skeleton scratch)", cudaMalloc(&G.skel_scr, sizeof(double) * 6 * G.skel_len));
  if (want64) TRY_CUDA("cudaMalloc(3D defect)", cudaMalloc(&G.d64, sizeof(double) * nn0));
  if (want32) {
    TRY_CUDA("cudaMalloc(3D defect)", cudaMalloc(&G.d32, sizeof(float) * nn0));
    TRY_CUDA("cudaMalloc(e32)", cudaMalloc(&g.e32, sizeof(float) * nn0));
    TRY_CUDA("cudaMalloc(r32)", cudaMalloc(&g.r32, sizeof(float) * nn0));
    TRY_CUDA("cudaMemset(e32)", cudaMemset(g.e32, 0, sizeof(float) * nn0));
    TRY_CUDA("cudaMemset(r32)", cudaMemset(g.r32, 0, sizeof(float) * nn0));
    if (g.tile_cap > 0) TRY_CUDA("3D tile couple constants", setup_couple_consts3(g));
  }
  return MG_OK;
}

void free3(Grid &g) {
  if (!g.g3) return;
  for (Level3 &L : g.g3->lev) {
    cudaFree(L.dev_block);
    cudaFree(L.u64); cudaFree(L.f64); cudaFree(L.u32); cudaFree(L.f32);
    for (int m = 0; m < 2; ++m)
      for (int c = 0; c < 2; ++c) cudaFree(L.wp[m][c].mem);
    for (int c = 0; c < 2; ++c) cudaFree(L.t3[c].mem);
  }
  cudaFree(g.g3->cinv);
  cudaFree(g.g3->skel_scr);
  cudaFree(g.g3->d64);
  cudaFree(g.g3->d32);
  delete g.g3;
  g.g3 = nullptr;
}

template <typename T>
mg_status colour_pass3(Grid &g, int l, int sm, int colour, T *u, const T *f, cudaStream_t s) {
  Level3 &L = g.g3->lev[l];
  if (l + 1 >= g.nlev) return MG_ERR_UNSUPPORTED;  // the coarsest level is solved directly
  if (sm == SM3_WIREFRAME && !L.wf_ok) {
    set_error_text("3D wireframe: a block of this level is not a ring, line, point or cuboid edge skeleton");
    return MG_ERR_UNSUPPORTED;
  }
  if (sm == SM3_TWEED && tiled3(L))
    return cuda_status("3D tweed pass (tiled)", launch_tile3_pass<T>(g, L, L.t3[colour], u, f, s));
  return cuda_status(sm == SM3_WIREFRAME ? "3D wireframe pass" : "3D tweed pass",
                     L.wp[sm][colour].multi ? launch_seq3_multi<T>(*g.g3, L, L.wp[sm][colour], u, f, s)
                                            : launch_warp3_t<T, false>(*g.g3, L, L.wp[sm][colour], u, f, s));
}

template <typename T>
mg_status residual3(Grid &g, int l, const T *u, const T *f, T *d, cudaStream_t s) {
  const Level3 &L = g.g3->lev[l];
  TRY_CUDA("cudaMemsetAsync(3D defect)", cudaMemsetAsync(d, 0, sizeof(T) * L.nn, s));
  count_launch(1);
  return cuda_status("3D defect", launch_pdl(defect3_kernel<T>, interior_grid(L), dim3(T3), 0, s, coefs3<T>(L), L.nx,
                                             L.ny, L.nz, u, f, d));
}

template <typename T>
mg_status residual_restrict3(Grid &g, int l, const T *u, const T *f, T *fc, T *uc, cudaStream_t s) {
  const Level3 &F = g.g3->lev[l], &C = g.g3->lev[l + 1];
  T *d = defect_scratch<T>(g);
  count_launch(2);
  TRY_CUDA("3D defect", launch_pdl(defect3_kernel<T>, interior_grid(F), dim3(T3), 0, s, coefs3<T>(F), F.nx, F.ny,
                                   F.nz, u, f, d));
  return cuda_status("3D restriction", launch_pdl(restrict3_kernel<T>, interior_grid(C), dim3(T3), 0, s, F.nx, F.ny,
                                                  C.nx, C.ny, C.nz, (const T *)d, fc, uc));
}

template <typename T>
mg_status prolong_add3(Grid &g, int l, const T *uc, T *u, cudaStream_t s) {
  const Level3 &F = g.g3->lev[l], &C = g.g3->lev[l + 1];
  count_launch(1);
  return cuda_status("3D prolongation", launch_pdl(prolong3_kernel<T>, interior_grid(F), dim3(T3), 0, s, F.nx, F.ny,
                                                   C.nx, C.ny, uc, u));
}

template <typename T>
mg_status coarse_solve3(Grid &g, T *u, const T *f, cudaStream_t s) {
  const Level3 &L = g.g3->lev[g.nlev - 1];
  if (g.g3->cn <= 0) return MG_OK;
  count_launch(1);
  return cuda_status("3D coarse solve", launch_pdl(coarse3_kernel<T>, dim3(1), dim3(CS3_THREADS),
                                                   sizeof(double) * g.g3->cn, s, coefs3<double>(L), L.nx, L.ny, L.nz,
                                                   (const double *)g.g3->cinv, u, f));
}

// One relaxation (red pass, black pass; alternating tweed/wireframe: one of
// each) and the cycle of Sec. 4 steps (2)-(6).
template <typename T>
mg_status smooth3(Grid &g, int l, int smoother, T *u, const T *f, cudaStream_t s) {
  if (smoother == MG_SMOOTH_ALT_TW) {
    TRY(smooth3<T>(g, l, MG_SMOOTH_TWEED, u, f, s));
    return smooth3<T>(g, l, MG_SMOOTH_WIREFRAME, u, f, s);
  }
  const int sm = smoother == MG_SMOOTH_WIREFRAME ? SM3_WIREFRAME : SM3_TWEED;
  TRY(colour_pass3<T>(g, l, sm, 0, u, f, s));
  return colour_pass3<T>(g, l, sm, 1, u, f, s);
}

template <typename T>
mg_status cycle3(Grid &g, const mg_params &p, int l, T *u, const T *f, cudaStream_t s) {
  if (l == g.nlev - 1) return coarse_solve3<T>(g, u, f, s);
  for (int k = 0; k < p.nu1; ++k) TRY(smooth3<T>(g, l, p.smoother, u, f, s));
  T *uc = lev_u<T>(g, l + 1), *fc = lev_f<T>(g, l + 1);
  TRY(residual_restrict3<T>(g, l, u, f, fc, uc, s));
  for (int k = 0; k < p.cycle; ++k) TRY(cycle3<T>(g, p, l + 1, uc, fc, s));
  TRY(prolong_add3<T>(g, l, uc, u, s));
  for (int k = 0; k < p.nu2; ++k) TRY(smooth3<T>(g, l, p.smoother, u, f, s));
  return MG_OK;
}

mg_status zero_interior3(Grid &g, double *u, cudaStream_t s) {
  const Level3 &L = g.g3->lev[0];
  interior3_kernel<<<interior_grid(L), T3, 0, s>>>(L.nx, L.ny, u, nullptr, 0);
  count_launch(1);
  return cuda_status("3D zero interior", cudaGetLastError());
}

mg_status ir_update3(Grid &g, double *u, const float *e, cudaStream_t s) {
  const Level3 &L = g.g3->lev[0];
  interior3_kernel<<<interior_grid(L), T3, 0, s>>>(L.nx, L.ny, u, e, 1);
  count_launch(1);
  return cuda_status("3D refinement update", cudaGetLastError());
}

mg_status norms3(Grid &g, const double *u, const double *f, int bnd_only, float *r32, float *e32, cudaStream_t s) {
  const Level3 &L = g.g3->lev[0];
  norm3_stage1<<<g.npartial, N3_THREADS, 0, s>>>(coefs3<double>(L), L.nx, L.ny, L.nz, u, f, bnd_only, r32, e32,
                                                 g.partial);
  norm3_stage2<<<1, N3_THREADS, 0, s>>>(g.partial, g.npartial, g.scal);
  count_launch(2);
  return cuda_status("3D norms", cudaGetLastError());
}

template mg_status colour_pass3<double>(Grid &, int, int, int, double *, const double *, cudaStream_t);
template mg_status colour_pass3<float>(Grid &, int, int, int, float *, const float *, cudaStream_t);
template mg_status cycle3<double>(Grid &, const mg_params &, int, double *, const double *, cudaStream_t);
template mg_status cycle3<float>(Grid &, const mg_params &, int, float *, const float *, cudaStream_t);
template mg_status residual3<double>(Grid &, int, const double *, const double *, double *, cudaStream_t);
template mg_status residual3<float>(Grid &, int, const float *, const float *, float *, cudaStream_t);
template mg_status residual_restrict3<double>(Grid &, int, const double *, const double *, double *, double *,
                                              cudaStream_t);
template mg_status residual_restrict3<float>(Grid &, int, const float *, const float *, float *, float *, cudaStream_t);
template mg_status prolong_add3<double>(Grid &, int, const double *, double *, cudaStream_t);
template mg_status prolong_add3<float>(Grid &, int, const float *, float *, cudaStream_t);
template mg_status coarse_solve3<double>(Grid &, double *, const double *, cudaStream_t);
template mg_status coarse_solve3<float>(Grid &, float *, const float *, cudaStream_t);

}  // namespace tmg
