// transfer.cu -- defect, restriction, prolongation, coarsest solve, norms and
// the iterative-refinement kernels of tweedmg (sm_103a).
//
//   residual_kernel          d = f - L u (Sec. 4 step (3)), boundary 0
//   residual_restrict_kernel defect and its half / full weighting restriction
//                            fused (the storage-free fusion of Sec. 4), plus
//                            zeroing of the coarse correction
//   prolong_add_kernel       bilinear prolongation added to u (Sec. 4 step
//                            (5), fused as the paper suggests)
//   coarse_solve_kernel      u = L_0^{-1} (f - boundary terms) with the dense
//                            inverse prepared at setup (FP64)
//   resnorm                  FP64 sum of squares of the defect with a
//                            fixed-order reduction (deterministic)
//   refine_residual          the refinement step's update and FP64 residual
//                            in one launch (u + e, f - L(u + e), its FP32
//                            copy and norm), the iterate alternating between
//                            two FP64 arrays
#include <algorithm>

#include "fp_bits.h"
#include "packed.h"

namespace tmg {

template <typename T>
using CoefQ = Coefs<T>;
template <typename T>
static CoefQ<T> cq(const Level &L) {
  return level_coefs<T>(L);
}

// Defect at interior node (i, j): f - (W u_w + E u_e + S u_s + N u_n + C u).
template <typename T>
__device__ __forceinline__ T defect_at(const CoefQ<T> &c, const T *__restrict__ u, const T *__restrict__ f,
                                       int i, int j, int nx1) {
  const size_t p = (size_t)j * nx1 + i;
  const T w = __ldg(c.W + i), e = __ldg(c.E + i), s = __ldg(c.S + j), n = __ldg(c.N + j);
  const T cc = -((w + e) + (s + n));
  return f[p] - (w * u[p - 1] + e * u[p + 1] + s * u[p - nx1] + n * u[p + nx1] + cc * u[p]);
}

template <typename T>
__global__ void residual_kernel(CoefQ<T> c, int nx, int ny, const T *__restrict__ u, const T *__restrict__ f,
                                T *__restrict__ d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i > nx) return;
  const int nx1 = nx + 1;
  T v = T(0);
  if (i > 0 && i < nx && j > 0 && j < ny) v = defect_at(c, u, f, i, j, nx1);
  d[(size_t)j * nx1 + i] = v;
}

template <typename T>
cudaError_t launch_residual(const Level &L, const T *u, const T *f, T *d, cudaStream_t s) {
  dim3 b(128), g((L.nx + 1 + 127) / 128, L.ny + 1);
  residual_kernel<T><<<g, b, 0, s>>>(cq<T>(L), L.nx, L.ny, u, f, d);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_residual<double>(const Level &, const double *, const double *, double *, cudaStream_t);
template cudaError_t launch_residual<float>(const Level &, const float *, const float *, float *, cudaStream_t);

// One CTA per strip of RR_J coarse rows x RR_I coarse columns.  Every coarse
// interior node (I, J) takes the defects of fine node (2I, 2J) and its 8
// neighbours, all of them interior fine nodes; each fine defect of the strip
// is computed once into shared memory (fine rows 2J0-1 .. 2J0+2RR_J-1, fine
// columns 2I0-1 .. 2I0+2RR_I-1), then combined.  kind: 0 = half weighting
// (1/2, 1/8 x 4), 1 = full weighting (1/4, 1/8 x 4, 1/16 x 4).  The coarse
// correction uc is zeroed on the way.
constexpr int RR_I = 127, RR_J = 4, RR_THREADS = 256;  // 2 RR_I + 1 fine columns <= threads: one each
constexpr int RR_FI = 2 * RR_I + 1, RR_FJ = 2 * RR_J + 1;

template <typename T>
__global__ void __launch_bounds__(RR_THREADS) residual_restrict_kernel(CoefQ<T> c, int nx, int ny, int nxc,
                                                                       int nyc, int kind,
                                                                       const T *__restrict__ u,
                                                                       const T *__restrict__ f,
                                                                       T *__restrict__ fc, T *__restrict__ uc,
                                                                       const RRArgs<T> *__restrict__ tab,
                                                                       const int *__restrict__ active) {
  __shared__ T dd[RR_FJ][RR_FI + 1];
  if (tab) {  // packed launch: blockIdx.z selects the problem
    if (!active[blockIdx.z]) return;
    const RRArgs<T> a = tab[blockIdx.z];
    c = a.c; u = a.u; f = a.f; fc = a.fc; uc = a.uc;
  }
  pdl_trigger();
  pdl_wait();
  const int I0 = 1 + blockIdx.x * RR_I, J0 = 1 + blockIdx.y * RR_J;
  const int fi0 = 2 * I0 - 1, fj0 = 2 * J0 - 1, nx1 = nx + 1;
  // fine nodes of the strip that some coarse interior node of it uses
  const int fi_end = min(fi0 + RR_FI, nx), fj_end = min(fj0 + RR_FJ, ny);
  // thread = fine column: its 11 u values down the column, the 9 left and
  // right neighbours and 9 f values are all loaded before any is used (rows
  // clamped into the array; defects only for rows of the strip)
  for (int tcol = threadIdx.x; tcol < RR_FI; tcol += RR_THREADS) {
    const int i = fi0 + tcol;
    if (i >= fi_end) continue;
    const T w = c.W[i], e = c.E[i];
    T uc[RR_FJ + 2], ul[RR_FJ], ur[RR_FJ], ff[RR_FJ], sv[RR_FJ], nv[RR_FJ];
#pragma unroll
    for (int r = 0; r < RR_FJ + 2; ++r) uc[r] = u[(size_t)min(fj0 - 1 + r, ny) * nx1 + i];
#pragma unroll
    for (int r = 0; r < RR_FJ; ++r) {
      const int j = min(fj0 + r, ny - 1);
      const size_t p = (size_t)j * nx1 + i;
      ul[r] = u[p - 1];
      ur[r] = u[p + 1];
      ff[r] = f[p];
      sv[r] = c.S[j];
      nv[r] = c.N[j];
    }
#pragma unroll
    for (int r = 0; r < RR_FJ; ++r)
      if (fj0 + r < fj_end) {
        const T cc = -((w + e) + (sv[r] + nv[r]));
        dd[r][tcol] = ff[r] - (w * ul[r] + e * ur[r] + sv[r] * uc[r] + nv[r] * uc[r + 2] + cc * uc[r + 1]);
      }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < RR_I * RR_J; k += RR_THREADS) {
    const int li = k % RR_I, lj = k / RR_I;
    const int I = I0 + li, J = J0 + lj;
    if (I >= nxc || J >= nyc) continue;
    const int ci = 2 * li + 1, cj = 2 * lj + 1;  // the centre's place in dd
    const T centre = dd[cj][ci];
    const T edge = (dd[cj][ci - 1] + dd[cj - 1][ci]) + (dd[cj][ci + 1] + dd[cj + 1][ci]);
    T v;
    if (kind == MG_RESTRICT_HW) {
      v = T(0.5) * centre + T(0.125) * edge;
    } else {
      const T corner = (dd[cj - 1][ci - 1] + dd[cj - 1][ci + 1]) + (dd[cj + 1][ci - 1] + dd[cj + 1][ci + 1]);
      v = T(0.25) * centre + T(0.125) * edge + T(0.0625) * corner;
    }
    const size_t q = (size_t)J * (nxc + 1) + I;
    fc[q] = v;
    if (uc) uc[q] = T(0);
  }
}

template <typename T>
cudaError_t launch_residual_restrict(const Level &F, const Level &C, int kind, const T *u, const T *f, T *fc,
                                     T *uc, cudaStream_t s) {
  if (C.nx < 2 || C.ny < 2) return cudaSuccess;
  dim3 g((C.nx - 1 + RR_I - 1) / RR_I, (C.ny - 1 + RR_J - 1) / RR_J);
  count_launch(1);
  return launch_pdl(residual_restrict_kernel<T>, g, dim3(RR_THREADS), 0, s, cq<T>(F), F.nx, F.ny, C.nx, C.ny, kind,
                    u, f, fc, uc, (const RRArgs<T> *)nullptr, (const int *)nullptr);
}
template <typename T>
cudaError_t launch_residual_restrict_packed(const Level &F, const Level &C, int kind, const PackedLaunch &pk,
                                            cudaStream_t s) {
  if (C.nx < 2 || C.ny < 2 || pk.count == 0) return cudaSuccess;
  dim3 g((C.nx - 1 + RR_I - 1) / RR_I, (C.ny - 1 + RR_J - 1) / RR_J, pk.count);
  count_launch(1);
  return launch_pdl(residual_restrict_kernel<T>, g, dim3(RR_THREADS), 0, s, cq<T>(F), F.nx, F.ny, C.nx, C.ny, kind,
                    (const T *)nullptr, (const T *)nullptr, (T *)nullptr, (T *)nullptr,
                    static_cast<const RRArgs<T> *>(pk.tab), pk.active);
}
template cudaError_t launch_residual_restrict_packed<float>(const Level &, const Level &, int, const PackedLaunch &,
                                                            cudaStream_t);
template cudaError_t launch_residual_restrict_packed<double>(const Level &, const Level &, int, const PackedLaunch &,
                                                             cudaStream_t);
template cudaError_t launch_residual_restrict<double>(const Level &, const Level &, int, const double *,
                                                      const double *, double *, double *, cudaStream_t);
template cudaError_t launch_residual_restrict<float>(const Level &, const Level &, int, const float *,
                                                     const float *, float *, float *, cudaStream_t);

// Bilinear interpolation of the coarse correction (index-based weights,
// Sec. 4), added to the fine interior.  Thread (I, j) owns the fine pair
// (2I-1, j), (2I, j), I = 1..nxc, which uses coarse columns I-1 and I of
// coarse rows j/2 (and j/2 + 1 for odd j): no divergence between lanes, and
// the loads of a warp are contiguous.
constexpr int PR_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(PR_THREADS) prolong_add_kernel(int nx, int ny, int nxc, const T *__restrict__ uc,
                                                                 T *__restrict__ u,
                                                                 const ProlongArgs<T> *__restrict__ tab,
                                                                 const int *__restrict__ active) {
  if (tab) {  // packed launch: blockIdx.z selects the problem
    if (!active[blockIdx.z]) return;
    const ProlongArgs<T> a = tab[blockIdx.z];
    uc = a.uc; u = a.u;
  }
  pdl_trigger();
  pdl_wait();
  const int j = blockIdx.y + 1;
  const int c1 = nxc + 1, Jc = j >> 1;
  const bool jodd = j & 1;
  const T *r0 = uc + (size_t)Jc * c1, *r1 = r0 + (jodd ? c1 : 0);
  T *ur = u + (size_t)j * (nx + 1);
  for (int I = 1 + blockIdx.x * PR_THREADS + threadIdx.x; I <= nxc; I += gridDim.x * PR_THREADS) {
    const T a0 = r0[I - 1], b0 = r0[I];
    T vo, ve;
    if (jodd) {
      const T a1 = r1[I - 1], b1 = r1[I];
      vo = T(0.25) * ((a0 + b0) + (a1 + b1));
      ve = T(0.5) * (b0 + b1);
    } else {
      vo = T(0.5) * (a0 + b0);
      ve = b0;
    }
    ur[2 * I - 1] += vo;
    if (2 * I < nx) ur[2 * I] += ve;
  }
}

template <typename T>
cudaError_t launch_prolong_add(const Level &F, const Level &C, const T *uc, T *u, cudaStream_t s) {
  const int bx = std::min((C.nx + PR_THREADS - 1) / PR_THREADS, 8);
  dim3 g(bx, F.ny - 1);
  count_launch(1);
  return launch_pdl(prolong_add_kernel<T>, g, dim3(PR_THREADS), 0, s, F.nx, F.ny, C.nx, uc, u,
                    (const ProlongArgs<T> *)nullptr, (const int *)nullptr);
}
template <typename T>
cudaError_t launch_prolong_add_packed(const Level &F, const Level &C, const PackedLaunch &pk, cudaStream_t s) {
  if (pk.count == 0) return cudaSuccess;
  const int bx = std::min((C.nx + PR_THREADS - 1) / PR_THREADS, 8);
  dim3 g(bx, F.ny - 1, pk.count);
  count_launch(1);
  return launch_pdl(prolong_add_kernel<T>, g, dim3(PR_THREADS), 0, s, F.nx, F.ny, C.nx, (const T *)nullptr,
                    (T *)nullptr, static_cast<const ProlongArgs<T> *>(pk.tab), pk.active);
}
template cudaError_t launch_prolong_add_packed<float>(const Level &, const Level &, const PackedLaunch &,
                                                      cudaStream_t);
template cudaError_t launch_prolong_add_packed<double>(const Level &, const Level &, const PackedLaunch &,
                                                       cudaStream_t);
template cudaError_t launch_prolong_add<double>(const Level &, const Level &, const double *, double *,
                                                cudaStream_t);
template cudaError_t launch_prolong_add<float>(const Level &, const Level &, const float *, float *,
                                               cudaStream_t);

// Coarsest level: x = A^{-1} b in FP64, b = f - (boundary neighbours).  One
// CTA; unknown index (j-1)(nx-1) + (i-1).  One warp per row of A^{-1}, its
// lanes over the columns (coalesced loads), fixed-order shuffle reduction.
constexpr int CS_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(CS_THREADS) coarse_solve_kernel(CoefQ<double> c, int nx, int ny,
                                                                  const double *__restrict__ inv,
                                                                  T *__restrict__ u, const T *__restrict__ f,
                                                                  const CoarseArgs<T> *__restrict__ tab,
                                                                  const int *__restrict__ active) {
  extern __shared__ double cb[];
  if (tab) {  // packed launch: blockIdx.x selects the problem
    if (!active[blockIdx.x]) return;
    const CoarseArgs<T> a = tab[blockIdx.x];
    c = a.c; inv = a.inv; u = a.u; f = a.f;
  }
  pdl_trigger();
  pdl_wait();
  const int n = (nx - 1) * (ny - 1), nx1 = nx + 1;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const int i = k % (nx - 1) + 1, j = k / (nx - 1) + 1;
    const size_t p = (size_t)j * nx1 + i;
    double b = (double)f[p];
    if (i == 1) b -= c.W[i] * (double)u[p - 1];
    if (i == nx - 1) b -= c.E[i] * (double)u[p + 1];
    if (j == 1) b -= c.S[j] * (double)u[p - nx1];
    if (j == ny - 1) b -= c.N[j] * (double)u[p + nx1];
    cb[k] = b;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int k = threadIdx.x >> 5; k < n; k += nw) {
    double x = 0.0;
    for (int q = lane; q < n; q += 32) x += inv[(size_t)k * n + q] * cb[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) {
      const int i = k % (nx - 1) + 1, j = k / (nx - 1) + 1;
      u[(size_t)j * nx1 + i] = (T)x;
    }
  }
}

template <typename T>
cudaError_t launch_coarse_solve(const Grid &g, T *u, const T *f, cudaStream_t s) {
  const Level &L = g.lev[g.nlev - 1];
  if (g.cn <= 0) return cudaSuccess;
  count_launch(1);
  return launch_pdl(coarse_solve_kernel<T>, dim3(1), dim3(CS_THREADS), sizeof(double) * g.cn, s, cq<double>(L), L.nx,
                    L.ny, (const double *)g.cinv, u, f, (const CoarseArgs<T> *)nullptr, (const int *)nullptr);
}
template <typename T>
cudaError_t launch_coarse_solve_packed(const Grid &g, const PackedLaunch &pk, cudaStream_t s) {
  const Level &L = g.lev[g.nlev - 1];
  if (g.cn <= 0 || pk.count == 0) return cudaSuccess;
  count_launch(1);
  return launch_pdl(coarse_solve_kernel<T>, dim3(pk.count), dim3(CS_THREADS), sizeof(double) * g.cn, s,
                    cq<double>(L), L.nx, L.ny, (const double *)nullptr, (T *)nullptr, (const T *)nullptr,
                    static_cast<const CoarseArgs<T> *>(pk.tab), pk.active);
}
template cudaError_t launch_coarse_solve_packed<float>(const Grid &, const PackedLaunch &, cudaStream_t);
template cudaError_t launch_coarse_solve_packed<double>(const Grid &, const PackedLaunch &, cudaStream_t);
template cudaError_t launch_coarse_solve<double>(const Grid &, double *, const double *, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(const Grid &, float *, const float *, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 norms with a deterministic two-stage reduction.  Stage 1: NPART CTAs,
// grid-stride over interior rows, tree reduction in shared memory; stage 2:
// one CTA sums the partials in index order.
constexpr int NORM_THREADS = 256;

__device__ __forceinline__ double block_sum(double s) {
  __shared__ double ss[NORM_THREADS];
  ss[threadIdx.x] = s;
  __syncthreads();
  for (int h = NORM_THREADS / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) ss[threadIdx.x] += ss[threadIdx.x + h];
    __syncthreads();
  }
  return ss[0];
}

// Sum of squares of r over the interior, r = f - L u (u may be NULL: r = f;
// bnd_only: r = f - B u_b, the boundary neighbours alone, i.e. the residual of
// u with its interior taken as zero -- the scale of the relative residual).
// CTA b takes interior rows 1 + b, 1 + b + gridDim.x, ...; every thread its
// columns in order, so the result does not depend on timing.  FP64 issue is
// the bound on GB300 (about two FP64 operations per SM per clock): the defect
// takes 6 per node, with W_i + E_i per column precomputed (we) and f folded
// into the FMA chain,
//   r = f + C u_c - W u_w - E u_e - S u_s - N u_n,  C = (W + E) + (S + N),
// and the sum of squares one more.
__global__ void __launch_bounds__(NORM_THREADS) norm_stage1(CoefQ<double> c, const double *__restrict__ we,
                                                            int nx, int ny,
                                                            const double *__restrict__ u,
                                                            const double *__restrict__ f, int bnd_only,
                                                            double *__restrict__ part, float *__restrict__ r32,
                                                            float *__restrict__ e32,
                                                            const NormArgs *__restrict__ tab,
                                                            const int *__restrict__ active) {
  if (tab) {  // packed launch: blockIdx.y selects the problem
    if (!active[blockIdx.y]) return;
    const NormArgs a = tab[blockIdx.y];
    c = a.c; we = a.we; u = a.u; f = a.f; part = a.part;
    if (r32) { r32 = a.r32; e32 = a.e32; }
  }
  const int nx1 = nx + 1;
  double s = 0.0;
  // f - B g: only the boundary neighbours of u (its interior taken as 0), at
  // the nodes next to the boundary; elsewhere r = f.  Those nodes take their
  // own loops (rows 1 and ny - 1; columns 1 and nx - 1 by thread 0), so that
  // the FP64 operations of the boundary terms are not issued, predicated off,
  // at every node.
  auto rhs_edge = [&](int i, int j) {
    const size_t p = (size_t)j * nx1 + i;
    double r = f[p];
    if (i == 1) r -= __ldg(c.W + i) * u[p - 1];
    if (i == nx - 1) r -= __ldg(c.E + i) * u[p + 1];
    if (j == 1) r -= __ldg(c.S + j) * u[p - nx1];
    if (j == ny - 1) r -= __ldg(c.N + j) * u[p + nx1];
    return r;
  };
  for (int j = 1 + blockIdx.x; j < ny; j += gridDim.x) {
    const double sj = __ldg(c.S + j), nj = __ldg(c.N + j), snj = sj + nj;
    const size_t row = (size_t)j * nx1;
    if (bnd_only) {
      // with r32: also the FP32 copy of f - B g, the defect of a zero
      // interior, and a zero FP32 correction (the first refinement step)
      auto keep = [&](int i, double r) {
        if (r32) { r32[row + i] = narrow_rne(r); e32[row + i] = 0.0f; }
      };
      if (j == 1 || j == ny - 1) {
        for (int i = 1 + threadIdx.x; i < nx; i += NORM_THREADS) {
          const double r = rhs_edge(i, j);
          keep(i, r);
          s = fma(r, r, s);
        }
      } else {
        for (int i = 2 + threadIdx.x; i < nx - 1; i += NORM_THREADS) {
          const double r = f[row + i];
          keep(i, r);
          s = fma(r, r, s);
        }
        if (threadIdx.x == 0) {
          const double r1 = rhs_edge(1, j);
          keep(1, r1);
          s = fma(r1, r1, s);
          if (nx - 1 > 1) {
            const double r2 = rhs_edge(nx - 1, j);
            keep(nx - 1, r2);
            s = fma(r2, r2, s);
          }
        }
      }
      continue;
    }
    for (int i = 1 + threadIdx.x; i < nx; i += NORM_THREADS) {
      const size_t p = row + i;
      double r = f[p];
      if (u) {
        const double cc = __ldg(we + i) + snj;
        r = fma(cc, u[p], r);
        r = fma(-__ldg(c.W + i), u[p - 1], r);
        r = fma(-__ldg(c.E + i), u[p + 1], r);
        r = fma(-sj, u[p - nx1], r);
        r = fma(-nj, u[p + nx1], r);
      }
      s = fma(r, r, s);
    }
  }
  s = block_sum(s);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(NORM_THREADS) norm_stage2(const double *__restrict__ part, int npart,
                                                            double *__restrict__ out,
                                                            const NormArgs *__restrict__ tab,
                                                            const int *__restrict__ active) {
  if (tab) {  // packed launch: blockIdx.x selects the problem
    if (!active[blockIdx.x]) return;
    part = tab[blockIdx.x].part;
    out = tab[blockIdx.x].out;
  }
  double s = 0.0;
  for (int k = threadIdx.x; k < npart; k += NORM_THREADS) s += part[k];
  s = block_sum(s);
  if (threadIdx.x == 0) out[0] = s;
}

// norm_stage2 for packed refinement launches: each member's partials and output
__global__ void __launch_bounds__(NORM_THREADS) norm_stage2_refine(int npart, const RefineArgs *__restrict__ tab,
                                                                   const int *__restrict__ active) {
  if (!active[blockIdx.x]) return;
  const double *part = tab[blockIdx.x].part;
  double s = 0.0;
  for (int k = threadIdx.x; k < npart; k += NORM_THREADS) s += part[k];
  s = block_sum(s);
  if (threadIdx.x == 0) tab[blockIdx.x].out[0] = s;
}

static cudaError_t norms(const Grid &g, const double *u, const double *f, int bnd_only, cudaStream_t s,
                         float *r32 = nullptr, float *e32 = nullptr) {
  const Level &L = g.lev[0];
  norm_stage1<<<g.npartial, NORM_THREADS, 0, s>>>(cq<double>(L), L.WE64, L.nx, L.ny, u, f, bnd_only, g.partial,
                                                  r32, e32, nullptr, nullptr);
  norm_stage2<<<1, NORM_THREADS, 0, s>>>(g.partial, g.npartial, g.scal, nullptr, nullptr);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_norms_packed(const Grid &g, int bnd_only, const PackedLaunch &pk, cudaStream_t s, bool with_r32) {
  if (pk.count == 0) return cudaSuccess;
  const Level &L = g.lev[0];
  const NormArgs *tab = static_cast<const NormArgs *>(pk.tab);
  // a non-null placeholder tells the kernel to take each problem's r32 and e32
  float *mark = with_r32 ? g.r32 : nullptr;
  norm_stage1<<<dim3(g.npartial, pk.count), NORM_THREADS, 0, s>>>(cq<double>(L), L.WE64, L.nx, L.ny, nullptr,
                                                                  nullptr, bnd_only, nullptr, mark, mark, tab,
                                                                  pk.active);
  norm_stage2<<<pk.count, NORM_THREADS, 0, s>>>(nullptr, g.npartial, nullptr, tab, pk.active);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_resnorm64(const Grid &g, const double *u, const double *f, cudaStream_t s) {
  return norms(g, u, f, 0, s);
}
cudaError_t launch_rhsnorm64(const Grid &g, const double *u, const double *f, cudaStream_t s, float *r32,
                             float *e32) {
  return norms(g, u, f, 1, s, r32, e32);
}

// Row-wise elementwise kernels: CTA (x, j) covers interior row j + 1 with a
// grid-stride loop over its columns.
constexpr int EW_THREADS = 256;
static dim3 row_grid(const Level &L) { return dim3(std::min((L.nx - 1 + EW_THREADS - 1) / EW_THREADS, 4), L.ny - 1); }

// ---- Refinement residual with the update fused (Sec. 4 step (6) on the
// FP64 iterate of the FP32+FP64 refinement).  v = u + e, the correction of
// the FP32 cycles just run widened exactly (none on the first step);
// r = f - L v in FP64; r32 = float(r) by the integer-pipe rounding of
// fp_bits.h; the sum of r^2 per CTA (fixed order, deterministic).  v goes to
// a second array, not back into u: the CTAs next to a tile read u and e along
// its edges while the launch runs.  The host alternates the iterate between
// the caller's u and Grid::u2.
//
// CTA (bx, by) owns columns [i0, i0 + RR_TW) and rows [j0, j0 + rows): one
// column per thread, marching down its rows with v of the rows above, at and
// below in registers and the current row's v (with the halo columns left and
// right of the tile) in shared memory, three row buffers and one barrier per
// row.  Halo values are computed, not exchanged.  FP64 work per node: the
// update's add, the five FMAs of the defect (its diagonal read from cd64),
// the FMA of the norm; nothing else touches the FP64 pipe.
constexpr int RR_TW = NORM_THREADS;

template <bool UPD>
__global__ void __launch_bounds__(RR_TW) refine_residual_kernel(RefineArgs a, int nx, int ny, int rows,
                                                                const RefineArgs *__restrict__ tab,
                                                                const int *__restrict__ active) {
  const double *in = a.ua;
  double *out = a.ub;
  if (tab) {  // packed launch: blockIdx.z selects the problem; flag 2 swaps the iterates
    const int act = active[blockIdx.z];
    if (!act) return;
    a = tab[blockIdx.z];
    in = act == 2 ? a.ub : a.ua;
    out = act == 2 ? a.ua : a.ub;
  }
  __shared__ double sv[3][RR_TW + 2];
  const int nx1 = nx + 1, t = threadIdx.x;
  const int i0 = 1 + blockIdx.x * RR_TW, iend = min(i0 + RR_TW, nx);
  const int j0 = 1 + blockIdx.y * rows, jend = min(j0 + rows, ny);
  const int i = i0 + t;
  const bool own = i < iend;
  const bool edge_l = t == 0, edge_r = t == 1;  // the two halo columns
  const int ih = edge_l ? i0 - 1 : iend;
  const int kh = edge_l ? 0 : iend - i0 + 1;
  // v at (ii, jj): u + e inside, u on the boundary
  auto vat = [&](int ii, int jj) {
    const size_t p = (size_t)jj * nx1 + ii;
    double x = in[p];
    if (UPD && ii >= 1 && ii < nx && jj >= 1 && jj < ny) x += widen_exact(a.e[p]);
    return x;
  };
  double vm = 0.0, vc = 0.0, vn = 0.0, s = 0.0;
  if (own) {
    vm = vat(i, j0 - 1);
    vc = vat(i, j0);
    sv[j0 % 3][t + 1] = vc;
    if (UPD && j0 == 1) out[i] = vm;  // boundary row 0 of the other iterate
  }
  if (edge_l || edge_r) {
    const double x = vat(ih, j0);
    sv[j0 % 3][kh] = x;
    if (UPD && (ih == 0 || ih == nx)) out[(size_t)j0 * nx1 + ih] = x;
  }
  const double wi = own ? __ldg(a.c.W + i) : 0.0, ei = own ? __ldg(a.c.E + i) : 0.0;
  for (int j = j0; j < jend; ++j) {
    const int b0 = j % 3, b1 = (j + 1) % 3;
    if (own) {
      vn = vat(i, j + 1);
      sv[b1][t + 1] = vn;
    }
    if (edge_l || edge_r) {
      const double x = vat(ih, j + 1);
      sv[b1][kh] = x;
      if (UPD && (ih == 0 || ih == nx)) out[(size_t)(j + 1) * nx1 + ih] = x;
    }
    __syncthreads();
    if (own) {
      const size_t p = (size_t)j * nx1 + i;
      double r = fma(a.cd[p], vc, a.f[p]);
      r = fma(-wi, sv[b0][t], r);
      r = fma(-ei, sv[b0][t + 2], r);
      r = fma(-__ldg(a.c.S + j), vm, r);
      r = fma(-__ldg(a.c.N + j), vn, r);
      a.r32[p] = narrow_rne(r);
      if (UPD) out[p] = vc;
      else a.e32[p] = 0.0f;
      s = fma(r, r, s);
    }
    vm = vc;
    vc = vn;
  }
  if (UPD && own && jend == ny) out[(size_t)ny * nx1 + i] = vc;  // boundary row ny
  s = block_sum(s);
  if (t == 0) a.part[blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// cd[p] = W_i + E_i + S_j + N_j at interior nodes, 0 on the boundary, summed
// as norm_stage1 sums it ((W_i + E_i) + (S_j + N_j)), so both give the same
// defect bit for bit.
__global__ void diag_sum_kernel(CoefQ<double> c, const double *__restrict__ we, int nx, int ny,
                                double *__restrict__ cd) {
  const int j = blockIdx.y;
  const size_t row = (size_t)j * (nx + 1);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= nx; i += gridDim.x * blockDim.x)
    cd[row + i] = (i >= 1 && i < nx && j >= 1 && j < ny) ? we[i] + (c.S[j] + c.N[j]) : 0.0;
}

mg_status setup_refine_residual(Grid &g) {
  const Level &L = g.lev[0];
  const size_t nn = L.nn;
  if (cudaMalloc(&g.u2, nn * sizeof(double)) != cudaSuccess || cudaMalloc(&g.cd64, nn * sizeof(double)) != cudaSuccess ||
      cudaMemset(g.u2, 0, nn * sizeof(double)) != cudaSuccess)
    return MG_ERR_CUDA;
  diag_sum_kernel<<<dim3(std::max(1, std::min(8, (L.nx + 256) / 256)), L.ny + 1), 256>>>(cq<double>(L), L.WE64, L.nx,
                                                                                          L.ny, g.cd64);
  if (cudaGetLastError() != cudaSuccess) return MG_ERR_CUDA;
  // about four waves of CTAs, at least 8 rows each
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine_residual_kernel<true>, RR_TW, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  const int gx = (L.nx - 1 + RR_TW - 1) / RR_TW;
  const int target = std::max(1, 4 * per_sm * std::max(1, g.sms) / gx);
  int rows = std::max(8, (L.ny - 1 + target - 1) / target);
  rows = std::min(rows, L.ny - 1);
  g.rr_rows = rows;
  g.rr_gx = gx;
  g.rr_gy = (L.ny - 1 + rows - 1) / rows;
  if (cudaMalloc(&g.rpart, (size_t)g.rr_gx * g.rr_gy * sizeof(double)) != cudaSuccess) return MG_ERR_CUDA;
  return MG_OK;
}

cudaError_t launch_refine_residual(const Grid &g, const double *u, const float *e, double *uo, const double *f,
                                   cudaStream_t s) {
  const Level &L = g.lev[0];
  const RefineArgs a{cq<double>(L), g.cd64, const_cast<double *>(u), uo, e, f, g.r32, g.e32, g.rpart, nullptr};
  const dim3 grid(g.rr_gx, g.rr_gy);
  if (e) refine_residual_kernel<true><<<grid, RR_TW, 0, s>>>(a, L.nx, L.ny, g.rr_rows, nullptr, nullptr);
  else refine_residual_kernel<false><<<grid, RR_TW, 0, s>>>(a, L.nx, L.ny, g.rr_rows, nullptr, nullptr);
  norm_stage2<<<1, NORM_THREADS, 0, s>>>(g.rpart, g.rr_gx * g.rr_gy, g.scal, nullptr, nullptr);
  count_launch(2);
  if (e) {
    // the next cycles start from e = 0; zeroed only now, since the kernel
    // read e along the tile edges of every CTA
    const cudaError_t z = cudaMemsetAsync(g.e32, 0, L.nn * sizeof(float), s);
    if (z != cudaSuccess) return z;
  }
  return cudaGetLastError();
}

cudaError_t launch_refine_residual_packed(const Grid &g, bool update, const PackedLaunch &pk, float *const *e32s,
                                          cudaStream_t s) {
  if (pk.count == 0) return cudaSuccess;
  const Level &L = g.lev[0];
  const RefineArgs none{};
  const RefineArgs *tab = static_cast<const RefineArgs *>(pk.tab);
  const dim3 grid(g.rr_gx, g.rr_gy, pk.count);
  if (update) refine_residual_kernel<true><<<grid, RR_TW, 0, s>>>(none, L.nx, L.ny, g.rr_rows, tab, pk.active);
  else refine_residual_kernel<false><<<grid, RR_TW, 0, s>>>(none, L.nx, L.ny, g.rr_rows, tab, pk.active);
  norm_stage2_refine<<<pk.count, NORM_THREADS, 0, s>>>(g.rr_gx * g.rr_gy, tab, pk.active);
  count_launch(2);
  if (update)
    for (int k = 0; k < pk.count; ++k)
      if (e32s[k]) {
        const cudaError_t z = cudaMemsetAsync(e32s[k], 0, L.nn * sizeof(float), s);
        if (z != cudaSuccess) return z;
      }
  return cudaGetLastError();
}

// out = in * (dx_i dy_j) (inverse = 0) or in / (dx_i dy_j) (inverse = 1) at
// interior nodes, 0 on the boundary; dx_i = (x_{i+1} - x_{i-1})/2.
__global__ void diag_scale_kernel(const double *__restrict__ x, const double *__restrict__ y, int nx, int ny,
                                  double *__restrict__ out, const double *__restrict__ in, int inverse) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i > nx) return;
  const size_t p = (size_t)j * (nx + 1) + i;
  if (i == 0 || j == 0 || i == nx || j == ny) { out[p] = 0.0; return; }
  const double dxy = (0.5 * (x[i + 1] - x[i - 1])) * (0.5 * (y[j + 1] - y[j - 1]));
  out[p] = inverse ? in[p] / dxy : in[p] * dxy;
}
cudaError_t launch_diag_scale(const Grid &g, double *out, const double *in, int inverse, cudaStream_t s) {
  const Level &L = g.lev[0];
  dim3 b(128), gr((L.nx + 1 + 127) / 128, L.ny + 1);
  diag_scale_kernel<<<gr, b, 0, s>>>(L.xd, L.yd, L.nx, L.ny, out, in, inverse);
  count_launch(1);
  return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(EW_THREADS) zero_interior_kernel(int nx, T *__restrict__ a,
                                                                   const UpdateArgs *__restrict__ tab,
                                                                   const int *__restrict__ active) {
  if constexpr (sizeof(T) == 8) {
    if (tab) {  // packed launch: blockIdx.z selects the problem; zeroes its u
      if (!active[blockIdx.z]) return;
      a = tab[blockIdx.z].u;
    }
  }
  const size_t row = (size_t)(blockIdx.y + 1) * (nx + 1);
  for (int i = 1 + blockIdx.x * EW_THREADS + threadIdx.x; i < nx; i += gridDim.x * EW_THREADS) a[row + i] = T(0);
}
template <typename T>
cudaError_t launch_zero_interior(const Level &L, T *a, cudaStream_t s) {
  zero_interior_kernel<T><<<row_grid(L), EW_THREADS, 0, s>>>(L.nx, a, nullptr, nullptr);
  count_launch(1);
  return cudaGetLastError();
}
cudaError_t launch_zero_interior_packed(const Grid &g, const PackedLaunch &pk, cudaStream_t s) {
  if (pk.count == 0) return cudaSuccess;
  const Level &L = g.lev[0];
  dim3 gr = row_grid(L);
  gr.z = pk.count;
  zero_interior_kernel<double><<<gr, EW_THREADS, 0, s>>>(L.nx, nullptr, static_cast<const UpdateArgs *>(pk.tab),
                                                         pk.active);
  count_launch(1);
  return cudaGetLastError();
}
// Gradient of a loss with respect to the Dirichlet data, from the adjoint
// state: u_int = A^{-1} (f - B g), (B g)_p = sum over boundary neighbours b
// of p of coef(p -> b) g_b, so dloss/dg_b = dloss/du_b - sum_p coef(p -> b)
// lambda_p.  One thread per boundary node (bottom row, top row, left and
// right columns without the corners); interior entries of grad_g are 0.
__global__ void boundary_adjoint_kernel(const double *__restrict__ W, const double *__restrict__ E,
                                        const double *__restrict__ S, const double *__restrict__ N, int nx, int ny,
                                        const double *__restrict__ lam, const double *__restrict__ gu,
                                        double *__restrict__ gg) {
  const int nx1 = nx + 1, nb = 2 * nx1 + 2 * (ny - 1);
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    int i, j;
    if (k < nx1) { i = k; j = 0; }
    else if (k < 2 * nx1) { i = k - nx1; j = ny; }
    else if (k < 2 * nx1 + (ny - 1)) { i = 0; j = k - 2 * nx1 + 1; }
    else { i = nx; j = k - 2 * nx1 - (ny - 1) + 1; }
    const size_t b = (size_t)j * nx1 + i;
    double v = gu[b];
    if (j == 0 && i > 0 && i < nx) v -= S[1] * lam[b + nx1];
    if (j == ny && i > 0 && i < nx) v -= N[ny - 1] * lam[b - nx1];
    if (i == 0 && j > 0 && j < ny) v -= W[1] * lam[b + 1];
    if (i == nx && j > 0 && j < ny) v -= E[nx - 1] * lam[b - 1];
    gg[b] = v;
  }
}
cudaError_t launch_boundary_adjoint(const Grid &g, const double *lam, const double *gu, double *gg,
                                    cudaStream_t s) {
  const Level &L = g.lev[0];
  const int nb = 2 * (L.nx + 1) + 2 * (L.ny - 1);
  zero_interior_kernel<double><<<row_grid(L), EW_THREADS, 0, s>>>(L.nx, gg, nullptr, nullptr);
  boundary_adjoint_kernel<<<(nb + 255) / 256, 256, 0, s>>>(L.W64, L.E64, L.S64, L.N64, L.nx, L.ny, lam, gu, gg);
  count_launch(2);
  return cudaGetLastError();
}

template cudaError_t launch_zero_interior<double>(const Level &, double *, cudaStream_t);
template cudaError_t launch_zero_interior<float>(const Level &, float *, cudaStream_t);

}  // namespace tmg
