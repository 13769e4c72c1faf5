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
//   resnorm / ir_residual    FP64 defect norms with a fixed-order reduction
//                            (deterministic), optionally writing the FP32 copy
//                            of the defect for the refinement loop
//   ir_update                u64 += e32
#include "mg_internal.h"

namespace tmg {

template <typename T>
struct CoefQ {
  const T *W, *E, *S, *N;
};
template <typename T>
static CoefQ<T> cq(const Level &L);
template <>
CoefQ<double> cq<double>(const Level &L) { return {L.W64, L.E64, L.S64, L.N64}; }
template <>
CoefQ<float> cq<float>(const Level &L) { return {L.W32, L.E32, L.S32, L.N32}; }

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

// One thread per coarse interior node (I, J); fine node (2I, 2J) and its 8
// neighbours (defect 0 on the fine boundary).  kind: 0 = half weighting
// (1/2, 1/8 x 4), 1 = full weighting (1/4, 1/8 x 4, 1/16 x 4).
template <typename T>
__global__ void residual_restrict_kernel(CoefQ<T> c, int nx, int ny, int nxc, int kind,
                                         const T *__restrict__ u, const T *__restrict__ f, T *__restrict__ fc,
                                         T *__restrict__ uc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x + 1, J = blockIdx.y + 1;
  if (I >= nxc) return;
  const int nx1 = nx + 1, i = 2 * I, j = 2 * J;
  auto dd = [&](int a, int b) -> T {
    return (a > 0 && a < nx && b > 0 && b < ny) ? defect_at(c, u, f, a, b, nx1) : T(0);
  };
  const T centre = dd(i, j);
  const T edge = (dd(i - 1, j) + dd(i, j - 1)) + (dd(i + 1, j) + dd(i, j + 1));
  T v;
  if (kind == MG_RESTRICT_HW) {
    v = T(0.5) * centre + T(0.125) * edge;
  } else {
    const T corner = (dd(i - 1, j - 1) + dd(i + 1, j - 1)) + (dd(i - 1, j + 1) + dd(i + 1, j + 1));
    v = T(0.25) * centre + T(0.125) * edge + T(0.0625) * corner;
  }
  const size_t q = (size_t)J * (nxc + 1) + I;
  fc[q] = v;
  if (uc) uc[q] = T(0);
}

template <typename T>
cudaError_t launch_residual_restrict(const Level &F, const Level &C, int kind, const T *u, const T *f, T *fc,
                                     T *uc, cudaStream_t s) {
  dim3 b(128), g((C.nx - 1 + 127) / 128, C.ny - 1);
  if (C.nx < 2 || C.ny < 2) return cudaSuccess;
  residual_restrict_kernel<T><<<g, b, 0, s>>>(cq<T>(F), F.nx, F.ny, C.nx, kind, u, f, fc, uc);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_residual_restrict<double>(const Level &, const Level &, int, const double *,
                                                      const double *, double *, double *, cudaStream_t);
template cudaError_t launch_residual_restrict<float>(const Level &, const Level &, int, const float *,
                                                     const float *, float *, float *, cudaStream_t);

// Bilinear interpolation of the coarse correction (index-based weights,
// Sec. 4), added to the fine interior.
template <typename T>
__global__ void prolong_add_kernel(int nx, int ny, int nxc, const T *__restrict__ uc, T *__restrict__ u) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i >= nx) return;
  const int c1 = nxc + 1;
  const int I = i >> 1, Jc = j >> 1;
  T v;
  if (!(i & 1) && !(j & 1)) v = uc[(size_t)Jc * c1 + I];
  else if (!(i & 1)) v = T(0.5) * (uc[(size_t)Jc * c1 + I] + uc[(size_t)(Jc + 1) * c1 + I]);
  else if (!(j & 1)) v = T(0.5) * (uc[(size_t)Jc * c1 + I] + uc[(size_t)Jc * c1 + I + 1]);
  else
    v = T(0.25) * ((uc[(size_t)Jc * c1 + I] + uc[(size_t)Jc * c1 + I + 1]) +
                   (uc[(size_t)(Jc + 1) * c1 + I] + uc[(size_t)(Jc + 1) * c1 + I + 1]));
  u[(size_t)j * (nx + 1) + i] += v;
}

template <typename T>
cudaError_t launch_prolong_add(const Level &F, const Level &C, const T *uc, T *u, cudaStream_t s) {
  dim3 b(128), g((F.nx - 1 + 127) / 128, F.ny - 1);
  prolong_add_kernel<T><<<g, b, 0, s>>>(F.nx, F.ny, C.nx, uc, u);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_prolong_add<double>(const Level &, const Level &, const double *, double *,
                                                cudaStream_t);
template cudaError_t launch_prolong_add<float>(const Level &, const Level &, const float *, float *,
                                               cudaStream_t);

// Coarsest level: x = A^{-1} b in FP64, b = f - (boundary neighbours).  One
// CTA; unknown index (j-1)(nx-1) + (i-1).
template <typename T>
__global__ void coarse_solve_kernel(CoefQ<double> c, int nx, int ny, const double *__restrict__ inv,
                                    T *__restrict__ u, const T *__restrict__ f) {
  extern __shared__ double cb[];
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
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    double x = 0.0;
    for (int q = 0; q < n; ++q) x += inv[(size_t)k * n + q] * cb[q];
    const int i = k % (nx - 1) + 1, j = k / (nx - 1) + 1;
    u[(size_t)j * nx1 + i] = (T)x;
  }
}

template <typename T>
cudaError_t launch_coarse_solve(const Grid &g, T *u, const T *f, cudaStream_t s) {
  const Level &L = g.lev[g.nlev - 1];
  if (g.cn <= 0) return cudaSuccess;
  coarse_solve_kernel<T><<<1, 256, sizeof(double) * g.cn, s>>>(cq<double>(L), L.nx, L.ny, g.cinv, u, f);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_coarse_solve<double>(const Grid &, double *, const double *, cudaStream_t);
template cudaError_t launch_coarse_solve<float>(const Grid &, float *, const float *, cudaStream_t);

// ---------------------------------------------------------------------------
// FP64 norms with a deterministic two-stage reduction.  Stage 1: NPART CTAs,
// grid-stride over interior rows, tree reduction in shared memory; stage 2:
// one CTA sums the partials in index order.
constexpr int NORM_THREADS = 256;

__device__ __forceinline__ void block_reduce2(double &s, double &m) {
  __shared__ double ss[NORM_THREADS], sm[NORM_THREADS];
  ss[threadIdx.x] = s; sm[threadIdx.x] = m;
  __syncthreads();
  for (int h = NORM_THREADS / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      ss[threadIdx.x] += ss[threadIdx.x + h];
      sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + h]);
    }
    __syncthreads();
  }
  s = ss[0]; m = sm[0];
}

// mode 0: r = f - L u (u may be NULL: r = f); mode 1: same, and r32 = float(r).
__global__ void __launch_bounds__(NORM_THREADS) norm_stage1(CoefQ<double> c, int nx, int ny,
                                                            const double *__restrict__ u,
                                                            const double *__restrict__ f,
                                                            float *__restrict__ r32, double *__restrict__ part) {
  const int nx1 = nx + 1;
  const long long ni = (long long)(nx - 1) * (ny - 1);
  double s = 0.0, m = 0.0;
  for (long long k = (long long)blockIdx.x * NORM_THREADS + threadIdx.x; k < ni;
       k += (long long)gridDim.x * NORM_THREADS) {
    const int i = (int)(k % (nx - 1)) + 1, j = (int)(k / (nx - 1)) + 1;
    const double r = u ? defect_at(c, u, f, i, j, nx1) : f[(size_t)j * nx1 + i];
    if (r32) r32[(size_t)j * nx1 + i] = (float)r;
    s += r * r;
    m = fmax(m, fabs(r));
  }
  block_reduce2(s, m);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = s; part[2 * blockIdx.x + 1] = m; }
}

__global__ void __launch_bounds__(NORM_THREADS) norm_stage2(const double *__restrict__ part, int npart,
                                                            double *__restrict__ out) {
  double s = 0.0, m = 0.0;
  for (int k = threadIdx.x; k < npart; k += NORM_THREADS) { s += part[2 * k]; m = fmax(m, part[2 * k + 1]); }
  block_reduce2(s, m);
  if (threadIdx.x == 0) { out[0] = s; out[1] = m; }
}

static cudaError_t norms(const Grid &g, const double *u, const double *f, float *r32, cudaStream_t s) {
  const Level &L = g.lev[0];
  norm_stage1<<<g.npartial, NORM_THREADS, 0, s>>>(cq<double>(L), L.nx, L.ny, u, f, r32, g.partial);
  norm_stage2<<<1, NORM_THREADS, 0, s>>>(g.partial, g.npartial, g.scal);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t launch_resnorm64(const Grid &g, const double *u, const double *f, cudaStream_t s) {
  return norms(g, u, f, nullptr, s);
}
cudaError_t launch_ir_residual(const Grid &g, const double *u, const double *f, float *r32, cudaStream_t s) {
  return norms(g, u, f, r32, s);
}

__global__ void ir_update_kernel(int nx, int ny, double *__restrict__ u, const float *__restrict__ e) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i >= nx) return;
  const size_t p = (size_t)j * (nx + 1) + i;
  u[p] += (double)e[p];
}
cudaError_t launch_ir_update(const Grid &g, double *u, const float *e, cudaStream_t s) {
  const Level &L = g.lev[0];
  dim3 b(128), gr((L.nx - 1 + 127) / 128, L.ny - 1);
  ir_update_kernel<<<gr, b, 0, s>>>(L.nx, L.ny, u, e);
  count_launch(1);
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
__global__ void zero_interior_kernel(int nx, int ny, T *__restrict__ a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x + 1, j = blockIdx.y + 1;
  if (i >= nx) return;
  a[(size_t)j * (nx + 1) + i] = T(0);
}
template <typename T>
cudaError_t launch_zero_interior(const Level &L, T *a, cudaStream_t s) {
  dim3 b(128), gr((L.nx - 1 + 127) / 128, L.ny - 1);
  zero_interior_kernel<T><<<gr, b, 0, s>>>(L.nx, L.ny, a);
  count_launch(1);
  return cudaGetLastError();
}
template cudaError_t launch_zero_interior<double>(const Level &, double *, cudaStream_t);
template cudaError_t launch_zero_interior<float>(const Level &, float *, cudaStream_t);

}  // namespace tmg
