// fd.cu -- direct solve of one coarse level's interior system, for the FP32
// cycles of FP32+refine (mg_params.coarse_direct).
//
// On a rectilinear grid the 5-point operator of Sec. 2 is a Kronecker sum:
// for U[j][i] on the interior, L(U) = U Ax^T + Ay U, with Ax the tridiagonal
// of (W_i, -(W_i + E_i), E_i) along x and Ay the same along y.  Each factor
// is similar to a symmetric tridiagonal matrix: with d_1 = 1 and
// d_{i+1} = d_i E_i / W_{i+1} (so d_i E_i = d_{i+1} W_{i+1}, the symmetry of
// D L), S = D^{1/2} A D^{-1/2} has off-diagonal sqrt(E_i W_{i+1}).  With
// S = Q diag(lambda) Q^T (cyclic Jacobi, at setup, FP64) the solve is the
// fast diagonalisation method of Lynch, Rice & Thomas (1964):
//   R^ = Qy^T (Dy^{1/2} R Dx^{1/2}) Qx,   U^_ji = R^_ji / (lambda_x,i + lambda_y,j),
//   U  = Dy^{-1/2} Qy U^ Qx^T Dx^{-1/2},
// four small dense products in one CTA (shared memory).  The transforms are
// orthogonal, so in FP32 the solution's relative error stays near the FP32
// rounding level even when L is badly conditioned.  Used on the finest level
// with both sides at most FD_MAX_SIDE intervals, below the finest level; the
// levels under it are then not visited by the FP32 cycles.
#include <cmath>
#include <vector>

#include "device_util.cuh"
#include "fd_host.h"
#include "solve.h"

namespace tmg {

namespace {

constexpr int FD_THREADS = 1024;

// One CTA.  Shared memory: Qx (mx^2), Qy (my^2), two my x mx buffers.
__global__ void __launch_bounds__(FD_THREADS) fd_solve_kernel(Coefs<float> c, int nx, int ny,
                                                              const float *__restrict__ tr, float *__restrict__ u,
                                                              const float *__restrict__ f) {
  extern __shared__ float fs[];
  const int mx = nx - 1, my = ny - 1, n = mx * my, nx1 = nx + 1, t = threadIdx.x;
  float *Qx = fs, *Qy = Qx + mx * mx, *A1 = Qy + my * my, *A2 = A1 + n;
  const float *gQx = tr, *gQy = gQx + mx * mx, *lx = gQy + my * my, *ly = lx + mx, *sx = ly + my, *sy = sx + mx;
  pdl_trigger();
  for (int k = t; k < mx * mx; k += FD_THREADS) Qx[k] = gQx[k];
  for (int k = t; k < my * my; k += FD_THREADS) Qy[k] = gQy[k];
  pdl_wait();
  // 1. scaled right-hand side, the boundary neighbours moved over
  for (int e = t; e < n; e += FD_THREADS) {
    const int j = e / mx, i = e - j * mx, ii = i + 1, jj = j + 1;
    const size_t p = (size_t)jj * nx1 + ii;
    float b = f[p];
    if (ii == 1) b -= c.W[ii] * u[p - 1];
    if (ii == nx - 1) b -= c.E[ii] * u[p + 1];
    if (jj == 1) b -= c.S[jj] * u[p - nx1];
    if (jj == ny - 1) b -= c.N[jj] * u[p + nx1];
    A1[e] = sy[j] * sx[i] * b;
  }
  __syncthreads();
  // 2. A2 = Qy^T A1
  for (int e = t; e < n; e += FD_THREADS) {
    const int j = e / mx, i = e - j * mx;
    float s = 0.0f;
    for (int k = 0; k < my; ++k) s = fmaf(Qy[k * my + j], A1[k * mx + i], s);
    A2[e] = s;
  }
  __syncthreads();
  // 3. A1 = A2 Qx, 4. divided by the eigenvalue sums
  for (int e = t; e < n; e += FD_THREADS) {
    const int j = e / mx, i = e - j * mx;
    float s = 0.0f;
    for (int k = 0; k < mx; ++k) s = fmaf(A2[j * mx + k], Qx[k * mx + i], s);
    A1[e] = s / (lx[i] + ly[j]);
  }
  __syncthreads();
  // 5. A2 = Qy A1
  for (int e = t; e < n; e += FD_THREADS) {
    const int j = e / mx, i = e - j * mx;
    float s = 0.0f;
    for (int k = 0; k < my; ++k) s = fmaf(Qy[j * my + k], A1[k * mx + i], s);
    A2[e] = s;
  }
  __syncthreads();
  // 6. U = A2 Qx^T, unscaled, written to u
  for (int e = t; e < n; e += FD_THREADS) {
    const int j = e / mx, i = e - j * mx;
    float s = 0.0f;
    for (int k = 0; k < mx; ++k) s = fmaf(A2[j * mx + k], Qx[i * mx + k], s);
    u[(size_t)(j + 1) * nx1 + (i + 1)] = s / (sy[j] * sx[i]);
  }
}

size_t fd_smem(int nx, int ny) {
  const size_t mx = nx - 1, my = ny - 1;
  return sizeof(float) * (mx * mx + my * my + 2 * mx * my);
}

}  // namespace

mg_status setup_direct_level(Grid &g) {
  g.fd_level = -1;
  if (!(g.prec_mask & 2)) return MG_OK;
  int l = -1;
  for (int k = 1; k + 1 < g.nlev; ++k)
    if (g.lev[k].nx <= FD_MAX_SIDE && g.lev[k].ny <= FD_MAX_SIDE && g.lev[k].nx >= 2 && g.lev[k].ny >= 2) {
      l = k;
      break;
    }
  if (l < 0) return MG_OK;
  const Level &L = g.lev[l];
  std::vector<double> Qx, lx, sx, Qy, ly, sy;
  if (!fd::axis_transform(L.hW, L.hE, L.nx, Qx, lx, sx) || !fd::axis_transform(L.hS, L.hN, L.ny, Qy, ly, sy))
    return MG_OK;
  std::vector<float> h;
  for (double v : Qx) h.push_back((float)v);
  for (double v : Qy) h.push_back((float)v);
  for (double v : lx) h.push_back((float)v);
  for (double v : ly) h.push_back((float)v);
  for (double v : sx) h.push_back((float)v);
  for (double v : sy) h.push_back((float)v);
  TRY_CUDA("cudaMalloc(direct level)", cudaMalloc(&g.fd_tr, sizeof(float) * h.size()));
  TRY_CUDA("cudaMemcpy(direct level)", cudaMemcpy(g.fd_tr, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice));
  TRY_CUDA("direct level kernel attributes",
           cudaFuncSetAttribute(fd_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fd_smem(L.nx, L.ny)));
  g.fd_level = l;
  return MG_OK;
}

cudaError_t launch_direct_level(const Grid &g, float *u, const float *f, cudaStream_t s) {
  if (g.fd_level < 0) return cudaErrorInvalidValue;
  const Level &L = g.lev[g.fd_level];
  count_launch(1);
  return launch_pdl(fd_solve_kernel, dim3(1), dim3(FD_THREADS), fd_smem(L.nx, L.ny), s, level_coefs<float>(L), L.nx,
                    L.ny, (const float *)g.fd_tr, u, f);
}

}  // namespace tmg
