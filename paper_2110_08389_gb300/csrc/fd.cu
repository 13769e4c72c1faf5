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
#include "solve.h"

namespace tmg {

namespace {

constexpr int FD_THREADS = 1024;

// cyclic Jacobi eigen-decomposition of the symmetric m x m matrix A (row
// major, destroyed): A = V diag(lam) V^T, V's columns the eigenvectors
bool jacobi_eig(int m, std::vector<double> &A, std::vector<double> &V, std::vector<double> &lam) {
  V.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) V[(size_t)i * m + i] = 1.0;
  auto a = [&](int r, int c) -> double & { return A[(size_t)r * m + c]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < m; ++c) (r == c ? diag : off) += a(r, c) * a(r, c);
    if (off <= 1e-30 * diag) {
      lam.resize(m);
      for (int i = 0; i < m; ++i) lam[i] = a(i, i);
      return true;
    }
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = a(p, q);
        if (apq == 0.0) continue;
        // rotation that zeroes a(p, q) (Golub & Van Loan, the symmetric Schur decomposition)
        const double theta = (a(q, q) - a(p, p)) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // A <- A J
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {  // A <- J^T A
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < m; ++k) {  // V <- V J
          double &vkp = V[(size_t)k * m + p], &vkq = V[(size_t)k * m + q];
          const double x = vkp, y = vkq;
          vkp = c * x - s * y;
          vkq = s * x + c * y;
        }
      }
  }
  return false;
}

// The transforms of one axis: Q (m x m, row major), lambda, sqrt(d).
bool axis_transform(const std::vector<double> &lo, const std::vector<double> &hi, int n, std::vector<double> &Q,
                    std::vector<double> &lam, std::vector<double> &sd) {
  const int m = n - 1;
  std::vector<double> d(m, 1.0), S((size_t)m * m, 0.0);
  for (int r = 0; r + 1 < m; ++r) d[r + 1] = d[r] * hi[r + 1] / lo[r + 2];
  for (int r = 0; r < m; ++r) {
    const int i = r + 1;
    S[(size_t)r * m + r] = -(lo[i] + hi[i]);
    if (r + 1 < m) S[(size_t)r * m + r + 1] = S[(size_t)(r + 1) * m + r] = std::sqrt(hi[i] * lo[i + 1]);
  }
  sd.resize(m);
  for (int r = 0; r < m; ++r) sd[r] = std::sqrt(d[r]);
  return jacobi_eig(m, S, Q, lam);
}

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
  if (!axis_transform(L.hW, L.hE, L.nx, Qx, lx, sx) || !axis_transform(L.hS, L.hN, L.ny, Qy, ly, sy)) return MG_OK;
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
