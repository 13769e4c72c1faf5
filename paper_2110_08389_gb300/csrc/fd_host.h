// fd_host.h -- host part of the direct level solve (fd.cu): the symmetrised
// 1D factors of the Kronecker-sum operator and their eigen-decomposition.
// Plain C++ (no CUDA), so that it is also checked on the CPU.
#pragma once
#include <cmath>
#include <vector>

namespace tmg {
namespace fd {

// cyclic Jacobi eigen-decomposition of the symmetric m x m matrix A (row
// major, destroyed): A = V diag(lam) V^T, V's columns the eigenvectors
inline bool jacobi_eig(int m, std::vector<double> &A, std::vector<double> &V, std::vector<double> &lam) {
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
inline bool axis_transform(const std::vector<double> &lo, const std::vector<double> &hi, int n, std::vector<double> &Q,
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

}  // namespace fd
}  // namespace tmg
