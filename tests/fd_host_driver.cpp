// Prints the transforms of csrc/fd_host.h for the 1D operator read on stdin:
// n, then W_1..W_{n-1}, then E_1..E_{n-1}.  Output: ok, lambda (n-1 values),
// sqrt(d) (n-1), Q row-major ((n-1)^2).
#include <cstdio>
#include <vector>

#include "fd_host.h"

int main() {
  int n = 0;
  if (std::scanf("%d", &n) != 1 || n < 2) return 2;
  std::vector<double> lo(n + 1, 0.0), hi(n + 1, 0.0);
  for (int i = 1; i < n; ++i) std::scanf("%lf", &lo[i]);
  for (int i = 1; i < n; ++i) std::scanf("%lf", &hi[i]);
  std::vector<double> Q, lam, sd;
  const bool ok = tmg::fd::axis_transform(lo, hi, n, Q, lam, sd);
  std::printf("%d\n", ok ? 1 : 0);
  for (double v : lam) std::printf("%.17g\n", v);
  for (double v : sd) std::printf("%.17g\n", v);
  for (double v : Q) std::printf("%.17g\n", v);
  return 0;
}
