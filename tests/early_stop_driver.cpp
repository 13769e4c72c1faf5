// Evaluates the early-stop helpers of csrc/solve.h on cases read from stdin,
// one per line.  "h steps rel prev left tol" prints tmg::hopeless (1 or 0);
// "s f64 max_cycles max_outer inner cycles outer" prints tmg::steps_left.
#include <cstdio>

#include "solve.h"

int main() {
  char kind[4];
  while (std::scanf("%3s", kind) == 1) {
    if (kind[0] == 'h') {
      int steps, left;
      double rel, prev, tol;
      if (std::scanf("%d %lf %lf %d %lf", &steps, &rel, &prev, &left, &tol) != 5) return 1;
      std::printf("%d\n", tmg::hopeless(steps, rel, prev, left, tol) ? 1 : 0);
    } else {
      int f64, mc, mo, inner, cyc, outer;
      if (std::scanf("%d %d %d %d %d %d", &f64, &mc, &mo, &inner, &cyc, &outer) != 6) return 1;
      std::printf("%d\n", tmg::steps_left(f64 != 0, mc, mo, inner, cyc, outer));
    }
  }
  return 0;
}
