// Evaluates tmg::hopeless (csrc/solve.h) on the cases read from stdin, one
// per line: steps rel prev left tol; prints 1 or 0 per case.
#include <cstdio>

#include "solve.h"

int main() {
  int steps, left;
  double rel, prev, tol;
  while (std::scanf("%d %lf %lf %d %lf", &steps, &rel, &prev, &left, &tol) == 5)
    std::printf("%d\n", tmg::hopeless(steps, rel, prev, left, tol) ? 1 : 0);
  return 0;
}
