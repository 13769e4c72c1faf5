// Runs the closed-form 2D block builders of csrc/blocks.h for (nx ny
// smoother colour) read on stdin (smoother 0 zebra x, 1 zebra y, 2 tweed,
// 3 wireframe) and prints: for every node (x fastest) its block, -1 if not in
// a block of that colour; then 1 if every chain is a path of adjacent nodes
// and every junction link points at the junction, else 0.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "blocks.h"

using namespace tmg;

int main() {
  int nx, ny, sm, colour;
  if (std::scanf("%d %d %d %d", &nx, &ny, &sm, &colour) != 4) return 2;
  std::vector<HBlock> bl;
  if (sm <= 1) zebra_blocks(nx, ny, colour, sm == 0, bl);
  else if (sm == 2) tweed_blocks(nx, ny, colour, bl);
  else wireframe_blocks(nx, ny, colour, bl);
  const int nx1 = nx + 1;
  std::vector<int> owner((size_t)nx1 * (ny + 1), -1);
  const int di[4] = {1, -1, 0, 0}, dj[4] = {0, 0, 1, -1};
  bool shapes = true;
  auto put = [&](int i, int j, int b) {
    if (i < 1 || i >= nx || j < 1 || j >= ny) { shapes = false; return; }
    int &o = owner[(size_t)j * nx1 + i];
    if (o != -1) shapes = false;
    o = b;
  };
  for (size_t b = 0; b < bl.size(); ++b) {
    const HBlock &h = bl[b];
    if (h.junc) put(h.ji, h.jj, (int)b);
    for (const HChain &c : h.ch) {
      int pi = -1, pj = -1, fi = -1, fj = -1;
      for (const HSeg &s : c.s)
        for (int t = 0; t < s.len; ++t) {
          const int i = s.i0 + t * di[s.dir], j = s.j0 + t * dj[s.dir];
          if (pi >= 0 && std::abs(i - pi) + std::abs(j - pj) != 1) shapes = false;
          if (fi < 0) { fi = i; fj = j; }
          put(i, j, (int)b);
          pi = i; pj = j;
        }
      if (c.lj && (!h.junc || pi + di[c.ljdir] != h.ji || pj + dj[c.ljdir] != h.jj)) shapes = false;
      if (c.fj && (!h.junc || std::abs(fi - h.ji) + std::abs(fj - h.jj) != 1)) shapes = false;
    }
  }
  for (int v : owner) std::printf("%d\n", v);
  std::printf("%d\n", shapes ? 1 : 0);
  return 0;
}
