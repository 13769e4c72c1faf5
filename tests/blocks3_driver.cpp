// Runs the 3D block builder of csrc/blocks3_host.h on the sizes read from
// stdin (nx ny nz smoother) and prints: ok; then for every node of the level
// (x fastest) its block, -1 off the interior; then every block's colour; then
// whether every chain is a path of adjacent nodes, every junction attachment
// is adjacent to its junction in the stated direction, and every skeleton
// edge runs straight between its two corners.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "blocks3_host.h"

using namespace tmg;

static long long step_of(int d, int nx1, long long plane) {
  const long long s[6] = {1, -1, nx1, -(long long)nx1, plane, -plane};
  return s[d];
}

int main() {
  int nx, ny, nz, sm;
  if (std::scanf("%d %d %d %d", &nx, &ny, &nz, &sm) != 4) return 2;
  Level3 L;
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int nx1 = nx + 1;
  const long long plane = (long long)nx1 * (ny + 1);
  std::vector<HBlock3> bl;
  const bool ok = blocks3(L, sm, bl);
  std::printf("%d %zu\n", ok ? 1 : 0, bl.size());
  if (!ok) return 0;
  std::vector<int> owner(L.nn, -1);
  bool shapes = true;
  auto adj = [&](long long a, long long b) {
    const long long d = a > b ? a - b : b - a;
    return d == 1 || d == nx1 || d == plane;
  };
  for (size_t b = 0; b < bl.size(); ++b) {
    const HBlock3 &h = bl[b];
    if (h.skel) {
      for (int c = 0; c < 8; ++c) owner[h.corner[c]] = (int)b;
      for (const auto &e : h.edges) {
        const long long st = step_of(e.dir, nx1, plane);
        for (size_t r = 0; r < e.nodes.size(); ++r) {
          owner[e.nodes[r]] = (int)b;
          if (e.nodes[r] != h.corner[e.a] + (long long)(r + 1) * st) shapes = false;
        }
        if (h.corner[e.b] != h.corner[e.a] + (long long)(e.nodes.size() + 1) * st) shapes = false;
      }
      continue;
    }
    if (h.junc >= 0) owner[h.junc] = (int)b;
    for (size_t c = 0; c < h.chains.size(); ++c) {
      const auto &ch = h.chains[c];
      for (size_t r = 0; r < ch.size(); ++r) {
        owner[ch[r]] = (int)b;
        if (r > 0 && !adj(ch[r], ch[r - 1])) shapes = false;
      }
      if (h.jlast[c] >= 0 && ch.back() + step_of(h.jlast[c], nx1, plane) != h.junc) shapes = false;
      if (h.jfirst[c] >= 0 && ch.front() + step_of(h.jfirst[c], nx1, plane) != h.junc) shapes = false;
    }
  }
  for (size_t p = 0; p < L.nn; ++p) std::printf("%d\n", owner[p]);
  for (const auto &h : bl) std::printf("%d\n", h.colour);
  std::printf("%d\n", shapes ? 1 : 0);
  return 0;
}
