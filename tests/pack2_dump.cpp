// Prints the 2D warp list of csrc/pack2_host.h for (nx ny smoother colour
// kmax kpref) read on stdin (smoother 0 zebra x, 1 zebra y, 2 tweed,
// 3 wireframe): "ok nwarp K W", every slot (i j fl) and every sequence's
// junction record (has_j ji jj natt adirs as[0..3]); "none" if the blocks do
// not fit the warp path.
#include <cstdio>
#include <vector>

#include "pack2_host.h"

using namespace tmg;

int main() {
  int nx, ny, sm, colour, kmax, kpref;
  if (std::scanf("%d %d %d %d %d %d", &nx, &ny, &sm, &colour, &kmax, &kpref) != 6) return 2;
  std::vector<HBlock> bl;
  if (sm <= 1) zebra_blocks(nx, ny, colour, sm == 0, bl);
  else if (sm == 2) tweed_blocks(nx, ny, colour, bl);
  else wireframe_blocks(nx, ny, colour, bl);
  Pack2 pk;
  if (!pack2(bl, kmax, kpref, pk)) { std::printf("none\n"); return 0; }
  std::printf("ok %d %d %d\n", pk.nwarp, pk.K, pk.W);
  for (const auto &n : pk.nodes) std::printf("%u %u %u\n", (unsigned)n.i, (unsigned)n.j, n.fl);
  for (const auto &b : pk.blk) {
    std::printf("%u %u %u %u %u", (unsigned)b.has_j, (unsigned)b.ji, (unsigned)b.jj, (unsigned)b.natt,
                (unsigned)b.adirs);
    for (int e = 0; e < 4; ++e) std::printf(" %u", (unsigned)b.as[e]);
    std::printf("\n");
  }
  return 0;
}
