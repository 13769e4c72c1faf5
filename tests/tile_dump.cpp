// Prints the tiled-path layout of csrc/tile_host.h for (nx ny wl colour) read
// on stdin (wl 0 zebra x, 1 zebra y, 2 tweed): "ntile nblock", every tile
// (base dir), every lane (line q0 q1 flags), every block record (ji jj nleg
// junc jdirs lane leg_tile0[4] leg_len[4]).
#include <cstdio>

#include "tile_host.h"

using namespace tmg;

int main() {
  int nx, ny, wl, colour;
  if (std::scanf("%d %d %d %d", &nx, &ny, &wl, &colour) != 4) return 2;
  tile::TileHost th;
  tile::layout(nx, ny, wl, colour, th);
  std::printf("%zu %zu\n", th.tiles.size(), th.blocks.size());
  for (const auto &t : th.tiles) std::printf("%u %u\n", (unsigned)t.base, (unsigned)t.dir);
  for (const auto &l : th.lanes) std::printf("%u %u %u %u\n", (unsigned)l.line, (unsigned)l.q0, (unsigned)l.q1, (unsigned)l.flags);
  for (const auto &b : th.blocks) {
    std::printf("%u %u %u %u %u %u", (unsigned)b.ji, (unsigned)b.jj, (unsigned)b.nleg, (unsigned)b.junc,
                (unsigned)b.jdirs, (unsigned)b.lane);
    for (int l = 0; l < 4; ++l) std::printf(" %u", b.leg_tile0[l]);
    for (int l = 0; l < 4; ++l) std::printf(" %u", (unsigned)b.leg_len[l]);
    std::printf("\n");
  }
  return 0;
}
