// Prints the 3D tiled tweed layout of csrc/tile3_host.h for (nx ny nz colour)
// read on stdin: "ok ntile nblock ngroup nslot", every tile (base
// dir), every lane (c1 c2 q1 flags), every block record (ji jj jk nleg junc
// jdirs leg_slot0[6] leg_len[6]), the slots; or "fail".
#include <cstdio>

#include "tile3_host.h"

using namespace tmg;

int main() {
  int nx, ny, nz, colour;
  if (std::scanf("%d %d %d %d", &nx, &ny, &nz, &colour) != 4) return 2;
  Level3 L;
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  std::vector<HBlock3> bl;
  tile3::Tile3Host th;
  if (!blocks3(L, SM3_TWEED, bl) || !tile3::layout(L, bl, colour, th)) {
    std::printf("fail\n");
    return 0;
  }
  std::printf("ok %zu %zu %d %zu\n", th.tiles.size(), th.blocks.size(), th.ngroup, th.slots.size());
  for (const auto &t : th.tiles) std::printf("%u %u\n", (unsigned)t.base, (unsigned)t.dir);
  for (const auto &l : th.lanes)
    std::printf("%u %u %u %u\n", (unsigned)l.c1, (unsigned)l.c2, (unsigned)l.q1, (unsigned)l.flags);
  for (const auto &b : th.blocks) {
    std::printf("%u %u %u %u %u %u", (unsigned)b.ji, (unsigned)b.jj, (unsigned)b.jk, (unsigned)b.nleg,
                (unsigned)b.junc, (unsigned)b.jdirs);
    for (int l = 0; l < 6; ++l) std::printf(" %u", b.leg_slot0[l]);
    for (int l = 0; l < 6; ++l) std::printf(" %u", (unsigned)b.leg_len[l]);
    std::printf("\n");
  }
  for (uint32_t v : th.slots) std::printf("%u\n", v);
  return 0;
}
