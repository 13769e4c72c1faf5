// Prints the 3D warp lists of csrc/pack3_host.h for (nx ny nz smoother
// colour) read on stdin: "nwarp K W nj nskel", then every slot (ijk fl),
// jofs, every junction record (ijk natt adirs as[0..5]) and every skeleton
// (cijk[8] eoff[13] ea[12] eb[12] ed[12]).
#include <cstdio>
#include <vector>

#include "pack3_host.h"

using namespace tmg;

int main() {
  int nx, ny, nz, sm, colour;
  if (std::scanf("%d %d %d %d %d", &nx, &ny, &nz, &sm, &colour) != 5) return 2;
  Level3 L;
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  std::vector<HBlock3> bl;
  if (!blocks3(L, sm, bl)) return 3;
  Pack3 pk;
  if (pack3(L, bl, colour, sm == SM3_WIREFRAME, pk) != MG_OK) return 4;
  std::printf("%d %d %d %zu %zu\n", pk.nwarp, pk.K, pk.W, pk.jn.size(), pk.skel.size());
  for (const auto &n : pk.nodes) std::printf("%u %u\n", n.ijk, n.fl);
  for (int v : pk.jofs) std::printf("%d\n", v);
  for (const auto &J : pk.jn) {
    std::printf("%u %u %u", J.ijk, (unsigned)J.natt, J.adirs);
    for (int e = 0; e < 6; ++e) std::printf(" %u", (unsigned)J.as[e]);
    std::printf("\n");
  }
  for (const auto &S : pk.skel) {
    for (int c = 0; c < 8; ++c) std::printf("%u ", S.cijk[c]);
    for (int e = 0; e < 13; ++e) std::printf("%u ", S.eoff[e]);
    for (int e = 0; e < 12; ++e) std::printf("%u ", (unsigned)S.ea[e]);
    for (int e = 0; e < 12; ++e) std::printf("%u ", (unsigned)S.eb[e]);
    for (int e = 0; e < 12; ++e) std::printf("%u ", (unsigned)S.ed[e]);
    std::printf("\n");
  }
  return 0;
}
