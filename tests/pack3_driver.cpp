// Lays out the 3D warp lists of csrc/pack3_host.h for the sizes, smoother and
// colour read on stdin (nx ny nz smoother colour) and checks the layout the
// kernels of seq3.cuh rely on.  Prints "ok nwarp K W valid_slots nskel" or
// "fail <what>".
#include <cstdio>
#include <set>
#include <vector>

#include "pack3_host.h"

using namespace tmg;

static long long step_of(unsigned d, int nx1, long long plane) {
  const long long s[6] = {1, -1, nx1, -(long long)nx1, plane, -plane};
  return s[d];
}

int main() {
  int nx, ny, nz, sm, colour;
  if (std::scanf("%d %d %d %d %d", &nx, &ny, &nz, &sm, &colour) != 5) return 2;
  Level3 L;
  L.nx = nx; L.ny = ny; L.nz = nz;
  L.nn = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
  const int nx1 = nx + 1;
  const long long plane = (long long)nx1 * (ny + 1);
  std::vector<HBlock3> bl;
  if (!blocks3(L, sm, bl)) { std::printf("fail blocks\n"); return 0; }
  const bool multi = sm == SM3_WIREFRAME;
  Pack3 pk;
  if (pack3(L, bl, colour, multi, pk) != MG_OK) { std::printf("fail pack\n"); return 0; }
  auto fail = [](const char *w) { std::printf("fail %s\n", w); return 0; };
  auto pos = [&](uint32_t ijk) {
    return (long long)(ijk >> 20) * plane + (long long)((ijk >> 10) & 1023u) * nx1 + (long long)(ijk & 1023u);
  };
  const int cap = 32 * pk.W * pk.K;
  if (pk.nodes.size() != (size_t)pk.nwarp * cap || pk.jofs.size() != (size_t)pk.nwarp + 1) return fail("sizes");
  // the nodes each block must contribute (chains; junctions and skeletons apart)
  std::vector<int> want(L.nn, -1);
  long long nwant = 0;
  for (size_t b = 0; b < bl.size(); ++b)
    if (bl[b].colour == colour && !bl[b].skel)
      for (const auto &ch : bl[b].chains)
        for (long long p : ch) { want[p] = (int)b; ++nwant; }
  std::vector<int> seen(L.nn, 0);
  long long valid = 0;
  for (int w = 0; w < pk.nwarp; ++w) {
    const int j0 = multi ? pk.jofs[w] : w, nj = multi ? pk.jofs[w + 1] - pk.jofs[w] : 1;
    if (nj < 0 || nj > (multi ? WJ3_MAX : 1)) return fail("junction count");
    for (int s = 0; s < cap; ++s) {
      const WNode3 &n = pk.nodes[(size_t)w * cap + s];
      if (!(n.fl & WN3_VALID)) {
        if (n.fl != 0 || n.ijk != 0) return fail("unused slot not zero");
        continue;
      }
      ++valid;
      const long long p = pos(n.ijk);
      if (p < 0 || (size_t)p >= L.nn || want[p] < 0 || seen[p]++) return fail("node placement");
      const WNode3 *prev = s > 0 ? &pk.nodes[(size_t)w * cap + s - 1] : nullptr;
      const WNode3 *next = s + 1 < cap ? &pk.nodes[(size_t)w * cap + s + 1] : nullptr;
      if (n.fl & WN3_PRED) {
        if (!prev || !(prev->fl & WN3_VALID) || pos(prev->ijk) != p + step_of(n.fl & 7u, nx1, plane))
          return fail("predecessor");
        if (!(prev->fl & WN3_SUCC)) return fail("predecessor without successor");
      } else if (prev && (prev->fl & WN3_SUCC)) {
        return fail("chain break");
      }
      if ((n.fl & WN3_SUCC) && (!next || pos(next->ijk) != p + step_of((n.fl >> 4) & 7u, nx1, plane)))
        return fail("successor");
      if (n.fl & WN3_JUNC) {
        const unsigned jl = (n.fl >> WN3_JSHIFT) & 31u;
        if ((int)jl >= nj) return fail("junction index");
        const WJunc3 &J = pk.jn[j0 + jl];
        if (pos(J.ijk) != p + step_of((n.fl >> 8) & 7u, nx1, plane)) return fail("junction direction");
        bool found = false;
        for (int e = 0; e < J.natt; ++e)
          if (J.as[e] == s && ((J.adirs >> (3 * e)) & 7u) == (((n.fl >> 8) & 7u) ^ 1u)) found = true;
        if (!found) return fail("junction attachment");
      }
    }
    for (int e = 0; e < nj; ++e) {
      const WJunc3 &J = pk.jn[j0 + e];
      for (int a = 0; a < J.natt; ++a) {
        const WNode3 &n = pk.nodes[(size_t)w * cap + J.as[a]];
        if (!(n.fl & WN3_VALID) || !(n.fl & WN3_JUNC)) return fail("attachment slot");
      }
    }
  }
  if (valid != nwant) return fail("node count");
  for (size_t p = 0; p < L.nn; ++p)
    if (want[p] >= 0 && seen[p] != 1) return fail("node missing");
  // skeletons: offsets consecutive from 0, corners of the right colour
  unsigned off = 0;
  for (const auto &S : pk.skel) {
    if (S.eoff[0] != off) return fail("skeleton offsets");
    for (int e = 0; e < 12; ++e)
      if (S.eoff[e + 1] <= S.eoff[e] || S.ea[e] >= 8 || S.eb[e] >= 8 || S.ed[e] >= 6) return fail("skeleton edge");
    off = S.eoff[12];
  }
  if ((int)off != pk.skel_nodes) return fail("skeleton nodes");
  std::printf("ok %d %d %d %lld %zu\n", pk.nwarp, pk.K, pk.W, valid, pk.skel.size());
  return 0;
}
