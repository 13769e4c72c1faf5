// Statistics of the cluster plan of csrc/cluster_host.h at the default sizes
// for (nx ny wl colour) read on stdin: ok ncta ntile chunk_nodes junctions
// total max_segments_per_cta idle_ctas.
#include <algorithm>
#include <cstdio>

#include "cluster_host.h"

using namespace tmg;

int main() {
  int nx, ny, wl, colour;
  if (std::scanf("%d %d %d %d", &nx, &ny, &wl, &colour) != 4) return 2;
  cluster::PlanHost P;
  cluster::plan(nx, ny, wl, colour, P);
  long nodes = 0, junc = 0;
  for (const auto &l : P.lanes) nodes += l.q1;
  for (const auto &b : P.blocks) junc += b.junc;
  int max_seg = 0, idle = 0;
  for (const auto &c : P.ctas) {
    max_seg = std::max(max_seg, (int)c.nseg);
    idle += c.group < 0;
  }
  std::printf("%d %zu %zu %ld %ld %d %d %d\n", P.ok ? 1 : 0, P.ctas.size(), P.tiles.size(), nodes, junc, P.total,
              max_seg, idle);
  return 0;
}
