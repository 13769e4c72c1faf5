// cluster_setup.cu -- host construction of the cluster pass (see ClusterPlan
// in mg_internal.h): the plans of cluster_host.h uploaded to the device.
#include <algorithm>
#include <cstring>

#include "cluster_host.h"
#include "mg_internal.h"

namespace tmg {

namespace {

template <typename X>
size_t align16(size_t n) { return (n * sizeof(X) + 15) & ~size_t(15); }

}  // namespace

// The cluster pass plans of both colours, uploaded; none (ncta = 0) when a
// colour's groups do not fit a cluster.
mg_status build_cluster_plans(Grid &g, int level, int wl) {
  Level &L = g.lev[level];
  if (!g.cluster_ok || std::min(L.nx, L.ny) < TILE_MIN_SIDE || L.cp[wl][0].ncta > 0 ||
      (wl != WL_TWEED && wl != WL_ZEBRA_X && wl != WL_ZEBRA_Y))
    return MG_OK;
  cluster::PlanHost ph[2];
  for (int colour = 0; colour < 2; ++colour) {
    cluster::plan(L.nx, L.ny, wl, colour, ph[colour]);
    if (!ph[colour].ok) return MG_OK;
  }
  for (int colour = 0; colour < 2; ++colour) {
    const cluster::PlanHost &P = ph[colour];
    ClusterPlan &C = L.cp[wl][colour];
    const size_t s0 = align16<CTile>(P.tiles.size() + 1), s1 = align16<CLane>(P.lanes.size() + 1),
                 s2 = align16<CCta>(P.ctas.size()), s3 = align16<CSeg>(P.segs.size() + 1),
                 s4 = align16<CBlock>(P.blocks.size()), s5 = align16<CChain>(P.chains.size());
    char *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, s0 + s1 + s2 + s3 + s4 + s5);
    if (e != cudaSuccess) { set_error("cudaMalloc(cluster plan)", e); return MG_ERR_ALLOC; }
    C.mem = mem;
    C.tile = reinterpret_cast<CTile *>(mem);
    C.lane = reinterpret_cast<CLane *>(mem + s0);
    C.cta = reinterpret_cast<CCta *>(mem + s0 + s1);
    C.seg = reinterpret_cast<CSeg *>(mem + s0 + s1 + s2);
    C.block = reinterpret_cast<CBlock *>(mem + s0 + s1 + s2 + s3);
    C.chain = reinterpret_cast<CChain *>(mem + s0 + s1 + s2 + s3 + s4);
    auto up = [&](void *dst, const void *src, size_t n) {
      if (e == cudaSuccess && n > 0) e = cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    };
    up(C.tile, P.tiles.data(), sizeof(CTile) * P.tiles.size());
    up(C.lane, P.lanes.data(), sizeof(CLane) * P.lanes.size());
    up(C.cta, P.ctas.data(), sizeof(CCta) * P.ctas.size());
    up(C.seg, P.segs.data(), sizeof(CSeg) * P.segs.size());
    up(C.block, P.blocks.data(), sizeof(CBlock) * P.blocks.size());
    up(C.chain, P.chains.data(), sizeof(CChain) * P.chains.size());
    if (e != cudaSuccess) { set_error("cudaMemcpy(cluster plan)", e); return MG_ERR_CUDA; }
    C.ncta = (int)P.ctas.size();
    C.ntile = (int)P.tiles.size();
    C.nseg = (int)P.segs.size();
    C.ngroup = (int)P.blocks.size() / 32;
  }
  return MG_OK;
}

}  // namespace tmg
