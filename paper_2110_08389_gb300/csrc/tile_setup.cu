// tile_setup.cu -- host construction of the tiled line path (see TileList in
// mg_internal.h) for tweed and zebra relaxation on large levels.
//
// Every block is written as legs that start at a wall plus at most one
// junction: a tweed L-block (Sec. 3, Fig. 6) is the corner node (k, k) with a
// vertical leg from the y-wall and a horizontal leg from the x-wall (the
// m-legged system of Eq. mLThomas with m = 2); the centre cross and the
// T-blocks have 4 and 3 legs; the straight lines of a rectangle and the zebra
// lines are single legs from wall to wall; the corner points are junctions
// without legs.  Blocks with the same shape whose legs are parallel and start
// at the same wall (neighbouring same-colour levels of one corner, or
// neighbouring lines) form groups of up to 32, one per tile lane.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "mg_internal.h"
#include "tile_host.h"

namespace tmg {

namespace {

template <typename X>
size_t align16(size_t n) { return (n * sizeof(X) + 15) & ~size_t(15); }

}  // namespace

mg_status build_tiles(Grid &g, int level, int wl) {
  Level &L = g.lev[level];
  if (L.tl_built[wl]) return MG_OK;
  L.tl_built[wl] = true;
  if (std::min(L.nx, L.ny) < TILE_MIN_SIDE || (wl != WL_TWEED && wl != WL_ZEBRA_X && wl != WL_ZEBRA_Y))
    return MG_OK;
  for (int colour = 0; colour < 2; ++colour) {
    tile::TileHost th;
    tile::layout(L.nx, L.ny, wl, colour, th);
    const std::vector<TileDesc> &tiles = th.tiles;
    const std::vector<TileLane> &lanes = th.lanes;
    const std::vector<BlockDesc> &blocks = th.blocks;
    const int total = th.total, max_chunks = th.max_chunks;
    TileList &T = L.tl[wl][colour];
    T.ntile = (int)tiles.size();
    T.nblock = (int)blocks.size();
    T.ngroup = T.nblock / 32;
    T.total_nodes = total;
    T.max_leg_chunks = max_chunks;
    const size_t s0 = align16<TileDesc>(std::max<size_t>(tiles.size(), 1)),
                 s1 = align16<TileLane>(std::max<size_t>(lanes.size(), 1)),
                 s2 = align16<BlockDesc>(std::max<size_t>(blocks.size(), 1));
    const bool consts = (g.prec_mask & 2) && max_chunks <= TILE_PC_CHUNKS && !tiles.empty() && tile::pc_slots_ok(th);
    const size_t s3 = consts ? tiles.size() * 32 * (16 + 8) : 0;  // per lane chunk: float4 + float2
    char *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, s0 + s1 + s2 + s3);
    if (e != cudaSuccess) { set_error("cudaMalloc(tiles)", e); return MG_ERR_ALLOC; }
    T.mem = mem;
    T.tile = reinterpret_cast<TileDesc *>(mem);
    T.lane = reinterpret_cast<TileLane *>(mem + s0);
    T.block = reinterpret_cast<BlockDesc *>(mem + s0 + s1);
    T.cconst = consts ? mem + s0 + s1 + s2 : nullptr;
    if (!tiles.empty()) e = cudaMemcpy(T.tile, tiles.data(), sizeof(TileDesc) * tiles.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !lanes.empty())
      e = cudaMemcpy(T.lane, lanes.data(), sizeof(TileLane) * lanes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !blocks.empty())
      e = cudaMemcpy(T.block, blocks.data(), sizeof(BlockDesc) * blocks.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { set_error("cudaMemcpy(tiles)", e); return MG_ERR_CUDA; }
    g.tile_cap = std::max(g.tile_cap, (size_t)T.ntile);
  }
  return MG_OK;
}

}  // namespace tmg
