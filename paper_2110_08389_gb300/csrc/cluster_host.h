// cluster_host.h -- host part of the cluster pass (see ClusterPlan in
// mg_internal.h): the tiled path's groups of blocks (tile_host.h) spread over
// the CTAs of thread-block clusters.  Plain C++, so that the plan is also
// checked on the CPU.
//
// A group's tiles are taken leg by leg (chunks from the wall outwards) and
// split evenly over ceil(tiles / tiles_per_cta) CTAs of one cluster; groups
// are packed into clusters of ctas_per_cluster CTAs, largest first.  Every
// leg of every block becomes a chain of chunks, cut into one segment per CTA
// holding some of its chunks.  Block b of a group is solved by the group's
// CTA b mod (its number of CTAs).
#pragma once
#include <algorithm>
#include <cstring>
#include <vector>

#include "mg_internal.h"
#include "tile_host.h"

namespace tmg {
namespace cluster {

struct PlanHost {
  bool ok = false;           // false: a group needs more CTAs than a cluster has
  std::vector<CTile> tiles;
  std::vector<CLane> lanes;  // 32 per tile
  std::vector<CCta> ctas;    // a multiple of ctas_per_cluster
  std::vector<CSeg> segs;
  std::vector<CBlock> blocks;  // 32 per group
  std::vector<CChain> chains;  // 128 per group
  int total = 0;             // unknowns relaxed (junctions included)
};

namespace detail {

// A chunk of a chain: its tile within the group's tile list and its lane.
struct ChunkRef {
  int tile, lane;
};
struct GroupHost {
  std::vector<CTile> tiles;
  std::vector<CLane> lanes;
  std::vector<std::vector<ChunkRef>> chain;  // [l * 32 + b]: chunks from the wall
  CBlock blk[32];
  int nleg = 0;
  bool compact = false;
};

}  // namespace detail

// The plan of one colour of smoother wl (WL_TWEED, WL_ZEBRA_X, WL_ZEBRA_Y) on
// an nx x ny level.
inline void plan(int nx, int ny, int wl, int colour, PlanHost &out, int tiles_per_cta = CL_TILES,
                 int ctas_per_cluster = CL_CTAS) {
  using detail::ChunkRef;
  using detail::GroupHost;
  out = PlanHost();
  tile::TileHost th;
  tile::layout(nx, ny, wl, colour, th);
  out.total = th.total;
  const int ngroup = (int)th.blocks.size() / 32;
  std::vector<GroupHost> groups(ngroup);
  for (int g = 0; g < ngroup; ++g) {
    GroupHost &G = groups[g];
    const BlockDesc *bd = &th.blocks[(size_t)32 * g];
    int nb = 0;
    for (int b = 0; b < 32; ++b)
      if (bd[b].nleg > 0 || bd[b].junc) nb = b + 1;
    G.nleg = bd[0].nleg;
    G.chain.assign(128, {});
    for (int b = 0; b < 32; ++b) {
      CBlock &c = G.blk[b];
      std::memset(&c, 0, sizeof(c));
      if (b < nb) {
        c.ji = bd[b].ji; c.jj = bd[b].jj;
        c.nleg = bd[b].nleg; c.junc = bd[b].junc; c.jdirs = bd[b].jdirs;
      }
    }
    // one block with legs: compact tiles, 32 consecutive chunks of a leg per tile
    G.compact = nb == 1 && G.nleg > 0;
    for (int l = 0; l < G.nleg; ++l) {
      int maxlen = 0;
      for (int b = 0; b < nb; ++b) maxlen = std::max(maxlen, (int)bd[b].leg_len[l]);
      const int nch = (maxlen + CMAX - 1) / CMAX;
      const int t0 = (int)bd[0].leg_tile0[l];
      if (!G.compact) {
        for (int r = 0; r < nch; ++r) {
          const TileDesc &td = th.tiles[t0 + r];
          CTile ct;
          std::memset(&ct, 0, sizeof(ct));
          ct.base = td.base; ct.dir = td.dir;
          const int gt = (int)G.tiles.size();
          G.tiles.push_back(ct);
          for (int b = 0; b < 32; ++b) {
            const TileLane &tl = th.lanes[(size_t)32 * (t0 + r) + b];
            CLane cl;
            std::memset(&cl, 0, sizeof(cl));
            cl.line = tl.line; cl.q1 = tl.q1; cl.flags = tl.flags;
            G.lanes.push_back(cl);
            if (b < nb && tl.q1 > 0) G.chain[l * 32 + b].push_back(ChunkRef{gt, b});
          }
        }
      } else {
        for (int r0 = 0; r0 < nch; r0 += 32) {
          CTile ct;
          std::memset(&ct, 0, sizeof(ct));
          ct.dir = th.tiles[t0].dir; ct.kind = CT_COMPACT;
          const int gt = (int)G.tiles.size();
          G.tiles.push_back(ct);
          for (int k = 0; k < 32; ++k) {
            CLane cl;
            std::memset(&cl, 0, sizeof(cl));
            if (r0 + k < nch) {
              const TileLane &tl = th.lanes[(size_t)32 * (t0 + r0 + k)];
              cl.line = tl.line; cl.q1 = tl.q1; cl.flags = tl.flags;
              cl.cbase = th.tiles[t0 + r0 + k].base;
              if (tl.q1 > 0) G.chain[l * 32].push_back(ChunkRef{gt, k});
            }
            G.lanes.push_back(cl);
          }
        }
      }
    }
  }
  // CTAs per group, then clusters: largest groups first (compact groups, whose
  // legs are long single chains, before all others), first fit
  std::vector<int> need(ngroup), order(ngroup);
  for (int g = 0; g < ngroup; ++g) {
    const int nt = (int)groups[g].tiles.size();
    need[g] = std::max(1, (nt + tiles_per_cta - 1) / tiles_per_cta);
    if (need[g] > ctas_per_cluster) return;  // does not fit: no plan
    order[g] = g;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    if (groups[a].compact != groups[b].compact) return groups[a].compact;
    return need[a] > need[b];
  });
  std::vector<std::vector<int>> clusters;
  std::vector<int> used;
  for (int g : order) {
    size_t c = 0;
    while (c < clusters.size() && used[c] + need[g] > ctas_per_cluster) ++c;
    if (c == clusters.size()) { clusters.emplace_back(); used.push_back(0); }
    clusters[c].push_back(g);
    used[c] += need[g];
  }
  out.blocks.resize((size_t)32 * ngroup);
  out.chains.resize((size_t)128 * ngroup);
  std::memset(out.chains.data(), 0, sizeof(CChain) * out.chains.size());
  for (int g = 0; g < ngroup; ++g)
    for (int b = 0; b < 32; ++b) out.blocks[(size_t)32 * g + b] = groups[g].blk[b];
  for (size_t c = 0; c < clusters.size(); ++c) {
    int rank = 0;
    for (int g : clusters[c]) {
      const GroupHost &G = groups[g];
      const int nt = (int)G.tiles.size(), ngr = need[g];
      // the group's tiles, split as evenly as possible over its CTAs
      std::vector<int> first(ngr + 1);
      for (int r = 0; r <= ngr; ++r) first[r] = (int)((long long)nt * r / ngr);
      for (int r = 0; r < ngr; ++r) {
        CCta cta;
        std::memset(&cta, 0, sizeof(cta));
        cta.tile0 = (int)out.tiles.size();
        cta.group = g;
        cta.seg0 = (int)out.segs.size();
        cta.ntile = (uint8_t)(first[r + 1] - first[r]);
        cta.grank = (uint8_t)r;
        cta.rank0 = (uint8_t)rank;
        cta.ngr = (uint8_t)ngr;
        cta.nleg = (uint8_t)G.nleg;
        for (int t = first[r]; t < first[r + 1]; ++t) {
          out.tiles.push_back(G.tiles[t]);
          for (int k = 0; k < 32; ++k) out.lanes.push_back(G.lanes[(size_t)32 * t + k]);
        }
        // segments: each chain's chunks in this CTA's tiles (consecutive)
        int nseg = 0;
        for (int ch = 0; ch < 128; ++ch) {
          const std::vector<ChunkRef> &refs = G.chain[ch];
          size_t k = 0;
          while (k < refs.size() && refs[k].tile < first[r]) ++k;
          size_t k1 = k;
          while (k1 < refs.size() && refs[k1].tile < first[r + 1]) ++k1;
          if (k1 == k) continue;
          CSeg sg;
          std::memset(&sg, 0, sizeof(sg));
          sg.slot0 = (uint16_t)((refs[k].tile - first[r]) * 32 + refs[k].lane);
          sg.nchunk = (uint16_t)(k1 - k);
          sg.stride = G.compact ? 1 : 32;
          const CLane &lastl = G.lanes[(size_t)32 * refs[k1 - 1].tile + refs[k1 - 1].lane];
          sg.one = lastl.q1 == 1 ? 1 : 0;
          out.segs.push_back(sg);
          CChain &cc = out.chains[(size_t)128 * g + ch];
          cc.rank[cc.nseg] = (uint8_t)(rank + r);
          cc.slot[cc.nseg] = (uint8_t)nseg;
          ++cc.nseg;
          ++nseg;
        }
        cta.nseg = (uint16_t)nseg;
        out.ctas.push_back(cta);
      }
      rank += ngr;
    }
    // places of the (c', d') of each leg in the store of the CTA that solves
    // it: block b of a group by the group's CTA b mod ngr, legs in order
    for (int g : clusters[c]) {
      const GroupHost &G = groups[g];
      const int ngr = need[g];
      for (int r = 0; r < ngr; ++r) {
        int off = 0;
        for (int b = r; b < 32; b += ngr)
          for (int l = 0; l < G.nleg; ++l) {
            CChain &cc = out.chains[(size_t)128 * g + l * 32 + b];
            int rows = 0;
            for (const ChunkRef &ref : G.chain[l * 32 + b])
              rows += G.lanes[(size_t)32 * ref.tile + ref.lane].q1 == 1 ? 1 : 2;
            cc.roff = (uint16_t)off;
            cc.nrow = (uint16_t)rows;
            off += rows;
          }
        if (off > CL_LEGROWS) return;  // more rows than the store holds: no plan
      }
    }
    // idle CTAs fill the cluster
    for (; rank < ctas_per_cluster; ++rank) {
      CCta cta;
      std::memset(&cta, 0, sizeof(cta));
      cta.group = -1;
      cta.tile0 = (int)out.tiles.size();
      cta.seg0 = (int)out.segs.size();
      out.ctas.push_back(cta);
    }
  }
  out.ok = true;
}

}  // namespace cluster
}  // namespace tmg
