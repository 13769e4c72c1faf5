// tile_host.h -- host part of the tiled line path (tile_setup.cu): every
// block of a tweed or zebra colour written as legs from a wall plus at most
// one junction, grouped (up to 32 blocks of one shape) into tiles of 32
// lanes x 32 positions and 32 block records per group, the layout tiles.cu
// reads.  Plain C++, so that the layout is also checked on the CPU.
#pragma once
#include <algorithm>
#include <cstring>
#include <tuple>
#include <vector>

#include "mg_internal.h"

namespace tmg {
namespace tile {

struct LegSpec {
  int start, line, dir, len;  // run coordinate of the first node, fixed coordinate, direction, nodes
};
struct BlockSpec {
  bool junc = false;
  int ji = 0, jj = 0;
  std::vector<LegSpec> legs;
  int gkey = 0, pos = 0;  // group key and order within the group
};

inline int colour_of(int k) { return (k & 1) ? 0 : 1; }

// leg in direction dir whose first node is (i, j)
inline LegSpec leg(int i, int j, int dir, int len) {
  const bool xrun = dir < 2;
  return LegSpec{xrun ? i : j, xrun ? j : i, dir, len};
}

inline void tweed_specs(int nx, int ny, int colour, std::vector<BlockSpec> &out) {
  const int hx = nx / 2, hy = ny / 2, K = std::max(hx, hy), m = std::min(hx, hy);
  for (int k = 1; k <= K; ++k) {
    if (colour_of(k) != colour) continue;
    if (k < m) {
      const int cx[2] = {k, nx - k}, cy[2] = {k, ny - k};
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          BlockSpec s;
          s.junc = true; s.ji = cx[a]; s.jj = cy[b];
          if (k >= 2) {
            s.legs.push_back(leg(cx[a], b == 0 ? 1 : ny - 1, b == 0 ? DIR_PY : DIR_MY, k - 1));
            s.legs.push_back(leg(a == 0 ? 1 : nx - 1, cy[b], a == 0 ? DIR_PX : DIR_MX, k - 1));
            s.gkey = 2 * a + b;
          } else {
            s.gkey = 10;  // the four corner points
          }
          s.pos = k;
          out.push_back(s);
        }
    } else if (k == m) {
      auto star = [&](int i, int j, std::vector<LegSpec> legs, int key) {
        BlockSpec s;
        s.junc = true; s.ji = i; s.jj = j;
        for (auto &l : legs)
          if (l.len > 0) s.legs.push_back(l);
        s.gkey = key;
        out.push_back(s);
      };
      if (hx == hy) {
        star(k, k, {leg(1, k, DIR_PX, k - 1), leg(nx - 1, k, DIR_MX, k - 1), leg(k, 1, DIR_PY, k - 1),
                    leg(k, ny - 1, DIR_MY, k - 1)}, 20);
      } else if (hx > hy) {
        star(k, k, {leg(1, k, DIR_PX, k - 1), leg(k, 1, DIR_PY, k - 1), leg(k, ny - 1, DIR_MY, ny - 1 - k)}, 21);
        star(nx - k, k, {leg(nx - 1, k, DIR_MX, k - 1), leg(nx - k, 1, DIR_PY, k - 1),
                         leg(nx - k, ny - 1, DIR_MY, ny - 1 - k)}, 22);
      } else {
        star(k, k, {leg(k, 1, DIR_PY, k - 1), leg(1, k, DIR_PX, k - 1), leg(nx - 1, k, DIR_MX, nx - 1 - k)}, 21);
        star(k, ny - k, {leg(k, ny - 1, DIR_MY, k - 1), leg(1, ny - k, DIR_PX, k - 1),
                         leg(nx - 1, ny - k, DIR_MX, nx - 1 - k)}, 22);
      }
    } else {
      // straight lines perpendicular to the nearest walls, wall to wall
      const int lines[2] = {k, (hx > hy ? nx : ny) - k};
      for (int t = 0; t < (lines[0] == lines[1] ? 1 : 2); ++t) {
        BlockSpec s;
        s.legs.push_back(hx > hy ? leg(lines[t], 1, DIR_PY, ny - 1) : leg(1, lines[t], DIR_PX, nx - 1));
        s.gkey = 30;
        s.pos = lines[t];
        out.push_back(s);
      }
    }
  }
}

inline void zebra_specs(int nx, int ny, int colour, bool along_x, std::vector<BlockSpec> &out) {
  const int n = along_x ? ny : nx;
  for (int t = 1; t < n; ++t) {
    if (colour_of(t) != colour) continue;
    BlockSpec s;
    s.legs.push_back(along_x ? leg(1, t, DIR_PX, nx - 1) : leg(t, 1, DIR_PY, ny - 1));
    s.gkey = 0;
    s.pos = t;
    out.push_back(s);
  }
}

struct TileHost {
  std::vector<TileDesc> tiles;
  std::vector<TileLane> lanes;   // 32 per tile
  std::vector<BlockDesc> blocks; // 32 per group
  int total = 0, max_chunks = 0;
};

// The tiles of one colour of smoother wl (WL_TWEED, WL_ZEBRA_X, WL_ZEBRA_Y)
// on an nx x ny level.
inline void layout(int nx, int ny, int wl, int colour, TileHost &out) {
  out = TileHost();
  std::vector<BlockSpec> specs;
  if (wl == WL_TWEED) tweed_specs(nx, ny, colour, specs);
  else zebra_specs(nx, ny, colour, wl == WL_ZEBRA_X, specs);
  // group: same key and shape (legs parallel, same wall), consecutive positions
  std::stable_sort(specs.begin(), specs.end(), [](const BlockSpec &a, const BlockSpec &b) {
    return std::make_tuple(a.gkey, (int)a.legs.size(), a.pos) < std::make_tuple(b.gkey, (int)b.legs.size(), b.pos);
  });
  std::vector<TileDesc> &tiles = out.tiles;
  std::vector<TileLane> &lanes = out.lanes;
  std::vector<BlockDesc> &blocks = out.blocks;
  int &total = out.total, &max_chunks = out.max_chunks;
  size_t b0 = 0;
  while (b0 < specs.size()) {
    size_t b1 = b0 + 1;
    auto same_shape = [&](const BlockSpec &a, const BlockSpec &b) {
      if (a.gkey != b.gkey || a.legs.size() != b.legs.size() || a.junc != b.junc) return false;
      for (size_t l = 0; l < a.legs.size(); ++l)
        if (a.legs[l].dir != b.legs[l].dir || a.legs[l].start != b.legs[l].start) return false;
      return true;
    };
    while (b1 < specs.size() && b1 - b0 < 32 && same_shape(specs[b0], specs[b1])) ++b1;
    const int nb = (int)(b1 - b0), nleg = (int)specs[b0].legs.size();
    std::vector<BlockDesc> bd(32);
    std::memset(bd.data(), 0, sizeof(BlockDesc) * 32);
    for (int l = 0; l < nleg; ++l) {
      int maxlen = 0;
      for (int b = 0; b < nb; ++b) maxlen = std::max(maxlen, specs[b0 + b].legs[l].len);
      const int nt = (maxlen + CMAX - 1) / CMAX;
      max_chunks = std::max(max_chunks, nt);
      const LegSpec &ref = specs[b0].legs[l];
      const int step = (ref.dir == DIR_PX || ref.dir == DIR_PY) ? 1 : -1;
      const uint32_t t0 = (uint32_t)tiles.size();
      for (int r = 0; r < nt; ++r) {
        TileDesc td;
        std::memset(&td, 0, sizeof(td));
        td.base = (uint16_t)(ref.start + CMAX * r * step);
        td.dir = (uint8_t)ref.dir;
        tiles.push_back(td);
        for (int b = 0; b < 32; ++b) {
          TileLane tl;
          std::memset(&tl, 0, sizeof(tl));
          if (b < nb) {
            const BlockSpec &s = specs[b0 + b];
            const int rem = s.legs[l].len - CMAX * r;
            tl.line = (uint16_t)s.legs[l].line;
            if (rem > 0) {
              tl.q0 = 0;
              tl.q1 = (uint8_t)std::min(CMAX, rem);
              if (r == 0) tl.flags |= TL_FIRST;
              if (rem <= CMAX) tl.flags |= s.junc ? TL_LAST_J : TL_LAST_W;
            }
          }
          lanes.push_back(tl);
        }
      }
      for (int b = 0; b < nb; ++b) {
        bd[b].leg_tile0[l] = t0;
        bd[b].leg_len[l] = (uint16_t)specs[b0 + b].legs[l].len;
      }
    }
    for (int b = 0; b < nb; ++b) {
      const BlockSpec &s = specs[b0 + b];
      bd[b].ji = (uint16_t)s.ji; bd[b].jj = (uint16_t)s.jj;
      bd[b].nleg = (uint8_t)nleg; bd[b].junc = s.junc ? 1 : 0; bd[b].lane = (uint8_t)b;
      for (int l = 0; l < nleg; ++l) bd[b].jdirs |= (uint8_t)((s.legs[l].dir ^ 1) << (2 * l));
      total += (s.junc ? 1 : 0);
      for (auto &lg : s.legs) total += lg.len;
    }
    blocks.insert(blocks.end(), bd.begin(), bd.end());
    b0 = b1;
  }
}

// True if every block of more than two legs is alone in its group (lane 0):
// tile_couple_pc then gives each leg of a group its own shared-memory slot
// among 64.
inline bool pc_slots_ok(const TileHost &th) {
  for (size_t k = 0; k < th.blocks.size(); ++k)
    if (th.blocks[k].nleg > 2 && k % 32 != 0) return false;
  return true;
}

}  // namespace tile
}  // namespace tmg
