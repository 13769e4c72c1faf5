// tile3_host.h -- host part of the 3D tiled tweed path (tiles3.cu): the 3D
// tweed blocks of one colour (blocks3_host.h) rewritten as straight legs plus
// at most one junction, their 32-node chunks packed into tiles of 32 lanes x
// 32 positions, and block records (32 per group) that list their legs'
// chunk slots: the layout tiles3.cu reads.  Plain C++, so that the layout is
// also checked on the CPU (tests/test_tile3_host.py).
//
// A 3D tweed block (Sec. 7: a level set of the two largest sorted wall
// distances) is a point, a straight line, an L of two straight arms (a line
// with one bend), or a star of three to six straight legs on one branch
// node.  The bend or the branch node is the junction; every leg runs from its
// free end (the node before it is outside the block) to the node next to the
// junction, or, in a line, from one free end to the other.
#pragma once
#include <algorithm>
#include <cstring>
#include <tuple>
#include <vector>

#include "blocks3_host.h"

namespace tmg {
namespace tile3 {

struct Leg3 {
  int dir = 0, start = 0, c1 = 0, c2 = 0, len = 0;  // run direction, run coordinate of the first node, fixed coordinates
};
struct Spec3 {
  bool junc = false;
  int ji = 0, jj = 0, jk = 0;
  std::vector<Leg3> legs;
};

struct Tile3Host {
  std::vector<Tile3Desc> tiles;
  std::vector<Tile3Lane> lanes;   // 32 per tile
  std::vector<Block3Desc> blocks; // 32 per group
  std::vector<uint32_t> slots;    // chunk lane slots of every leg, leg by leg
  int max_chunks = 0, ngroup = 0;
};

// run coordinate and fixed coordinates of node (i, j, k) for a run along dir
inline void run_coords(int dir, int i, int j, int k, int &v, int &c1, int &c2) {
  if (dir < 2) { v = i; c1 = j; c2 = k; }
  else if (dir < 4) { v = j; c1 = i; c2 = k; }
  else { v = k; c1 = i; c2 = j; }
}

// The legs and junction of every block of colour `colour`; false if a block
// is not a point, line, L or star of straight legs (at most six).
inline bool specs(const Level3 &L, const std::vector<HBlock3> &blocks, int colour, std::vector<Spec3> &out) {
  const int nx1 = L.nx + 1;
  const size_t plane = (size_t)nx1 * (L.ny + 1);
  auto ijk = [&](long long p, int &i, int &j, int &k) {
    i = (int)(p % nx1); j = (int)((p / nx1) % (L.ny + 1)); k = (int)(p / (long long)plane);
  };
  const long long step[6] = {1, -1, nx1, -(long long)nx1, (long long)plane, -(long long)plane};
  // a straight chain from its first node: the leg (dir toward the chain's
  // end, or toward `toward` for a single node)
  auto make_leg = [&](const std::vector<long long> &ch, long long toward, Leg3 &lg) {
    int d = -1;
    if (ch.size() >= 2) d = dir_between(nx1, plane, ch[0], ch[1]);
    else if (toward >= 0) d = dir_between(nx1, plane, ch[0], toward);
    else return false;
    for (size_t r = 1; r < ch.size(); ++r)
      if (ch[r] - ch[r - 1] != step[d]) return false;
    if (toward >= 0 && toward - ch.back() != step[d]) return false;
    int i, j, k;
    ijk(ch[0], i, j, k);
    lg.dir = d;
    run_coords(d, i, j, k, lg.start, lg.c1, lg.c2);
    lg.len = (int)ch.size();
    return true;
  };
  for (const HBlock3 &hb : blocks) {
    if (hb.colour != colour) continue;
    if (hb.skel) return false;
    Spec3 s;
    long long junc = hb.junc;
    std::vector<std::vector<long long>> legs;
    if (junc >= 0) {
      for (size_t c = 0; c < hb.chains.size(); ++c) {
        if (hb.jfirst[c] >= 0 || hb.jlast[c] < 0) return false;  // tweed stars only: legs end next to the centre
        legs.push_back(hb.chains[c]);
      }
    } else {
      if (hb.chains.size() != 1) return false;
      const std::vector<long long> &ch = hb.chains[0];
      if (ch.size() == 1) {
        junc = ch[0];  // a point: its junction row alone
      } else {
        // bends: where the step changes
        std::vector<size_t> bends;
        for (size_t r = 1; r + 1 < ch.size(); ++r)
          if (ch[r + 1] - ch[r] != ch[r] - ch[r - 1]) bends.push_back(r);
        if (bends.size() > 1) return false;
        if (bends.empty()) {
          legs.push_back(ch);
        } else {
          const size_t b = bends[0];
          junc = ch[b];
          legs.emplace_back(ch.begin(), ch.begin() + (long)b);
          std::vector<long long> rev(ch.begin() + (long)b + 1, ch.end());
          std::reverse(rev.begin(), rev.end());
          legs.push_back(rev);
        }
      }
    }
    if (legs.size() > 6) return false;
    if (junc >= 0) {
      s.junc = true;
      ijk(junc, s.ji, s.jj, s.jk);
    }
    for (const auto &ch : legs) {
      if (ch.empty()) return false;
      Leg3 lg;
      if (!make_leg(ch, s.junc ? junc : -1, lg)) return false;
      s.legs.push_back(lg);
    }
    // canonical leg order
    std::sort(s.legs.begin(), s.legs.end(), [](const Leg3 &a, const Leg3 &b) {
      return std::make_tuple(a.dir, a.start, a.c2, a.c1) < std::make_tuple(b.dir, b.start, b.c2, b.c1);
    });
    out.push_back(std::move(s));
  }
  return true;
}

// The tiles: every chunk of every leg is one lane.  Chunks at the same 32
// positions (run direction and base) form a class; within a class, runs
// along y or z are ordered by their fixed coordinate other than x, then by
// x, so that consecutive lanes are neighbours in x (coalesced), and runs
// along x by (z, y).  Each class is packed densely, 32 lanes per tile, so a
// short leg's chunk shares its tile with chunks of other blocks.  The block
// records list their legs' chunk slots; blocks are grouped 32 per record
// group in order of their number of legs, so that a group's blocks take
// about the same time in tile3_couple.
inline bool layout(const Level3 &L, const std::vector<HBlock3> &blocks, int colour, Tile3Host &out) {
  out = Tile3Host();
  std::vector<Spec3> sp;
  if (!specs(L, blocks, colour, sp)) return false;
  struct Chunk {
    int dir, base, c1, c2, q1, flags, b, l, r;
  };
  std::vector<Chunk> ch;
  for (size_t b = 0; b < sp.size(); ++b)
    for (size_t l = 0; l < sp[b].legs.size(); ++l) {
      const Leg3 &lg = sp[b].legs[l];
      const int stp = (lg.dir & 1) ? -1 : 1, nt = (lg.len + CMAX - 1) / CMAX;
      out.max_chunks = std::max(out.max_chunks, nt);
      for (int r = 0; r < nt; ++r) {
        const int rem = lg.len - CMAX * r;
        int fl = r == 0 ? TL_FIRST : 0;
        if (rem <= CMAX) fl |= sp[b].junc ? TL_LAST_J : TL_LAST_W;
        ch.push_back(Chunk{lg.dir, lg.start + CMAX * r * stp, lg.c1, lg.c2, std::min(CMAX, rem), fl, (int)b, (int)l, r});
      }
    }
  std::stable_sort(ch.begin(), ch.end(), [](const Chunk &a, const Chunk &b) {
    return std::make_tuple(a.dir, a.base, a.c2, a.c1) < std::make_tuple(b.dir, b.base, b.c2, b.c1);
  });
  // slot of chunk r of leg l of block b
  std::vector<std::vector<std::vector<uint32_t>>> slot(sp.size());
  for (size_t b = 0; b < sp.size(); ++b) {
    slot[b].resize(sp[b].legs.size());
    for (size_t l = 0; l < sp[b].legs.size(); ++l) slot[b][l].resize((sp[b].legs[l].len + CMAX - 1) / CMAX);
  }
  size_t c0 = 0;
  while (c0 < ch.size()) {
    size_t c1 = c0 + 1;
    while (c1 < ch.size() && c1 - c0 < 32 && ch[c1].dir == ch[c0].dir && ch[c1].base == ch[c0].base) ++c1;
    const uint32_t t = (uint32_t)out.tiles.size();
    Tile3Desc td;
    std::memset(&td, 0, sizeof(td));
    td.base = (uint16_t)ch[c0].base;
    td.dir = (uint8_t)ch[c0].dir;
    out.tiles.push_back(td);
    for (size_t q = 0; q < 32; ++q) {
      Tile3Lane tl;
      std::memset(&tl, 0, sizeof(tl));
      if (c0 + q < c1) {
        const Chunk &c = ch[c0 + q];
        tl.c1 = (uint16_t)c.c1;
        tl.c2 = (uint16_t)c.c2;
        tl.q1 = (uint8_t)c.q1;
        tl.flags = (uint8_t)c.flags;
        slot[c.b][c.l][c.r] = t * 32 + (uint32_t)q;
      }
      out.lanes.push_back(tl);
    }
    c0 = c1;
  }
  std::vector<int> ord(sp.size());
  for (size_t b = 0; b < ord.size(); ++b) ord[b] = (int)b;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    return std::make_tuple(sp[a].legs.size(), sp[a].jk, sp[a].jj, sp[a].ji) <
           std::make_tuple(sp[b].legs.size(), sp[b].jk, sp[b].jj, sp[b].ji);
  });
  for (size_t g0 = 0; g0 < ord.size(); g0 += 32) {
    std::vector<Block3Desc> bd(32);
    std::memset(bd.data(), 0, sizeof(Block3Desc) * 32);
    for (size_t q = 0; q < 32 && g0 + q < ord.size(); ++q) {
      const int b = ord[g0 + q];
      const Spec3 &s = sp[b];
      Block3Desc &d = bd[q];
      d.ji = (uint16_t)s.ji; d.jj = (uint16_t)s.jj; d.jk = (uint16_t)s.jk;
      d.nleg = (uint8_t)s.legs.size();
      d.junc = s.junc ? 1 : 0;
      for (size_t l = 0; l < s.legs.size(); ++l) {
        d.jdirs |= (uint32_t)(s.legs[l].dir ^ 1) << (3 * l);
        d.leg_slot0[l] = (uint32_t)out.slots.size();
        d.leg_len[l] = (uint16_t)s.legs[l].len;
        out.slots.insert(out.slots.end(), slot[b][l].begin(), slot[b][l].end());
      }
    }
    out.blocks.insert(out.blocks.end(), bd.begin(), bd.end());
    ++out.ngroup;
  }
  return true;
}

}  // namespace tile3
}  // namespace tmg
