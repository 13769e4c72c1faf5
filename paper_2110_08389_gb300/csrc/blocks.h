// blocks.h -- host description of the blocks of every smoother (Sec. 3):
// chains of straight segments plus at most one junction node.  Built in
// closed form by setup.cu; consumed by its work-list packer.
#pragma once
#include <algorithm>
#include <vector>

#include "mg_internal.h"

namespace tmg {

// A segment: len nodes from (i0, j0) in direction dir (DIR_*).  The first
// node of a chain's next segment is this segment's last node plus one step in
// the next segment's direction.
struct HSeg {
  int i0, j0, dir, len;
};
struct HChain {
  std::vector<HSeg> s;
  bool fj = false, lj = false;
  int ljdir = 0;  // direction from the last node to the junction
};
struct HBlock {
  bool junc = false;
  int ji = 0, jj = 0;
  std::vector<HChain> ch;
  int nodes = 0, chunks = 0;
  int group = 0, pos = 0;  // packing order: blocks of one group in order of pos are
                           // neighbours (adjacent same-colour legs / lines)
};

// The blocks of one colour (0 = red, relaxed first) of each line smoother,
// in closed form from the node's distances to the walls (see setup.cu):
// tweed_blocks, wireframe_blocks, zebra_blocks.  Plain C++, so that they are
// also checked on the CPU against the oracle's partition.
namespace blk {
inline HBlock keyed(HBlock b, int group, int pos) {
  b.group = group;
  b.pos = pos;
  return b;
}

inline HChain line(int i0, int j0, int dir, int len) {
  HChain c;
  c.s.push_back({i0, j0, dir, len});
  return c;
}
inline HChain leg_to_junction(int i0, int j0, int dir, int len) {
  HChain c = line(i0, j0, dir, len);
  c.lj = true;
  c.ljdir = dir;
  return c;
}
inline HBlock point(int i, int j) {
  HBlock b;
  b.junc = true; b.ji = i; b.jj = j;
  return b;
}
inline HBlock single(HChain c) {
  HBlock b;
  b.ch.push_back(c);
  return b;
}
inline HBlock star(int i, int j, std::vector<HChain> legs) {
  HBlock b = point(i, j);
  for (auto &l : legs)
    if (!l.s.empty() && l.s[0].len > 0) b.ch.push_back(l);
  return b;
}
inline int colour_of(int k) { return (k & 1) ? 0 : 1; }
inline HBlock keyed5(HBlock b) { return keyed(b, 5, 0); }

inline void tweed_blocks(int nx, int ny, int colour, std::vector<HBlock> &out) {
  const int hx = nx / 2, hy = ny / 2, K = std::max(hx, hy), m = std::min(hx, hy);
  for (int k = 1; k <= K; ++k) {
    if (colour_of(k) != colour) continue;
    if (k < m) {
      if (k == 1) {
        out.push_back(keyed(point(1, 1), 4, 0)); out.push_back(keyed(point(nx - 1, 1), 4, 1));
        out.push_back(keyed(point(1, ny - 1), 4, 2)); out.push_back(keyed(point(nx - 1, ny - 1), 4, 3));
        continue;
      }
      // leg from the y-wall up to the corner (k,k) of the level, then the leg
      // back along x to the x-wall: one tridiagonal chain of 2k-1 nodes
      const int cx[2] = {k, nx - k}, cy[2] = {k, ny - k};
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          HChain c;
          const int vdir = b == 0 ? DIR_PY : DIR_MY, hdir = a == 0 ? DIR_MX : DIR_PX;
          c.s.push_back({cx[a], b == 0 ? 1 : ny - 1, vdir, k});
          c.s.push_back({a == 0 ? k - 1 : nx - k + 1, cy[b], hdir, k - 1});
          out.push_back(keyed(single(c), 2 * a + b, k));
        }
    } else if (k == m) {
      if (hx == hy) {  // centre cross, m = 4 legs (Eq. mLThomas)
        out.push_back(keyed5(star(k, k, {leg_to_junction(1, k, DIR_PX, k - 1), leg_to_junction(nx - 1, k, DIR_MX, k - 1),
                                  leg_to_junction(k, 1, DIR_PY, k - 1), leg_to_junction(k, ny - 1, DIR_MY, k - 1)})));
      } else if (hx > hy) {  // two T-blocks, arms from the x-walls
        out.push_back(keyed5(star(k, k, {leg_to_junction(1, k, DIR_PX, k - 1), leg_to_junction(k, 1, DIR_PY, k - 1),
                                  leg_to_junction(k, ny - 1, DIR_MY, ny - 1 - k)})));
        out.push_back(keyed5(star(nx - k, k, {leg_to_junction(nx - 1, k, DIR_MX, k - 1),
                                       leg_to_junction(nx - k, 1, DIR_PY, k - 1),
                                       leg_to_junction(nx - k, ny - 1, DIR_MY, ny - 1 - k)})));
      } else {  // two T-blocks, arms from the y-walls
        out.push_back(keyed5(star(k, k, {leg_to_junction(k, 1, DIR_PY, k - 1), leg_to_junction(1, k, DIR_PX, k - 1),
                                  leg_to_junction(nx - 1, k, DIR_MX, nx - 1 - k)})));
        out.push_back(keyed5(star(k, ny - k, {leg_to_junction(k, ny - 1, DIR_MY, k - 1),
                                       leg_to_junction(1, ny - k, DIR_PX, k - 1),
                                       leg_to_junction(nx - 1, ny - k, DIR_MX, nx - 1 - k)})));
      }
    } else if (hx > hy) {  // full columns perpendicular to the y-walls
      out.push_back(keyed(single(line(k, 1, DIR_PY, ny - 1)), 6, k));
      if (nx - k != k) out.push_back(keyed(single(line(nx - k, 1, DIR_PY, ny - 1)), 6, nx - k));
    } else {  // full rows perpendicular to the x-walls
      out.push_back(keyed(single(line(1, k, DIR_PX, nx - 1)), 6, k));
      if (ny - k != k) out.push_back(keyed(single(line(1, ny - k, DIR_PX, nx - 1)), 6, ny - k));
    }
  }
}

inline void wireframe_blocks(int nx, int ny, int colour, std::vector<HBlock> &out) {
  const int hx = nx / 2, hy = ny / 2, m = std::min(hx, hy);
  for (int k = 1; k <= m; ++k) {
    if (colour_of(k) != colour) continue;
    if (k < m) {
      // ring around the box [k, nx-k] x [k, ny-k], opened at the corner (k,k)
      HChain c;
      c.s.push_back({k + 1, k, DIR_PX, nx - 2 * k});
      c.s.push_back({nx - k, k + 1, DIR_PY, ny - 2 * k});
      c.s.push_back({nx - k - 1, ny - k, DIR_MX, nx - 2 * k});
      c.s.push_back({k, ny - k - 1, DIR_MY, ny - 2 * k - 1});
      c.fj = true; c.lj = true; c.ljdir = DIR_MY;
      HBlock b = point(k, k);
      b.ch.push_back(c);
      out.push_back(keyed(b, 0, k));
    } else if (hx == hy) {
      out.push_back(keyed(point(k, k), 1, k));
    } else if (hx > hy) {
      out.push_back(single(line(k, k, DIR_PX, nx - 2 * k + 1)));
    } else {
      out.push_back(single(line(k, k, DIR_PY, ny - 2 * k + 1)));
    }
  }
}

inline void zebra_blocks(int nx, int ny, int colour, bool along_x, std::vector<HBlock> &out) {
  if (along_x) {
    for (int j = 1; j < ny; ++j)
      if (colour_of(j) == colour) out.push_back(keyed(single(line(1, j, DIR_PX, nx - 1)), 0, j));
  } else {
    for (int i = 1; i < nx; ++i)
      if (colour_of(i) == colour) out.push_back(keyed(single(line(i, 1, DIR_PY, ny - 1)), 0, i));
  }
}

}  // namespace blk
using blk::tweed_blocks;
using blk::wireframe_blocks;
using blk::zebra_blocks;

}  // namespace tmg
