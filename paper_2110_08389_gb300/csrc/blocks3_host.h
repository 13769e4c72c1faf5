// blocks3_host.h -- host part of the 3D block builder (grid3d.cu): the
// tweed and wireframe blocks of one level (Sec. 7) as chains, junctions and
// cuboid edge skeletons.  Plain C++ over Level3's sizes, so that it is also
// checked on the CPU against the oracle's partition.
#pragma once
#include <algorithm>
#include <cstddef>
#include <numeric>
#include <utility>
#include <vector>

#include "mg_internal.h"

namespace tmg {

inline int dir_between(int nx1, size_t plane, long long p, long long q) {
  const long long d = q - p;
  if (d == 1) return 0;
  if (d == -1) return 1;
  if (d == nx1) return 2;
  if (d == -(long long)nx1) return 3;
  if (d == (long long)plane) return 4;
  return 5;
}

// The blocks of one level for one smoother (tweed: level sets of (d2, d3) of
// the sorted wall distances; wireframe: of (d1, d2)), as chains of node
// offsets in order.  A chain may end next to the block's junction (a tweed
// star's centre, or the node chosen to close a wireframe ring); a wireframe
// edge skeleton is kept as its corners and edges.  False if a block is none
// of: a line, a star, a ring, a cuboid's edge skeleton (a side with an odd
// number of intervals closes other loops).
struct HSkelEdge {
  int a = 0, b = 0, dir = 0;
  std::vector<long long> nodes;  // interior nodes in order from corner a
};
struct HBlock3 {
  std::vector<std::vector<long long>> chains;
  std::vector<int> jfirst, jlast;  // per chain: direction from its first / last node to the junction, or -1
  long long junc = -1;
  bool skel = false;
  long long corner[8] = {};
  std::vector<HSkelEdge> edges;
  int colour = 0;
  int nodes = 0;  // chain nodes (the junction and the skeleton not counted)
};

inline bool blocks3(const Level3 &L, int sm, std::vector<HBlock3> &out) {
  const int nx = L.nx, ny = L.ny, nz = L.nz, nx1 = nx + 1;
  const size_t plane = (size_t)nx1 * (ny + 1), nn = L.nn;
  auto ijk = [&](size_t p, int &i, int &j, int &k) { i = (int)(p % nx1); j = (int)((p / nx1) % (ny + 1)); k = (int)(p / plane); };
  auto inside = [&](int i, int j, int k) { return i > 0 && i < nx && j > 0 && j < ny && k > 0 && k < nz; };
  auto key = [&](int i, int j, int k) {
    int a = std::min(i, nx - i), b = std::min(j, ny - j), c = std::min(k, nz - k);
    if (a > b) std::swap(a, b);
    if (b > c) std::swap(b, c);
    if (a > b) std::swap(a, b);
    return sm == SM3_WIREFRAME ? std::make_pair(a, b) : std::make_pair(b, c);
  };
  std::vector<int> par(nn);
  std::iota(par.begin(), par.end(), 0);
  auto fnd = [&](int x) {
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
  };
  const long long step[6] = {1, -1, nx1, -(long long)nx1, (long long)plane, -(long long)plane};
  const int di[6] = {1, -1, 0, 0, 0, 0}, dj[6] = {0, 0, 1, -1, 0, 0}, dk[6] = {0, 0, 0, 0, 1, -1};
  for (int k = 1; k < nz; ++k)
    for (int j = 1; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        const auto kp = key(i, j, k);
        const size_t p = (size_t)k * plane + (size_t)j * nx1 + i;
        for (int d = 0; d < 6; d += 2) {
          const int ii = i + di[d], jj = j + dj[d], kk = k + dk[d];
          if (!inside(ii, jj, kk) || key(ii, jj, kk) != kp) continue;
          const int r1 = fnd((int)p), r2 = fnd((int)(p + step[d]));
          if (r1 != r2) par[r1] = r2;
        }
      }
  // block of every node (-1 off the interior): an interior node's six
  // neighbours are all inside the array, so in-block tests need no bounds
  std::vector<int> id(nn, -1), own(nn, -1);
  std::vector<std::vector<long long>> members;
  for (int k = 1; k < nz; ++k)
    for (int j = 1; j < ny; ++j)
      for (int i = 1; i < nx; ++i) {
        const size_t p = (size_t)k * plane + (size_t)j * nx1 + i;
        const int r = fnd((int)p);
        if (id[r] < 0) { id[r] = (int)members.size(); members.emplace_back(); }
        own[p] = id[r];
        members[id[r]].push_back((long long)p);
      }
  std::vector<int>().swap(par);
  std::vector<int>().swap(id);
  std::vector<long long> nb, wv;
  for (size_t b = 0; b < members.size(); ++b) {
    const auto &mb = members[b];
    HBlock3 hb;
    hb.nodes = (int)mb.size();
    int i, j, k;
    ijk((size_t)mb[0], i, j, k);
    const auto kk0 = key(i, j, k);
    hb.colour = ((kk0.first + kk0.second) % 2 == 0) ? 0 : 1;
    // in-block neighbours
    auto nbrs = [&](long long p, std::vector<long long> &v) {
      v.clear();
      for (int d = 0; d < 6; ++d)
        if (own[p + step[d]] == (int)b) v.push_back(p + step[d]);
    };
    std::vector<long long> branch;
    int edges2 = 0, maxdeg = 0;
    long long endpoint = mb[0];
    for (long long p : mb) {
      nbrs(p, nb);
      edges2 += (int)nb.size();
      maxdeg = std::max(maxdeg, (int)nb.size());
      if (nb.size() >= 3) branch.push_back(p);
      if (nb.size() <= 1) endpoint = p;
    }
    const int edges = edges2 / 2;
    // follows the chain from cur (coming from prev) until a tip, a node with
    // three or more in-block neighbours (kept as the chain's last entry) or
    // the node `stop` (not kept); returns the node it stopped on
    auto walk = [&](long long prev, long long cur, long long stop, std::vector<long long> &chain) {
      std::vector<long long> &v = wv;
      while (true) {
        chain.push_back(cur);
        nbrs(cur, v);
        if (v.size() > 2) return cur;
        long long next = -1;
        for (long long q : v)
          if (q != prev) next = q;
        if (next < 0) return cur;
        if (next == stop) return next;
        prev = cur;
        cur = next;
      }
    };
    if (edges == hb.nodes - 1 && branch.size() <= 1) {
      if (!branch.empty()) {  // a star: legs tip .. node next to the centre
        const long long c0 = branch[0];
        hb.junc = c0;
        std::vector<long long> legs;
        nbrs(c0, legs);
        for (long long q : legs) {
          std::vector<long long> leg;
          walk(c0, q, -1, leg);
          std::reverse(leg.begin(), leg.end());
          hb.jfirst.push_back(-1);
          hb.jlast.push_back(dir_between(nx1, plane, q, c0));
          hb.chains.push_back(std::move(leg));
        }
        hb.nodes -= 1;
      } else {  // a line (or a point)
        std::vector<long long> line;
        walk(-1, endpoint, -1, line);
        hb.chains.push_back(std::move(line));
        hb.jfirst.push_back(-1);
        hb.jlast.push_back(-1);
      }
    } else if (edges == hb.nodes && maxdeg == 2 && hb.nodes >= 4) {  // a ring, closed by its first node
      const long long c0 = mb[0];
      std::vector<long long> two, ring;
      nbrs(c0, two);
      walk(c0, two[0], c0, ring);
      if ((int)ring.size() != hb.nodes - 1 || ring.back() != two[1]) return false;
      hb.junc = c0;
      hb.jfirst.push_back(dir_between(nx1, plane, ring.front(), c0));
      hb.jlast.push_back(dir_between(nx1, plane, ring.back(), c0));
      hb.chains.push_back(std::move(ring));
      hb.nodes -= 1;
    } else if (sm == SM3_WIREFRAME && branch.size() == 8 && edges == hb.nodes + 4 && maxdeg == 3) {
      // a cuboid's edge skeleton: eight corners, twelve edges between them
      hb.skel = true;
      for (int c = 0; c < 8; ++c) hb.corner[c] = branch[c];
      auto corner_of = [&](long long p) {
        for (int c = 0; c < 8; ++c)
          if (hb.corner[c] == p) return c;
        return -1;
      };
      for (int c = 0; c < 8; ++c) {
        std::vector<long long> v;
        nbrs(hb.corner[c], v);
        for (long long q : v) {
          if (corner_of(q) >= 0) return false;  // adjacent corners: no edge nodes
          HSkelEdge e;
          const long long end = walk(hb.corner[c], q, -1, e.nodes);
          e.nodes.pop_back();  // the walk stops on the far corner
          const int cb = corner_of(end);
          if (cb < 0 || e.nodes.empty()) return false;
          if (cb < c) continue;  // each edge once, from its lower corner
          e.a = c;
          e.b = cb;
          e.dir = dir_between(nx1, plane, hb.corner[c], q);
          // a straight edge: node s at the corner plus s + 1 steps (the
          // skeleton kernel recomputes the positions this way)
          const long long st = step[e.dir];
          for (size_t r = 0; r < e.nodes.size(); ++r)
            if (e.nodes[r] != hb.corner[c] + (long long)(r + 1) * st) return false;
          if (end != hb.corner[c] + (long long)(e.nodes.size() + 1) * st) return false;
          hb.edges.push_back(std::move(e));
        }
      }
      if (hb.edges.size() != 12) return false;
      int sum = 8;
      for (const auto &e : hb.edges) sum += (int)e.nodes.size();
      if (sum != (int)mb.size()) return false;
      hb.nodes = 0;
    } else {
      return false;
    }
    out.push_back(std::move(hb));
  }
  return true;
}

}  // namespace tmg
