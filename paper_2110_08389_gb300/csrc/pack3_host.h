// pack3_host.h -- host part of the 3D warp lists (grid3d.cu): the blocks of
// one colour (blocks3_host.h) packed into sequences of 32*W*K slots with
// their node descriptors, junction records and skeleton descriptors, the
// layout the kernels of seq3.cuh read.  Plain C++, so that the layout is
// also checked on the CPU.
#pragma once
#include <algorithm>
#include <cstring>
#include <functional>
#include <vector>

#include "blocks3_host.h"

namespace tmg {

// at most 8 nodes per thread, 8 warps per sequence; 4 nodes per thread preferred
constexpr int WARP3_KMAX = 8, WARP3_WMAX = 8, WARP3_KPREF = 4;

struct Pack3 {
  std::vector<WNode3> nodes;  // nwarp * 32 * W * K slots
  std::vector<WJunc3> jn;
  std::vector<int> jofs;      // nwarp + 1
  std::vector<WSkel3> skel;
  int nwarp = 0, K = 0, W = 1, total_nodes = 0, skel_nodes = 0;
  bool multi = false;
};

// Sequences of one colour (first fit, largest blocks first), K and W as in
// 2D (warp_line.cu) with at most 8 nodes per thread (both precisions use the
// same lists), and the colour's edge skeletons.  multi: up to WJ3_MAX
// junctions per sequence (wireframe rings), listed per sequence through
// jofs; otherwise at most one, the sequence's own junction record.
inline mg_status pack3(const Level3 &L, const std::vector<HBlock3> &all, int colour, bool multi, Pack3 &out) {
  const int jmax = multi ? WJ3_MAX : 1;
  std::vector<int> idx, sk;
  int maxn = 1, total = 0, skn = 0;
  for (size_t b = 0; b < all.size(); ++b) {
    if (all[b].colour != colour) continue;
    if (all[b].skel) {
      sk.push_back((int)b);
      for (const auto &e : all[b].edges) skn += (int)e.nodes.size();
      continue;
    }
    idx.push_back((int)b);
    maxn = std::max(maxn, all[b].nodes);
    total += all[b].nodes + (all[b].junc >= 0 ? 1 : 0);
  }
  out = Pack3();
  if (idx.empty() && sk.empty()) return MG_OK;
  if (maxn > 32 * WARP3_WMAX * WARP3_KMAX) return MG_ERR_SIZE;
  int K = 1, NW = 1;
  while (32 * K < maxn && K < WARP3_KPREF) K *= 2;
  while (32 * NW * K < maxn) NW *= 2;
  while (NW > WARP3_WMAX) {
    K *= 2;
    NW = 1;
    while (32 * NW * K < maxn) NW *= 2;
  }
  const int cap = 32 * NW * K;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return all[a].nodes > all[b].nodes; });
  struct Bin { int used = 0, nj = 0; std::vector<int> blocks; };
  std::vector<Bin> bins;
  // first fit: a max-tree over the free slots of every possible bin finds
  // the leftmost bin with room (log time per block)
  int P2 = 1;
  while (P2 < (int)idx.size()) P2 *= 2;
  std::vector<int> fr(2 * (size_t)P2, cap);
  auto first_fit = [&](int lo, int n) {  // leftmost bin >= lo with >= n free slots, or -1
    std::function<int(int, int, int)> go = [&](int v, int l, int r) -> int {
      if (r <= lo || fr[v] < n) return -1;
      if (r - l == 1) return l;
      const int m = (l + r) / 2, a = go(2 * v, l, m);
      return a >= 0 ? a : go(2 * v + 1, m, r);
    };
    return go(1, 0, P2);
  };
  for (int b : idx) {
    const int nj = all[b].junc >= 0 ? 1 : 0, n = all[b].nodes;
    int w = first_fit(0, n);
    while (w >= 0 && w < (int)bins.size() && bins[w].nj + nj > jmax) w = first_fit(w + 1, n);
    if (w < 0) return MG_ERR_SIZE;  // cannot happen: every block fits an empty bin
    while ((int)bins.size() <= w) bins.emplace_back();
    bins[w].used += n;
    bins[w].nj += nj;
    bins[w].blocks.push_back(b);
    int v = P2 + w;
    fr[v] = cap - bins[w].used;
    for (v >>= 1; v >= 1; v >>= 1) fr[v] = std::max(fr[2 * v], fr[2 * v + 1]);
  }
  const int nx1 = L.nx + 1;
  const size_t plane = (size_t)nx1 * (L.ny + 1);
  std::vector<WNode3> &nodes = out.nodes;
  std::vector<WJunc3> &jn = out.jn;
  std::vector<int> &jofs = out.jofs;
  std::vector<WSkel3> &skel = out.skel;
  nodes.assign(bins.size() * (size_t)cap, WNode3{});
  jofs.assign(bins.size() + 1, 0);
  skel.assign(sk.size(), WSkel3{});
  std::memset(nodes.data(), 0, sizeof(WNode3) * nodes.size());
  std::memset(skel.data(), 0, sizeof(WSkel3) * skel.size());
  auto pack = [&](long long p) {
    const uint32_t i = (uint32_t)(p % nx1), j = (uint32_t)((p / nx1) % (L.ny + 1)), k = (uint32_t)(p / plane);
    return i | (j << 10) | (k << 20);
  };
  for (size_t w = 0; w < bins.size(); ++w) {
    jofs[w] = (int)jn.size();
    if (!multi) {  // one record per sequence, natt = 0 without a junction
      jn.emplace_back();
      std::memset(&jn.back(), 0, sizeof(WJunc3));
    }
    int s = 0;
    for (int b : bins[w].blocks) {
      const HBlock3 &hb = all[b];
      const uint32_t jl = multi ? (uint32_t)(jn.size() - jofs[w]) : 0u;
      WJunc3 *jb = nullptr;
      if (hb.junc >= 0) {
        if (multi) {
          jn.emplace_back();
          std::memset(&jn.back(), 0, sizeof(WJunc3));
        }
        jb = &jn.back();
        jb->ijk = pack(hb.junc);
      }
      for (size_t c = 0; c < hb.chains.size(); ++c) {
        const auto &ch = hb.chains[c];
        const int m = (int)ch.size();
        for (int r = 0; r < m; ++r) {
          uint32_t fl = WN3_VALID | (jb ? jl << WN3_JSHIFT : 0u);
          if (r > 0) fl |= WN3_PRED | (uint32_t)dir_between(nx1, plane, ch[r], ch[r - 1]);
          if (r < m - 1) fl |= WN3_SUCC | ((uint32_t)dir_between(nx1, plane, ch[r], ch[r + 1]) << 4);
          const int dj = r == m - 1 && hb.jlast[c] >= 0 ? hb.jlast[c] : (r == 0 ? hb.jfirst[c] : -1);
          if (jb && dj >= 0) {
            fl |= WN3_JUNC | ((uint32_t)dj << 8);
            jb->as[jb->natt] = (uint16_t)s;
            jb->adirs |= (uint32_t)(dj ^ 1) << (3 * jb->natt);
            ++jb->natt;
          }
          WNode3 &nd = nodes[w * (size_t)cap + s];
          nd.ijk = pack(ch[r]);
          nd.fl = fl;
          ++s;
        }
      }
    }
  }
  jofs[bins.size()] = (int)jn.size();
  int off = 0;
  for (size_t q = 0; q < sk.size(); ++q) {
    const HBlock3 &hb = all[sk[q]];
    WSkel3 &S = skel[q];
    for (int c = 0; c < 8; ++c) S.cijk[c] = pack(hb.corner[c]);
    for (int e = 0; e < 12; ++e) {
      S.eoff[e] = (uint32_t)off;
      S.ea[e] = (uint8_t)hb.edges[e].a;
      S.eb[e] = (uint8_t)hb.edges[e].b;
      S.ed[e] = (uint8_t)hb.edges[e].dir;
      off += (int)hb.edges[e].nodes.size();
    }
    S.eoff[12] = (uint32_t)off;
  }
  out.nwarp = (int)bins.size();
  out.K = K;
  out.W = NW;
  out.total_nodes = total;
  out.skel_nodes = skn;
  out.multi = multi;
  return MG_OK;
}

}  // namespace tmg
