// pack2_host.h -- host part of the 2D warp lists (setup.cu): the blocks of
// one colour (blocks.h) packed, whole and largest first, into sequences of
// 32*W*K slots with their node descriptors and one junction record per
// sequence, the layout warp_line.cu reads.  Plain C++, so that the layout is
// also checked on the CPU.
#pragma once
#include <algorithm>
#include <cstring>
#include <numeric>
#include <tuple>
#include <vector>

#include "blocks.h"

namespace tmg {

inline int pk_step_i(int d) { return d == DIR_PX ? 1 : (d == DIR_MX ? -1 : 0); }
inline int pk_step_j(int d) { return d == DIR_PY ? 1 : (d == DIR_MY ? -1 : 0); }

struct Pack2 {
  std::vector<WNode> nodes;  // nwarp * 32 * W * K slots
  std::vector<WBlock> blk;   // one per sequence
  int nwarp = 0, K = 0, W = 1, total_nodes = 0;
};

// false: the blocks do not fit the warp path (the list stays empty)
inline bool pack2(const std::vector<HBlock> &blocks, int kmax, int kpref, Pack2 &out) {
  out = Pack2();
  std::vector<int> n(blocks.size(), 0);
  int maxn = 1, total = 0;
  for (size_t b = 0; b < blocks.size(); ++b) {
    for (const HChain &c : blocks[b].ch)
      for (const HSeg &sg : c.s) n[b] += sg.len;
    maxn = std::max(maxn, n[b]);
    total += n[b] + (blocks[b].junc ? 1 : 0);
  }
  if (blocks.empty() || maxn > 32 * WW_MAX * kmax) return false;
  int K = 1, NW = 1;
  while (32 * K < maxn && K < std::min(kpref, kmax)) K *= 2;
  while (32 * NW * K < maxn) NW *= 2;
  while (NW > WW_MAX) {
    K *= 2;
    NW = 1;
    while (32 * NW * K < maxn) NW *= 2;
  }
  const int cap = 32 * NW * K;
  std::vector<int> order(blocks.size());
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] > n[b]; });
  struct Bin {
    int used = 0;
    bool junc = false;
    std::vector<int> blocks;
  };
  std::vector<Bin> bins;
  for (int b : order) {
    size_t w = 0;
    while (w < bins.size() && (bins[w].used + n[b] > cap || (blocks[b].junc && bins[w].junc))) ++w;
    if (w == bins.size()) bins.emplace_back();
    bins[w].used += n[b];
    bins[w].junc |= blocks[b].junc;
    bins[w].blocks.push_back(b);
  }
  std::vector<WNode> &nodes = out.nodes;
  std::vector<WBlock> &blk = out.blk;
  nodes.assign(bins.size() * (size_t)cap, WNode{});
  blk.assign(bins.size(), WBlock{});
  std::memset(nodes.data(), 0, sizeof(WNode) * nodes.size());
  std::memset(blk.data(), 0, sizeof(WBlock) * blk.size());
  for (size_t w = 0; w < bins.size(); ++w) {
    WBlock &jb = blk[w];
    int s = 0;
    for (int b : bins[w].blocks) {
      const HBlock &hb = blocks[b];
      if (hb.junc) {
        jb.has_j = 1;
        jb.ji = (uint16_t)hb.ji;
        jb.jj = (uint16_t)hb.jj;
      }
      for (const HChain &c : hb.ch) {
        // the chain's nodes in order, with the direction of the step that
        // reaches each node (its segment's direction)
        std::vector<std::tuple<int, int, int>> cn;
        for (const HSeg &sg : c.s)
          for (int t = 0; t < sg.len; ++t) cn.emplace_back(sg.i0 + t * pk_step_i(sg.dir), sg.j0 + t * pk_step_j(sg.dir), sg.dir);
        const int m = (int)cn.size();
        for (int r = 0; r < m; ++r) {
          uint32_t fl = WN_VALID;
          if (r > 0) fl |= WN_PRED | (uint32_t)(std::get<2>(cn[r]) ^ 1);
          if (r < m - 1) fl |= WN_SUCC | ((uint32_t)std::get<2>(cn[r + 1]) << 3);
          int jd = -1;
          if (r == 0 && c.fj) jd = std::get<2>(cn[0]) ^ 1;
          if (r == m - 1 && c.lj) {
            if (jd >= 0) return false;  // a one-node chain on both sides of the junction: not supported here
            jd = c.ljdir;
          }
          if (jd >= 0) {
            if (!hb.junc || jb.natt >= 4) return false;
            fl |= WN_JUNC | ((uint32_t)jd << 6);
            jb.as[jb.natt] = (uint16_t)s;
            jb.adirs |= (uint8_t)((jd ^ 1) << (2 * jb.natt));
            ++jb.natt;
          }
          WNode &nd = nodes[w * (size_t)cap + s];
          nd.i = (uint16_t)std::get<0>(cn[r]);
          nd.j = (uint16_t)std::get<1>(cn[r]);
          nd.fl = fl;
          ++s;
        }
      }
    }
  }
  out.nwarp = (int)bins.size();
  out.K = K;
  out.W = NW;
  out.total_nodes = total;
  return true;
}

}  // namespace tmg
