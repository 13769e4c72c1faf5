// setup.cu -- host-side construction of tweedmg's block work lists.
//
// The blocks of every smoother are enumerated in closed form from the node's
// distances to the walls, d_x = min(i, nx-i) and d_y = min(j, ny-j):
//   tweed (Sec. 3, Figs. 4 and 6): level k = max(d_x, d_y).  For k below
//     min(nx,ny)/2 the level splits into four L-shaped blocks, one per corner
//     (a leg perpendicular to each wall meeting at (k,k)); k = 1 gives the
//     four corner points.  At k = nx/2 = ny/2 the four legs meet in the centre
//     cross (m = 4); on a rectangle the level k = min/2 gives two T-blocks
//     (m = 3) and the larger levels give straight lines perpendicular to the
//     nearest walls.
//   wireframe (Sec. 3, Figs. 5 and 7): level k = min(d_x, d_y): concentric
//     rings, then the centre point (square) or centre line (rectangle).
//   zebra: rows (x) or columns (y).
// Colour: odd k (or odd line index) is red = colour 0, relaxed first.
//
// Each block becomes chains of straight segments, the segments are cut into
// chunks of at most CMAX nodes, and whole blocks are packed into CTAs of at
// most NT_SMALL chunks (or NT_LARGE for the few blocks that need more).
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <tuple>

#include "mg_internal.h"
#include "blocks.h"
#include "pack2_host.h"

namespace tmg {

namespace {

inline int nchunks_of(int len) { return (len + CMAX - 1) / CMAX; }

struct Packed {
  std::vector<CtaWork> cta;
  std::vector<ChunkDesc> chunk;
  std::vector<JuncDesc> junc;
  std::vector<VGroup> vg;
  int total = 0;
};

// Group the CTA's vertical chunks that share rows and direction and sit in
// same-colour columns two apart, four at a time.
void group_vertical(Packed &P, CtaWork &w) {
  std::vector<int> ids;
  for (int t = 0; t < w.nchunk; ++t) {
    const ChunkDesc &cd = P.chunk[w.chunk0 + t];
    if ((cd.flags & 3) >= 2) ids.push_back(t);
  }
  auto key = [&](int t) {
    const ChunkDesc &cd = P.chunk[w.chunk0 + t];
    return std::make_tuple((int)cd.j0, (int)cd.len, cd.flags & 3, (int)cd.i0);
  };
  std::sort(ids.begin(), ids.end(), [&](int a, int b) { return key(a) < key(b); });
  w.vg0 = (int)P.vg.size();
  size_t k = 0;
  while (k < ids.size()) {
    size_t e = k + 1;
    while (e < ids.size() && e - k < 4) {
      const ChunkDesc &a = P.chunk[w.chunk0 + ids[e - 1]], &b = P.chunk[w.chunk0 + ids[e]];
      if (b.j0 != a.j0 || b.len != a.len || (b.flags & 3) != (a.flags & 3) || b.i0 != a.i0 + 2) break;
      ++e;
    }
    if (e - k >= 2) {
      VGroup g;
      for (int q = 0; q < 4; ++q) g.c[q] = 0xFFFF;
      for (size_t q = k; q < e; ++q) {
        g.c[q - k] = (uint16_t)ids[q];
        P.chunk[w.chunk0 + ids[q]].info |= GROUPED;
      }
      P.vg.push_back(g);
    }
    k = e;
  }
  w.nvg = (int)P.vg.size() - w.vg0;
}

inline int step_i(int d) { return d == DIR_PX ? 1 : (d == DIR_MX ? -1 : 0); }
inline int step_j(int d) { return d == DIR_PY ? 1 : (d == DIR_MY ? -1 : 0); }

// Append one block to the open CTA (the caller checked the capacity).  Each
// segment is cut into chunks of exactly CMAX nodes plus a ragged last one.
void emit_block(Packed &P, CtaWork &w, const HBlock &b) {
  int jidx = -1;
  if (b.junc) {
    JuncDesc jd;
    std::memset(&jd, 0, sizeof(jd));
    jd.i = (uint16_t)b.ji; jd.j = (uint16_t)b.jj;
    jidx = w.njunc++;
    P.junc.push_back(jd);
  }
  JuncDesc *jd = b.junc ? &P.junc.back() : nullptr;
  for (const HChain &c : b.ch) {
    const int ns = (int)c.s.size();
    for (int q = 0; q < ns; ++q) {
      const HSeg &s = c.s[q];
      const int nextdir = q < ns - 1 ? c.s[q + 1].dir : (c.lj ? c.ljdir : s.dir);
      const bool seg_lp = q > 0, seg_ln = q < ns - 1, seg_fj = q == 0 && c.fj, seg_lj = q == ns - 1 && c.lj;
      const int nch = nchunks_of(s.len);
      for (int t = 0; t < nch; ++t) {
        const int off = t * CMAX, len = std::min(CMAX, s.len - off);
        const bool first = t == 0, last = t == nch - 1;
        uint8_t fl = (uint8_t)(s.dir | ((last ? nextdir : s.dir) << 2));
        if (!first || seg_lp) fl |= F_LP;
        if (!last || seg_ln) fl |= F_LN;
        if (first && seg_fj) fl |= F_FJ;
        if (last && seg_lj) fl |= F_LJ;
        ChunkDesc cd;
        std::memset(&cd, 0, sizeof(cd));
        cd.i0 = (uint16_t)(s.i0 + off * step_i(s.dir));
        cd.j0 = (uint16_t)(s.j0 + off * step_j(s.dir));
        cd.len = (uint8_t)len;
        cd.flags = fl;
        cd.info = jidx >= 0 ? (uint16_t)jidx : JNONE;
        const int tloc = w.nchunk;  // CTA-local chunk index
        if (jd && (fl & F_FJ)) {
          jd->row[jd->nend] = (uint16_t)(2 * tloc);
          jd->dirs |= (uint8_t)(s.dir << (2 * jd->nend));
          ++jd->nend;
        }
        if (jd && (fl & F_LJ)) {
          jd->row[jd->nend] = (uint16_t)(len >= 2 ? 2 * tloc + 1 : 2 * tloc);
          jd->dirs |= (uint8_t)((c.ljdir ^ 1) << (2 * jd->nend));
          ++jd->nend;
        }
        P.chunk.push_back(cd);
        ++w.nchunk;
      }
      w.nnode += s.len;
    }
  }
}

// Pack whole blocks into CTAs of at most nt chunks (largest first, next fit).
void pack(const std::vector<HBlock> &blocks, const std::vector<int> &order, int nt, Packed &P) {
  CtaWork w;
  std::memset(&w, 0, sizeof(w));
  auto flush = [&]() {
    if (w.nchunk == 0 && w.njunc == 0) return;
    group_vertical(P, w);
    P.cta.push_back(w);
    CtaWork z;
    std::memset(&z, 0, sizeof(z));
    z.chunk0 = (int)P.chunk.size(); z.junc0 = (int)P.junc.size();
    w = z;
  };
  for (int bi : order) {
    const HBlock &b = blocks[bi];
    if (w.nchunk + b.chunks > nt || w.njunc + (b.junc ? 1 : 0) > nt) flush();
    emit_block(P, w, b);
    P.total += b.nodes + (b.junc ? 1 : 0);
  }
  flush();
}

template <typename X>
size_t align16(size_t n) { return (n * sizeof(X) + 15) & ~size_t(15); }

mg_status upload(const Packed &P, int nt, WorkList &W) {
  W.ncta = (int)P.cta.size();
  W.nt = nt;
  W.total_nodes = P.total;
  if (W.ncta == 0) return MG_OK;
  const size_t b0 = align16<CtaWork>(P.cta.size()), b1 = align16<ChunkDesc>(std::max<size_t>(P.chunk.size(), 1)),
               b2 = align16<JuncDesc>(std::max<size_t>(P.junc.size(), 1)),
               b3 = align16<VGroup>(std::max<size_t>(P.vg.size(), 1));
  char *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, b0 + b1 + b2 + b3);
  if (e != cudaSuccess) { set_error("cudaMalloc(work list)", e); return MG_ERR_ALLOC; }
  W.mem = mem;
  W.cta = reinterpret_cast<CtaWork *>(mem);
  W.chunk = reinterpret_cast<ChunkDesc *>(mem + b0);
  W.junc = reinterpret_cast<JuncDesc *>(mem + b0 + b1);
  W.vg = reinterpret_cast<VGroup *>(mem + b0 + b1 + b2);
  e = cudaMemcpy(W.cta, P.cta.data(), sizeof(CtaWork) * P.cta.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !P.chunk.empty())
    e = cudaMemcpy(W.chunk, P.chunk.data(), sizeof(ChunkDesc) * P.chunk.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !P.junc.empty())
    e = cudaMemcpy(W.junc, P.junc.data(), sizeof(JuncDesc) * P.junc.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !P.vg.empty())
    e = cudaMemcpy(W.vg, P.vg.data(), sizeof(VGroup) * P.vg.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { set_error("cudaMemcpy(work list)", e); return MG_ERR_CUDA; }
  return MG_OK;
}

// Warp path: lay the colour's blocks end to end in sequences of 32*W*K
// nodes (first fit, largest blocks first; at most one junction per sequence),
// K and W powers of two chosen as described with WK_PREF (kpref in its
// place).  Leaves W.nwarp = 0 when the largest block does not fit WW_MAX
// warps of kmax nodes per lane.
mg_status build_warplist(const std::vector<HBlock> &blocks, int kmax, int kpref, WarpList &W) {
  Pack2 pk;
  if (!pack2(blocks, kmax, kpref, pk)) return MG_OK;
  const std::vector<WNode> &nodes = pk.nodes;
  const std::vector<WBlock> &blk = pk.blk;
  const size_t bn = (sizeof(WNode) * nodes.size() + 15) & ~size_t(15);
  char *mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, bn + sizeof(WBlock) * blk.size());
  if (e != cudaSuccess) { set_error("cudaMalloc(warp list)", e); return MG_ERR_ALLOC; }
  W.mem = mem;
  W.node = reinterpret_cast<WNode *>(mem);
  W.blk = reinterpret_cast<WBlock *>(mem + bn);
  e = cudaMemcpy(W.node, nodes.data(), sizeof(WNode) * nodes.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(W.blk, blk.data(), sizeof(WBlock) * blk.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { set_error("cudaMemcpy(warp list)", e); return MG_ERR_CUDA; }
  W.nwarp = pk.nwarp;
  W.K = pk.K;
  W.W = pk.W;
  W.total_nodes = pk.total_nodes;
  return MG_OK;
}

}  // namespace

static void blocks_of(const Level &L, int wl, int colour, std::vector<HBlock> &blocks) {
  switch (wl) {
    case WL_TWEED: tweed_blocks(L.nx, L.ny, colour, blocks); break;
    case WL_WIREFRAME: wireframe_blocks(L.nx, L.ny, colour, blocks); break;
    case WL_ZEBRA_X: zebra_blocks(L.nx, L.ny, colour, true, blocks); break;
    default: zebra_blocks(L.nx, L.ny, colour, false, blocks); break;
  }
}

void free_warplist(WarpList &w) {
  cudaFree(w.mem);
  w = WarpList();
}

mg_status build_warp_path(Grid &g, int level, int wl, int prec, int kpref, WarpList out[2]) {
  const Level &L = g.lev[level];
  for (int colour = 0; colour < 2; ++colour) {
    std::vector<HBlock> blocks;
    blocks_of(L, wl, colour, blocks);
    const mg_status st = build_warplist(blocks, prec == 0 ? WK_MAX_F64 : WK_MAX_F32, kpref > 0 ? kpref : WK_PREF,
                                        out[colour]);
    if (st != MG_OK) return st;
  }
  return MG_OK;
}

mg_status build_worklists(Grid &g, int level, int wl, int prec) {
  Level &L = g.lev[level];
  if (L.wl_built[wl][prec]) return MG_OK;
  for (int colour = 0; colour < 2; ++colour) {
    std::vector<HBlock> blocks;
    blocks_of(L, wl, colour, blocks);
    // blocks of more than a quarter of a small CTA go to large CTAs, so that
    // every CTA holds about four neighbouring blocks; neighbours (same group,
    // consecutive positions) are packed together for the vertical groups
    std::vector<int> small, large;
    for (size_t bi = 0; bi < blocks.size(); ++bi) {
      HBlock &b = blocks[bi];
      b.nodes = 0;  // chain nodes (the junction is not kept in shared memory)
      b.chunks = 0;
      for (auto &c : b.ch)
        for (auto &s : c.s) { b.nodes += s.len; b.chunks += nchunks_of(s.len); }
      if (b.chunks > NT_LARGE) return MG_ERR_SIZE;
      (b.chunks > NT_SMALL / 4 ? large : small).push_back((int)bi);
    }
    auto by_key = [&](int a, int b) {
      return std::make_pair(blocks[a].group, blocks[a].pos) < std::make_pair(blocks[b].group, blocks[b].pos);
    };
    std::stable_sort(small.begin(), small.end(), by_key);
    std::stable_sort(large.begin(), large.end(), by_key);
    // small levels: fewer chunks per CTA, so that the level spreads over about
    // four CTAs per SM (the passes there are latency-bound: each thread of a
    // full CTA would walk hundreds of nodes one after the other)
    int small_chunks = 0, widest = 1;
    for (int bi : small) { small_chunks += blocks[bi].chunks; widest = std::max(widest, blocks[bi].chunks); }
    const int target = 4 * std::max(g.sms, 1);
    const int cap = std::min(NT_SMALL, std::max(widest, (small_chunks + target - 1) / target));
    Packed Ps, Pl;
    pack(blocks, small, cap, Ps);
    pack(blocks, large, NT_LARGE, Pl);
    mg_status st = upload(Ps, NT_SMALL, L.wl[wl][prec][colour][0]);
    if (st == MG_OK) st = upload(Pl, NT_LARGE, L.wl[wl][prec][colour][1]);
    if (st == MG_OK && L.nx < WARP_MAX_SIDE && L.ny < WARP_MAX_SIDE)
      st = build_warplist(blocks, prec == 0 ? WK_MAX_F64 : WK_MAX_F32, WK_PREF, L.wp[wl][prec][colour]);
    if (st != MG_OK) return st;
  }
  L.wl_built[wl][prec] = true;
  return MG_OK;
}

}  // namespace tmg
