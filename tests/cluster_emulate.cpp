// Runs one colour pass of the cluster path on the CPU, in FP64, exactly as
// the CTAs of the kernel divide the work: the plan of csrc/cluster_host.h and
// the chunk eliminations of csrc/cluster_math.h, with each CTA's shared
// memory an array of its own; the leg solve of a block runs in the CTA the
// kernel gives it (b mod the group's CTAs) and reads and writes the rows and
// end values in the arrays of the CTAs that hold the chunks, by cluster rank.
//
// stdin:  nx ny wl colour tiles_per_cta ctas_per_cluster, then W E (nx+1
//         each), S N (ny+1 each), u and f ((ny+1) x (nx+1), x fastest).
// stdout: "plan ncta ntile nseg ngroup total" and the relaxed u, or "noplan".
// Exit code 3 if a chunk's end values are written by no leg solve or twice.
#include <cmath>
#include <cstdio>
#include <vector>

#include "cluster_host.h"
#include "cluster_math.h"

using namespace tmg;
using clmath::Row;
typedef double T;

struct Level2 {
  int nx, ny;
  std::vector<T> W, E, S, N, u, f;
  T &U(int i, int j) { return u[(size_t)j * (nx + 1) + i]; }
  T F(int i, int j) const { return f[(size_t)j * (nx + 1) + i]; }
};

struct Geo {
  bool xrun;
  int step;
};
static Geo geo(int dir) { return Geo{dir < 2, (dir == DIR_PX || dir == DIR_PY) ? 1 : -1}; }

// coefficients of slot q of a run through (v(q), line)
struct Co {
  const Level2 *L;
  Geo g;
  int base, line;
  T lo(int q) const {
    const int v = base + q * g.step;
    return g.xrun ? (g.step > 0 ? L->W[v] : L->E[v]) : (g.step > 0 ? L->S[v] : L->N[v]);
  }
  T hi(int q) const {
    const int v = base + q * g.step;
    return g.xrun ? (g.step > 0 ? L->E[v] : L->W[v]) : (g.step > 0 ? L->N[v] : L->S[v]);
  }
};
struct Arr {
  const T *p;
  T operator()(int q) const { return p[q]; }
};
struct XArr {
  T *p;
  T get(int q) const { return p[q]; }
  void set(int q, T v) { p[q] = v; }
};

struct CtaMem {
  std::vector<T> D;                 // [slot][32]
  std::vector<Row<T>> rows;         // [slot][2]
  std::vector<int> mlen;            // [slot]
  std::vector<T> chx;               // [slot][2]
  std::vector<int> written;         // [slot][2]: times each end value was written
};

int main() {
  int nx, ny, wl, colour, S, CL;
  if (std::scanf("%d %d %d %d %d %d", &nx, &ny, &wl, &colour, &S, &CL) != 6) return 2;
  Level2 L;
  L.nx = nx; L.ny = ny;
  auto rd = [](std::vector<T> &v, size_t n) {
    v.resize(n);
    for (size_t k = 0; k < n; ++k)
      if (std::scanf("%lf", &v[k]) != 1) return false;
    return true;
  };
  const size_t nn = (size_t)(nx + 1) * (ny + 1);
  if (!rd(L.W, nx + 1) || !rd(L.E, nx + 1) || !rd(L.S, ny + 1) || !rd(L.N, ny + 1) || !rd(L.u, nn) || !rd(L.f, nn))
    return 2;
  cluster::PlanHost P;
  cluster::plan(nx, ny, wl, colour, P, S, CL);
  if (!P.ok) {
    std::printf("noplan\n");
    return 0;
  }
  const int ncta = (int)P.ctas.size();
  std::vector<CtaMem> mem(ncta);
  const std::vector<T> u0 = L.u;  // every read of a pass sees the other colour only
  // ---- phase 1: chunk right-hand sides and reduced rows
  for (int c = 0; c < ncta; ++c) {
    const CCta &cd = P.ctas[c];
    CtaMem &M = mem[c];
    const int nslot = CL_TILES > S ? CL_TILES * 32 : S * 32;
    M.D.assign((size_t)nslot * 32, 0.0);
    M.rows.assign((size_t)nslot * 2, Row<T>{0, 0, 0, 0});
    M.mlen.assign(nslot, 0);
    M.chx.assign((size_t)nslot * 2, 0.0);
    M.written.assign((size_t)nslot * 2, 0);
    for (int t = 0; t < cd.ntile; ++t) {
      const CTile &td = P.tiles[cd.tile0 + t];
      const Geo g = geo(td.dir);
      for (int lane = 0; lane < 32; ++lane) {
        const CLane &ln = P.lanes[(size_t)32 * (cd.tile0 + t) + lane];
        const int m = ln.q1, slot = t * 32 + lane;
        M.mlen[slot] = m;
        if (m == 0) continue;
        const int base = td.kind == CT_COMPACT ? ln.cbase : td.base;
        const Co co{&L, g, base, ln.line};
        const bool first = ln.flags & TL_FIRST, last_w = ln.flags & TL_LAST_W;
        T *d = &M.D[(size_t)slot * 32];
        for (int q = 0; q < m; ++q) {
          const int v = base + q * g.step;
          const int i = g.xrun ? v : ln.line, j = g.xrun ? ln.line : v;
          const size_t p = (size_t)j * (nx + 1) + i;
          T r = L.F(i, j);
          if (g.xrun) r -= L.S[j] * u0[p - (nx + 1)] + L.N[j] * u0[p + (nx + 1)];
          else r -= L.W[i] * u0[p - 1] + L.E[i] * u0[p + 1];
          const long sv = g.xrun ? g.step : (long)g.step * (nx + 1);
          if (q == 0 && first) r -= co.lo(0) * u0[p - sv];
          if (q == m - 1 && last_w) r -= co.hi(q) * u0[p + sv];
          d[q] = r;
        }
        const T cross = g.xrun ? L.S[ln.line] + L.N[ln.line] : L.W[ln.line] + L.E[ln.line];
        Row<T> rlo, rhi;
        clmath::chunk_reduce<T>(co, m, first, last_w, cross, Arr{d}, rlo, rhi);
        M.rows[(size_t)slot * 2] = rlo;
        M.rows[(size_t)slot * 2 + 1] = rhi;
      }
    }
  }
  // ---- phase 2: block b of a group is solved by the group's CTA b mod ngr:
  // Thomas on each leg's chunk rows from the wall, the junction row,
  // back-substitution; (c', d') overwrite the rows, end values go to chx
  int bad = 0;
  for (int c = 0; c < ncta; ++c) {
    const CCta &cd = P.ctas[c];
    if (cd.group < 0) continue;
    const int cbase = c - (c % CL);  // first CTA of the cluster
    const CBlock *blk = &P.blocks[(size_t)32 * cd.group];
    const CChain *chn = &P.chains[(size_t)128 * cd.group];
    for (int b = cd.grank; b < 32; b += cd.ngr) {
      const CBlock &bd = blk[b];
      T cpl[4] = {0, 0, 0, 0}, dpl[4] = {0, 0, 0, 0};
      auto rows_of = [&](const CChain &ch, int s, CtaMem *&M, CSeg &sg) {
        M = &mem[cbase + ch.rank[s]];
        sg = P.segs[P.ctas[cbase + ch.rank[s]].seg0 + ch.slot[s]];
      };
      for (int l = 0; l < bd.nleg; ++l) {
        const CChain &ch = chn[l * 32 + b];
        T cpv = 0, dpv = 0;
        for (int s = 0; s < ch.nseg; ++s) {
          CtaMem *M;
          CSeg sg;
          rows_of(ch, s, M, sg);
          const int R = 2 * sg.nchunk - sg.one;
          for (int k = 0; k < R; ++k) {
            Row<T> &r = M->rows[(size_t)(sg.slot0 + (k >> 1) * sg.stride) * 2 + (k & 1)];
            const T den = 1.0 / (1.0 - r.a * cpv);
            cpv = r.c * den;
            dpv = (r.y - r.a * dpv) * den;
            r = Row<T>{cpv, dpv, 0, 0};
          }
        }
        cpl[l] = cpv;
        dpl[l] = dpv;
      }
      T xj = 0.0;
      if (bd.junc) {
        const int i = bd.ji, j = bd.jj;
        const size_t p = (size_t)j * (nx + 1) + i;
        unsigned att = 0;
        for (int e = 0; e < bd.nleg; ++e) att |= 1u << ((bd.jdirs >> (2 * e)) & 3);
        T num = L.F(i, j);
        if (!(att & 2u)) num -= L.W[i] * u0[p - 1];
        if (!(att & 1u)) num -= L.E[i] * u0[p + 1];
        if (!(att & 8u)) num -= L.S[j] * u0[p - (nx + 1)];
        if (!(att & 4u)) num -= L.N[j] * u0[p + (nx + 1)];
        T den = -((L.W[i] + L.E[i]) + (L.S[j] + L.N[j]));
        for (int e = 0; e < bd.nleg; ++e) {
          const int d = (bd.jdirs >> (2 * e)) & 3;
          const T k = d == DIR_PX ? L.E[i] : d == DIR_MX ? L.W[i] : d == DIR_PY ? L.N[j] : L.S[j];
          num -= k * dpl[e];
          den -= k * cpl[e];
        }
        xj = num / den;
        L.U(i, j) = xj;
      }
      for (int l = 0; l < bd.nleg; ++l) {
        const CChain &ch = chn[l * 32 + b];
        T xn = bd.junc ? xj : 0.0;
        for (int s = ch.nseg - 1; s >= 0; --s) {
          CtaMem *M;
          CSeg sg;
          rows_of(ch, s, M, sg);
          const int R = 2 * sg.nchunk - sg.one;
          for (int k = R - 1; k >= 0; --k) {
            const size_t slot = sg.slot0 + (k >> 1) * sg.stride;
            const Row<T> &r = M->rows[slot * 2 + (k & 1)];
            xn = r.c - r.a * xn;  // x = d' - c' x_next
            M->chx[slot * 2 + (k & 1)] = xn;
            M->written[slot * 2 + (k & 1)] += 1;
            if (k == R - 1 && sg.one) {
              M->chx[slot * 2 + 1] = xn;
              M->written[slot * 2 + 1] += 1;
            }
          }
        }
      }
    }
  }
  // ---- phase 3: chunk interiors, u
  for (int c = 0; c < ncta; ++c) {
    const CCta &cd = P.ctas[c];
    CtaMem &M = mem[c];
    for (int t = 0; t < cd.ntile; ++t) {
      const CTile &td = P.tiles[cd.tile0 + t];
      const Geo g = geo(td.dir);
      for (int lane = 0; lane < 32; ++lane) {
        const CLane &ln = P.lanes[(size_t)32 * (cd.tile0 + t) + lane];
        const int m = ln.q1, slot = t * 32 + lane;
        if (m == 0) continue;
        if (M.written[(size_t)slot * 2] != 1 || M.written[(size_t)slot * 2 + 1] != 1) bad = 1;
        const int base = td.kind == CT_COMPACT ? ln.cbase : td.base;
        const Co co{&L, g, base, ln.line};
        const bool first = ln.flags & TL_FIRST, last_w = ln.flags & TL_LAST_W;
        const T cross = g.xrun ? L.S[ln.line] + L.N[ln.line] : L.W[ln.line] + L.E[ln.line];
        T x[32], cpv[32];
        XArr xa{x};
        clmath::chunk_expand<T>(co, m, first, last_w, cross, Arr{&M.D[(size_t)slot * 32]}, M.chx[(size_t)slot * 2],
                                M.chx[(size_t)slot * 2 + 1], xa, cpv);
        for (int q = 0; q < m; ++q) {
          const int v = base + q * g.step;
          if (g.xrun) L.U(v, ln.line) = x[q];
          else L.U(ln.line, v) = x[q];
        }
      }
    }
  }
  std::printf("plan %d %zu %zu %zu %d\n", ncta, P.tiles.size(), P.segs.size(), P.blocks.size() / 32, P.total);
  for (size_t k = 0; k < nn; ++k) std::printf("%.17g\n", L.u[k]);
  return bad ? 3 : 0;
}
