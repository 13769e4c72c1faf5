// batch.cu -- many independent problems solved together (mg_batch_create,
// mg_batch_solve, mg_batch_destroy).
//
// Problems whose grids have the same shape, whose parameters are equal
// (FP32 cycles with FP64 refinement) and whose FP32 line passes all take the
// warp path form packed groups: every kernel of their solve serves the whole
// group in one launch (packed.h), and the cycles of a refinement step are one
// CUDA graph per group.  Each member keeps its own solve state and stops at
// its own tolerance (its flag in the group's active array turns its CTAs
// into no-ops), so its arithmetic and results are those of mg_solve on the
// problem alone.  Other problems run their own solve.  Groups and single
// problems are spread over the batch's streams, with one host
// synchronisation per step for all of them.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "packed.h"
#include "solve.h"

using namespace tmg;

namespace {

constexpr int MAX_BATCH_STREAMS = 64;

size_t al16(size_t x) { return (x + 15) & ~size_t(15); }

// Table bytes one problem can take in a packed group (every array of a group
// starts on 16 bytes: at most 16 bytes of padding per array).
size_t problem_table_bytes(const Grid &g) {
  const size_t L = (size_t)g.nlev, arrays = 3 * L + 9;
  return L * (sizeof(PassArgs<float>) + sizeof(RRArgs<float>) + sizeof(ProlongArgs<float>)) +
         sizeof(CoarseArgs<float>) + sizeof(NormArgs) + sizeof(UpdateArgs) + sizeof(RefineArgs) + sizeof(int) +
         sizeof(double) +
         16 * arrays;
}

// The base line smoothers of a smoother (none for checkerboard).
int line_smoothers(int smoother, int wl[2]) {
  if (smoother == MG_SMOOTH_ALT_ZEBRA) { wl[0] = WL_ZEBRA_X; wl[1] = WL_ZEBRA_Y; return 2; }
  if (smoother == MG_SMOOTH_ALT_TW) { wl[0] = WL_TWEED; wl[1] = WL_WIREFRAME; return 2; }
  wl[0] = wl_of(smoother);
  return wl[0] < 0 ? 0 : 1;
}

// Every FP32 colour pass of the smoother takes the warp path on every level
// that is smoothed.
bool warp_everywhere(const Grid &g, int smoother) {
  int wl[2];
  const int n = line_smoothers(smoother, wl);
  if (n == 0) return false;
  for (int l = 0; l + 1 < g.nlev; ++l)
    for (int k = 0; k < n; ++k) {
      const Level &L = g.lev[l];
      const int chosen = L.path[wl[k]][1];
      if (chosen != MG_PATH_AUTO && chosen != MG_PATH_WARP) return false;
      if (L.wp[wl[k]][1][0].nwarp == 0 || L.wp[wl[k]][1][1].nwarp == 0) return false;
    }
  return true;
}

// Same levels, same blocks, same warp shapes: one grid's work lists serve both.
bool same_shape(const Grid &a, const Grid &b, int smoother) {
  if (a.nlev != b.nlev || a.cn != b.cn || a.npartial != b.npartial) return false;
  int wl[2];
  const int n = line_smoothers(smoother, wl);
  for (int l = 0; l < a.nlev; ++l) {
    const Level &A = a.lev[l], &B = b.lev[l];
    if (A.nx != B.nx || A.ny != B.ny) return false;
    for (int k = 0; k < n; ++k)
      for (int c = 0; c < 2; ++c) {
        const WarpList &x = A.wp[wl[k]][1][c], &y = B.wp[wl[k]][1][c];
        if (x.nwarp != y.nwarp || x.K != y.K || x.W != y.W) return false;
      }
  }
  return true;
}

struct Group {
  std::vector<int> members;  // problem indices, batch order
  Grid *g0 = nullptr;        // its work lists serve every member
  mg_params p{};
  size_t base = 0;           // region of the batch's tables
  std::vector<size_t> pass, rr, pr;  // per-level table offsets within the region
  size_t coarse = 0, norm = 0, upd = 0, refine = 0, active = 0, out = 0, end = 0;
  cudaStream_t s = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long graph_launches = 0;
  std::vector<SolveState> q;  // q[k]: member k
  bool done = false;
};

}  // namespace

struct CachedGraph {
  std::vector<const Grid *> grids;
  std::vector<unsigned long long> gens;
  mg_params p{};
  size_t base = 0;
  cudaStream_t s = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long launches = 0;
};

struct mg_batch {
  std::vector<Grid *> grids;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> joins;
  cudaEvent_t fork = nullptr;
  char *dev = nullptr, *host = nullptr;  // packed-group tables: device, pinned host image
  size_t table_bytes = 0;
  std::vector<CachedGraph> graphs;
};

namespace {

void free_batch(mg_batch *b) {
  if (!b) return;
  for (auto &cg : b->graphs) cudaGraphExecDestroy(cg.exec);
  for (auto e : b->joins) cudaEventDestroy(e);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  cudaFree(b->dev);
  if (b->host) cudaFreeHost(b->host);
  delete b;
}

PackedLaunch pk(const mg_batch &b, const Group &G, size_t off) {
  return PackedLaunch{b.dev + G.base + off, reinterpret_cast<const int *>(b.dev + G.base + G.active),
                      (int)G.members.size()};
}

mg_status packed_smooth(const mg_batch &b, const Group &G, int l, int smoother, cudaStream_t s) {
  if (smoother == MG_SMOOTH_ALT_ZEBRA) {
    mg_status st = packed_smooth(b, G, l, MG_SMOOTH_ZEBRA_X, s);
    return st != MG_OK ? st : packed_smooth(b, G, l, MG_SMOOTH_ZEBRA_Y, s);
  }
  if (smoother == MG_SMOOTH_ALT_TW) {
    mg_status st = packed_smooth(b, G, l, MG_SMOOTH_TWEED, s);
    return st != MG_OK ? st : packed_smooth(b, G, l, MG_SMOOTH_WIREFRAME, s);
  }
  const Level &L = G.g0->lev[l];
  const int wl = wl_of(smoother);
  for (int c = 0; c < 2; ++c) {
    const mg_status st =
        cuda_status("warp line pass (packed)", launch_warp_pass_packed<float>(L, L.wp[wl][1][c], pk(b, G, G.pass[l]), s));
    if (st != MG_OK) return st;
  }
  return MG_OK;
}

// Sec. 4 steps (2)-(6) on level l for every member (the FP32 correction
// equation, as run_cycles does for one problem).
mg_status packed_cycle(const mg_batch &b, const Group &G, int l, cudaStream_t s) {
  const Grid &g = *G.g0;
  const mg_params &p = G.p;
  if (l == g.nlev - 1) return cuda_status("coarse solve (packed)", launch_coarse_solve_packed<float>(g, pk(b, G, G.coarse), s));
  mg_status st = MG_OK;
  for (int k = 0; k < p.nu1 && st == MG_OK; ++k) st = packed_smooth(b, G, l, p.smoother, s);
  if (st == MG_OK)
    st = cuda_status("residual+restrict (packed)", launch_residual_restrict_packed<float>(
                                                       g.lev[l], g.lev[l + 1], p.restriction, pk(b, G, G.rr[l]), s));
  for (int k = 0; k < p.cycle && st == MG_OK; ++k) st = packed_cycle(b, G, l + 1, s);
  if (st == MG_OK)
    st = cuda_status("prolong+correct (packed)",
                     launch_prolong_add_packed<float>(g.lev[l], g.lev[l + 1], pk(b, G, G.pr[l]), s));
  for (int k = 0; k < p.nu2 && st == MG_OK; ++k) st = packed_smooth(b, G, l, p.smoother, s);
  return st;
}

// Lays out the group's tables at region `base` and fills their host image.
void build_tables(mg_batch &b, Group &G, double *const *u, const double *const *f) {
  const int P = (int)G.members.size(), nl = G.g0->nlev;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = al16(o + bytes); return at; };
  G.pass.assign(nl, 0); G.rr.assign(nl, 0); G.pr.assign(nl, 0);
  for (int l = 0; l + 1 < nl; ++l) {
    G.pass[l] = take(P * sizeof(PassArgs<float>));
    G.rr[l] = take(P * sizeof(RRArgs<float>));
    G.pr[l] = take(P * sizeof(ProlongArgs<float>));
  }
  G.coarse = take(P * sizeof(CoarseArgs<float>));
  G.norm = take(P * sizeof(NormArgs));
  G.upd = take(P * sizeof(UpdateArgs));
  G.refine = take(P * sizeof(RefineArgs));
  G.active = take(P * sizeof(int));
  G.out = take(P * sizeof(double));
  G.end = o;
  char *h = b.host + G.base;
  for (int k = 0; k < P; ++k) {
    const int i = G.members[k];
    Grid &g = *b.grids[i];
    auto lu = [&](int l) { return l == 0 ? g.e32 : g.lev[l].u32; };
    auto lf = [&](int l) { return l == 0 ? g.r32 : g.lev[l].f32; };
    for (int l = 0; l + 1 < nl; ++l) {
      const Level &L = g.lev[l], &C = g.lev[l + 1];
      reinterpret_cast<PassArgs<float> *>(h + G.pass[l])[k] = PassArgs<float>{level_coefs<float>(L), lu(l), lf(l)};
      reinterpret_cast<RRArgs<float> *>(h + G.rr[l])[k] = RRArgs<float>{level_coefs<float>(L), lu(l), lf(l), C.f32, C.u32};
      reinterpret_cast<ProlongArgs<float> *>(h + G.pr[l])[k] = ProlongArgs<float>{C.u32, lu(l)};
    }
    const Level &Lc = g.lev[nl - 1];
    reinterpret_cast<CoarseArgs<float> *>(h + G.coarse)[k] =
        CoarseArgs<float>{level_coefs<double>(Lc), g.cinv, lu(nl - 1), lf(nl - 1)};
    reinterpret_cast<NormArgs *>(h + G.norm)[k] =
        NormArgs{level_coefs<double>(g.lev[0]), g.lev[0].WE64, u[i], f[i], g.partial,
                 reinterpret_cast<double *>(b.dev + G.base + G.out) + k, g.r32, g.e32};
    reinterpret_cast<UpdateArgs *>(h + G.upd)[k] = UpdateArgs{u[i], g.e32};
    reinterpret_cast<RefineArgs *>(h + G.refine)[k] =
        RefineArgs{level_coefs<double>(g.lev[0]), g.cd64, u[i], g.u2, g.e32, f[i], g.r32, g.e32, g.rpart,
                   reinterpret_cast<double *>(b.dev + G.base + G.out) + k};
    reinterpret_cast<int *>(h + G.active)[k] = 1;
  }
}

// The group's inner FP32 cycles as one graph, reused across calls while the
// members, their work lists, the parameters and the table region stay.
mg_status group_graph(mg_batch &b, Group &G) {
  std::vector<const Grid *> grids;
  std::vector<unsigned long long> gens;
  for (int i : G.members) { grids.push_back(b.grids[i]); gens.push_back(b.grids[i]->gen); }
  for (auto &cg : b.graphs)
    if (cg.grids == grids && cg.gens == gens && cg.base == G.base && cg.s == G.s &&
        std::memcmp(&cg.p, &G.p, sizeof(mg_params)) == 0) {
      G.exec = cg.exec;
      G.graph_launches = cg.launches;
      return MG_OK;
    }
  const unsigned long long l0 = g_launches.load();
  mg_status st = cuda_status("cudaStreamBeginCapture (packed)", cudaStreamBeginCapture(G.s, cudaStreamCaptureModeThreadLocal));
  if (st != MG_OK) return st;
  for (int k = 0; k < G.p.inner_cycles && st == MG_OK; ++k) st = packed_cycle(b, G, 0, G.s);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(G.s, &graph);
  const unsigned long long nl = g_launches.load() - l0;
  g_launches.fetch_sub(nl);  // counted at every replay instead
  if (st == MG_OK) st = cuda_status("cudaStreamEndCapture (packed)", e);
  cudaGraphExec_t exec = nullptr;
  if (st == MG_OK) st = cuda_status("cudaGraphInstantiate (packed)", cudaGraphInstantiate(&exec, graph, 0));
  if (graph) cudaGraphDestroy(graph);
  if (st != MG_OK) return st;
  // replace a cached graph of the same region, else add one
  for (auto &cg : b.graphs)
    if (cg.base == G.base) {
      cudaGraphExecDestroy(cg.exec);
      cg = CachedGraph{grids, gens, G.p, G.base, G.s, exec, nl};
      G.exec = exec;
      G.graph_launches = nl;
      return MG_OK;
    }
  b.graphs.push_back(CachedGraph{grids, gens, G.p, G.base, G.s, exec, nl});
  G.exec = exec;
  G.graph_launches = nl;
  return MG_OK;
}

// One step of every member still running (as enqueue() does for one problem).
mg_status group_enqueue(mg_batch &b, Group &G) {
  const int P = (int)G.members.size();
  char *h = b.host + G.base;
  int phase = -1;
  for (int k = 0; k < P; ++k) {
    // 2: the member's iterate is in its Grid::u2 (refine_residual_kernel)
    reinterpret_cast<int *>(h + G.active)[k] = G.q[k].done ? 0 : (G.q[k].alt ? 2 : 1);
    if (!G.q[k].done) phase = G.q[k].phase;
  }
  cudaStream_t s = G.s;
  const Grid &g = *G.g0;
  mg_status st = cuda_status("cudaMemcpyAsync(active flags)",
                             cudaMemcpyAsync(b.dev + G.base + G.active, h + G.active, P * sizeof(int),
                                             cudaMemcpyHostToDevice, s));
  if (st != MG_OK) return st;
  if (phase == 0) {
    for (auto &x : G.q)
      if (x.info) { x.info->cycles = 0; x.info->outer_iters = 0; x.info->history_len = 0; x.info->rel_res = 0; x.info->conv_factor = 0; }
    if (!G.p.use_initial_guess) st = cuda_status("zero u (packed)", launch_zero_interior_packed(g, pk(b, G, G.upd), s));
    // a zeroed guess: f - B g is also the first defect (its FP32 copy written here)
    const bool merged = !G.p.use_initial_guess;
    if (st == MG_OK)
      st = cuda_status("norm(f - B g) (packed)", launch_norms_packed(g, 1, pk(b, G, G.norm), s, merged));
    for (auto &x : G.q) x.merged = merged;
  } else {
    if (phase == 2) {
      st = cuda_status("cudaGraphLaunch (packed cycles)", cudaGraphLaunch(G.exec, s));
      if (st == MG_OK) count_launch(G.graph_launches);
      std::vector<float *> e32s(P, nullptr);
      for (int k = 0; k < P; ++k)
        if (!G.q[k].done) e32s[k] = G.q[k].g->e32;
      if (st == MG_OK)
        st = cuda_status("refinement update and residual (packed)",
                         launch_refine_residual_packed(g, true, pk(b, G, G.refine), e32s.data(), s));
      for (auto &x : G.q)
        if (!x.done) x.alt = !x.alt;
    } else if (st == MG_OK) {
      st = cuda_status("refinement residual (packed)", launch_refine_residual_packed(g, false, pk(b, G, G.refine),
                                                                                   nullptr, s));
    }
  }
  if (st != MG_OK) return st;
  return cuda_status("cudaMemcpyAsync(norms, packed)", cudaMemcpyAsync(h + G.out, b.dev + G.base + G.out,
                                                                      P * sizeof(double), cudaMemcpyDeviceToHost, s));
}

}  // namespace

extern "C" {

mg_status mg_batch_create(mg_batch **out, int count, mg_grid *const *grids) {
  if (!out || count < 1 || !grids) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<Grid *> gs(count);
  for (int i = 0; i < count; ++i) {
    if (!grids[i]) return MG_ERR_INVALID_ARG;
    if (grids[i]->dim != 2) return MG_ERR_UNSUPPORTED;
    gs[i] = grids[i];
  }
  std::vector<Grid *> sorted(gs);
  std::sort(sorted.begin(), sorted.end());
  if (std::adjacent_find(sorted.begin(), sorted.end()) != sorted.end()) {
    set_error_text("mg_batch_create: a grid appears twice (each problem needs its own grid)");
    return MG_ERR_INVALID_ARG;
  }
  mg_batch *b = new (std::nothrow) mg_batch;
  if (!b) return MG_ERR_ALLOC;
  b->grids = gs;
  for (Grid *g : gs) b->table_bytes += problem_table_bytes(*g);
  const int k = std::min(count, MAX_BATCH_STREAMS);
  cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int i = 0; i < k && e == cudaSuccess; ++i) {
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) b->streams.push_back(s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) b->joins.push_back(ev);
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->dev, b->table_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&b->host, b->table_bytes);
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_status("mg_batch_create", e);
  }
  *out = b;
  return MG_OK;
}

void mg_batch_destroy(mg_batch *b) { free_batch(b); }

mg_status mg_batch_solve(mg_batch *b, double *const *u, const double *const *f, const mg_params *params,
                         int nparams, mg_info *infos, int *status, void *stream) {
  if (!b || !u || !f || !params) return MG_ERR_INVALID_ARG;
  const int n = (int)b->grids.size(), k = (int)b->streams.size();
  if (nparams != 1 && nparams != n) return MG_ERR_INVALID_ARG;
  std::vector<SolveState> q(n);
  for (int i = 0; i < n; ++i) {
    if (!u[i] || !f[i]) return MG_ERR_INVALID_ARG;
    const mg_params *p = params + (nparams == 1 ? 0 : i);
    mg_status st = check_params(b->grids[i], p);
    if (st != MG_OK) return st;
    q[i].g = b->grids[i]; q[i].u = u[i]; q[i].f = f[i]; q[i].p = *p;
    q[i].info = infos ? infos + i : nullptr;
  }
  // packed groups: same grid shape, equal parameters, FP32 cycles whose line
  // passes all take the warp path; at least two members
  std::vector<Group> groups;
  std::vector<int> single;
  {
    std::vector<bool> used(n, false);
    for (int i = 0; i < n; ++i) {
      if (used[i]) continue;
      const mg_params &p = q[i].p;
      const bool packable = p.precision == MG_PREC_F32_REFINE && !p.coarse_direct && q[i].g->dim == 2 &&
                            warp_everywhere(*q[i].g, p.smoother);
      Group G;
      G.members.push_back(i);
      used[i] = true;
      if (packable)
        for (int j = i + 1; j < n; ++j)
          if (!used[j] && std::memcmp(&q[j].p, &p, sizeof(mg_params)) == 0 && warp_everywhere(*q[j].g, p.smoother) &&
              same_shape(*q[i].g, *q[j].g, p.smoother)) {
            G.members.push_back(j);
            used[j] = true;
          }
      if (G.members.size() < 2) {
        single.push_back(i);
        continue;
      }
      G.g0 = q[i].g;
      G.p = p;
      groups.push_back(std::move(G));
    }
  }
  // tables, streams, states
  size_t base = 0;
  int next_stream = 0;
  for (auto &G : groups) {
    G.base = base;
    build_tables(*b, G, u, f);
    base += G.end;
    G.s = b->streams[next_stream++ % k];
    for (int i : G.members) {
      q[i].s = G.s;
      G.q.push_back(q[i]);
    }
  }
  for (int i : single) q[i].s = b->streams[next_stream++ % k];
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the batch's streams start after the caller's stream
  TRY_CUDA("cudaEventRecord(batch fork)", cudaEventRecord(b->fork, s));
  for (auto bs : b->streams) TRY_CUDA("cudaStreamWaitEvent(batch fork)", cudaStreamWaitEvent(bs, b->fork, 0));
  if (base > 0) {
    // the per-member tables in one copy (the group streams wait for it)
    TRY_CUDA("cudaMemcpyAsync(batch tables)", cudaMemcpyAsync(b->dev, b->host, base, cudaMemcpyHostToDevice, b->streams[0]));
    TRY_CUDA("cudaEventRecord(batch tables)", cudaEventRecord(b->fork, b->streams[0]));
    for (auto bs : b->streams) TRY_CUDA("cudaStreamWaitEvent(batch tables)", cudaStreamWaitEvent(bs, b->fork, 0));
  }
  for (auto &G : groups) TRY(group_graph(*b, G));
  mg_status worst = MG_OK;
  int active = n;
  while (active > 0) {
    for (auto &G : groups)
      if (!G.done) TRY(group_enqueue(*b, G));
    for (int i : single)
      if (!q[i].done) TRY(enqueue(q[i]));
    for (auto bs : b->streams) TRY_CUDA("cudaStreamSynchronize(batch)", cudaStreamSynchronize(bs));
    active = 0;
    for (auto &G : groups) {
      if (G.done) continue;
      const double *outv = reinterpret_cast<const double *>(b->host + G.base + G.out);
      bool all = true;
      for (size_t m = 0; m < G.members.size(); ++m) {
        SolveState &x = G.q[m];
        if (x.done) continue;
        consume_value(x, outv[m]);
        all &= x.done;
        active += x.done ? 0 : 1;
      }
      G.done = all;
    }
    for (int i : single)
      if (!q[i].done) {
        consume(q[i]);
        active += q[i].done ? 0 : 1;
      }
  }
  // iterates that ended in a member's Grid::u2 go back to its u, on its stream
  for (auto &G : groups)
    for (auto &x : G.q) TRY(finish_iterate(x));
  for (int i : single) TRY(finish_iterate(q[i]));
  for (auto &G : groups)
    for (size_t m = 0; m < G.members.size(); ++m) q[G.members[m]] = G.q[m];
  for (int i = 0; i < n; ++i)
    if (q[i].st != MG_OK && worst == MG_OK) worst = q[i].st;
  if (status)
    for (int i = 0; i < n; ++i) status[i] = (int)q[i].st;
  // the caller's stream continues after the batch's streams
  for (int i = 0; i < k; ++i) {
    TRY_CUDA("cudaEventRecord(batch join)", cudaEventRecord(b->joins[i], b->streams[i]));
    TRY_CUDA("cudaStreamWaitEvent(batch join)", cudaStreamWaitEvent(s, b->joins[i], 0));
  }
  return checked(worst);
}

}  // extern "C"
