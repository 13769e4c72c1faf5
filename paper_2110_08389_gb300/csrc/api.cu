// api.cu -- the C ABI of tweedmg (include/mg.h): grid setup, the cycle driver
// (Sec. 4 steps (1)-(6)), the FP64 solve, the FP32 + FP64 iterative
// refinement solve and the adjoint solve.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "solve.h"

namespace tmg {

std::atomic<unsigned long long> g_launches{0};
static thread_local char g_err[512] = "";

const char *set_error(const char *where, cudaError_t e) {
  std::snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return g_err;
}

void set_error_text(const char *msg) { std::snprintf(g_err, sizeof(g_err), "%s", msg); }

mg_status cuda_status(const char *where, cudaError_t e) {
  if (e == cudaSuccess) return MG_OK;
  set_error(where, e);
  return e == cudaErrorMemoryAllocation ? MG_ERR_ALLOC : MG_ERR_CUDA;
}

// Sec. 2 coefficients on one axis: lo_i = 1/(dx_i dx_{i-1/2}),
// hi_i = 1/(dx_i dx_{i+1/2}), dx_i = (x_{i+1} - x_{i-1})/2; 0 at the ends.
void axis_coefficients(const std::vector<double> &x, std::vector<double> &lo, std::vector<double> &hi) {
  const size_t n = x.size() - 1;
  lo.assign(n + 1, 0.0);
  hi.assign(n + 1, 0.0);
  for (size_t i = 1; i < n; ++i) {
    const double h_minus = x[i] - x[i - 1], h_plus = x[i + 1] - x[i];
    const double h_mid = 0.5 * (x[i + 1] - x[i - 1]);
    lo[i] = 1.0 / (h_mid * h_minus);
    hi[i] = 1.0 / (h_mid * h_plus);
  }
}

static void destroy_timer(Grid *g) {
  if (!g->timer_ev) return;
  for (int k = 0; k < 4 * g->timer_cap; ++k) cudaEventDestroy(g->timer_ev[k]);
  delete[] g->timer_ev;
  g->timer_ev = nullptr;
  g->timer_cap = g->timer_n = 0;
  g->timer_level = -1;
}

void drop_graphs(Grid &g) {
  for (auto &ge : g.graphs) cudaGraphExecDestroy(ge.exec);
  g.graphs.clear();
}

static void free_grid(Grid *g) {
  if (!g) return;
  destroy_timer(g);
  drop_graphs(*g);
  free3(*g);
  if (g->ev_fork) cudaEventDestroy(g->ev_fork);
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->gs) cudaStreamDestroy(g->gs);
  for (Level &L : g->lev) {
    cudaFree(L.dev_block);
    cudaFree(L.u64); cudaFree(L.f64); cudaFree(L.u32); cudaFree(L.f32);
    for (int w = 0; w < WL_COUNT; ++w)
      for (int c = 0; c < 2; ++c) {
        cudaFree(L.tl[w][c].mem);
        cudaFree(L.cp[w][c].mem);
        for (int p = 0; p < 2; ++p) {
          for (int z = 0; z < 2; ++z) cudaFree(L.wl[w][p][c][z].mem);
          cudaFree(L.wp[w][p][c].mem);
        }
      }
  }
  cudaFree(g->cinv);
  cudaFree(g->fd_tr);
  cudaFree(g->r64); cudaFree(g->e32); cudaFree(g->r32);
  cudaFree(g->u2); cudaFree(g->cd64); cudaFree(g->rpart);
  cudaFree(g->partial); cudaFree(g->scal); cudaFree(g->dev_status);
  cudaFree(g->tile_rows); cudaFree(g->tile_d); cudaFree(g->tile_x);
  if (g->hpinned) cudaFreeHost(g->hpinned);
  delete g;
}

template <typename X>
static mg_status dalloc(X **p, size_t n, const char *what) {
  TRY_CUDA(what, cudaMalloc(reinterpret_cast<void **>(p), sizeof(X) * n));
  TRY_CUDA(what, cudaMemset(*p, 0, sizeof(X) * n));
  return MG_OK;
}

// Gauss-Jordan inverse with partial pivoting (FP64, host), for the coarsest
// level's dense direct solve.
bool invert(int n, std::vector<double> &A, std::vector<double> &inv) {
  inv.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int k = 0; k < n; ++k) {
    int p = k;
    for (int r = k + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + k]) > std::fabs(A[(size_t)p * n + k])) p = r;
    if (A[(size_t)p * n + k] == 0.0) return false;
    if (p != k)
      for (int c = 0; c < n; ++c) {
        std::swap(A[(size_t)k * n + c], A[(size_t)p * n + c]);
        std::swap(inv[(size_t)k * n + c], inv[(size_t)p * n + c]);
      }
    const double d = 1.0 / A[(size_t)k * n + k];
    for (int c = 0; c < n; ++c) { A[(size_t)k * n + c] *= d; inv[(size_t)k * n + c] *= d; }
    for (int r = 0; r < n; ++r) {
      if (r == k) continue;
      const double l = A[(size_t)r * n + k];
      if (l == 0.0) continue;
      for (int c = 0; c < n; ++c) {
        A[(size_t)r * n + c] -= l * A[(size_t)k * n + c];
        inv[(size_t)r * n + c] -= l * inv[(size_t)k * n + c];
      }
    }
  }
  return true;
}

// What every solve needs besides the levels: norm partials and scalars, the
// pinned host copy of the norms, the graph stream and its events.
static mg_status setup_solver_state(Grid *g) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  g->sms = sms;
  g->npartial = 4 * sms;
  TRY(dalloc(&g->partial, 2 * (size_t)g->npartial, "cudaMalloc(partials)"));
  TRY(dalloc(&g->scal, 4, "cudaMalloc(scalars)"));
  TRY(dalloc(&g->dev_status, 1, "cudaMalloc(device status)"));
  TRY_CUDA("cudaMallocHost", cudaMallocHost(&g->hpinned, 4 * sizeof(double)));
  TRY_CUDA("cudaStreamCreate(graph stream)", cudaStreamCreateWithFlags(&g->gs, cudaStreamNonBlocking));
  TRY_CUDA("cudaEventCreate(fork)", cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
  TRY_CUDA("cudaEventCreate(join)", cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
  return MG_OK;
}

static mg_status setup(Grid *g, int nx, int ny, const double *x, const double *y) {
  // level hierarchy: drop every other line while both sides are even, keep at
  // least 2 intervals, and stop once max(nx, ny) <= 8
  int cx = nx, cy = ny;
  std::vector<double> xs(x, x + nx + 1), ys(y, y + ny + 1);
  while (true) {
    Level L;
    L.nx = cx; L.ny = cy; L.nn = (size_t)(cx + 1) * (cy + 1);
    L.hx = xs; L.hy = ys;
    axis_coefficients(xs, L.hW, L.hE);
    axis_coefficients(ys, L.hS, L.hN);
    g->lev.push_back(std::move(L));
    if (cx % 2 || cy % 2 || cx / 2 < 2 || cy / 2 < 2 || std::max(cx, cy) <= 8) break;
    std::vector<double> xn(cx / 2 + 1), yn(cy / 2 + 1);
    for (int i = 0; i <= cx / 2; ++i) xn[i] = xs[2 * i];
    for (int j = 0; j <= cy / 2; ++j) yn[j] = ys[2 * j];
    xs.swap(xn); ys.swap(yn);
    cx /= 2; cy /= 2;
  }
  g->nlev = (int)g->lev.size();
  TRY_CUDA("setup start (latched error)", cudaGetLastError());
  TRY_CUDA("line kernel attributes", prepare_line_kernels());
  TRY_CUDA("tile kernel attributes", prepare_tile_kernels());
  TRY_CUDA("warp kernel attributes", prepare_warp_kernels());
  TRY_CUDA("cluster kernel attributes", prepare_cluster_kernel());
  g->cluster_ok = (g->prec_mask & 2) && cluster_pass_capacity() > 0;
  const bool want64 = g->prec_mask & 1, want32 = g->prec_mask & 2;
  for (int l = 0; l < g->nlev; ++l) {
    Level &L = g->lev[l];
    const size_t a = L.nx + 1, b = L.ny + 1;
    // doubles: W E x W+E (a each), S N y (b each); floats after them
    const size_t nd = 4 * a + 3 * b, nf = 2 * a + 2 * b;
    const size_t bytes = sizeof(double) * nd + sizeof(float) * nf + 16;
    TRY_CUDA("cudaMalloc(coefficients)", cudaMalloc(&L.dev_block, bytes));
    double *dp = static_cast<double *>(L.dev_block);
    L.W64 = dp; L.E64 = dp + a; L.xd = dp + 2 * a; L.S64 = dp + 3 * a; L.N64 = dp + 3 * a + b; L.yd = dp + 3 * a + 2 * b;
    L.WE64 = dp + 3 * a + 3 * b;
    float *fp = reinterpret_cast<float *>(dp + nd);
    L.W32 = fp; L.E32 = fp + a; L.S32 = fp + 2 * a; L.N32 = fp + 2 * a + b;
    std::vector<double> hd(nd);
    std::vector<float> hf(nf);
    for (size_t i = 0; i < a; ++i) { hd[i] = L.hW[i]; hd[a + i] = L.hE[i]; hd[2 * a + i] = L.hx[i]; }
    for (size_t i = 0; i < a; ++i) hd[3 * a + 3 * b + i] = L.hW[i] + L.hE[i];
    for (size_t j = 0; j < b; ++j) { hd[3 * a + j] = L.hS[j]; hd[3 * a + b + j] = L.hN[j]; hd[3 * a + 2 * b + j] = L.hy[j]; }
    for (size_t i = 0; i < a; ++i) { hf[i] = (float)L.hW[i]; hf[a + i] = (float)L.hE[i]; }
    for (size_t j = 0; j < b; ++j) { hf[2 * a + j] = (float)L.hS[j]; hf[2 * a + b + j] = (float)L.hN[j]; }
    TRY_CUDA("cudaMemcpy(coefficients)", cudaMemcpy(dp, hd.data(), sizeof(double) * nd, cudaMemcpyHostToDevice));
    TRY_CUDA("cudaMemcpy(coefficients)", cudaMemcpy(fp, hf.data(), sizeof(float) * nf, cudaMemcpyHostToDevice));
    if (l > 0) {
      if (want64) { TRY(dalloc(&L.u64, L.nn, "cudaMalloc(level u64)")); TRY(dalloc(&L.f64, L.nn, "cudaMalloc(level f64)")); }
      if (want32) { TRY(dalloc(&L.u32, L.nn, "cudaMalloc(level u32)")); TRY(dalloc(&L.f32, L.nn, "cudaMalloc(level f32)")); }
    }
  }
  // coarsest level: dense inverse of the interior operator
  {
    const Level &L = g->lev[g->nlev - 1];
    const int n = (L.nx - 1) * (L.ny - 1);
    if (n > 1024) return MG_ERR_SIZE;
    g->cn = n;
    if (n > 0) {
      std::vector<double> A((size_t)n * n, 0.0), inv;
      for (int j = 1; j < L.ny; ++j)
        for (int i = 1; i < L.nx; ++i) {
          const int r = (j - 1) * (L.nx - 1) + (i - 1);
          A[(size_t)r * n + r] = -(L.hW[i] + L.hE[i] + L.hS[j] + L.hN[j]);
          if (i > 1) A[(size_t)r * n + r - 1] = L.hW[i];
          if (i < L.nx - 1) A[(size_t)r * n + r + 1] = L.hE[i];
          if (j > 1) A[(size_t)r * n + r - (L.nx - 1)] = L.hS[j];
          if (j < L.ny - 1) A[(size_t)r * n + r + (L.nx - 1)] = L.hN[j];
        }
      if (!invert(n, A, inv)) return MG_ERR_SIZE;
      TRY_CUDA("cudaMalloc(coarse)", cudaMalloc(&g->cinv, sizeof(double) * inv.size()));
      TRY_CUDA("cudaMemcpy(coarse)", cudaMemcpy(g->cinv, inv.data(), sizeof(double) * inv.size(), cudaMemcpyHostToDevice));
    }
  }
  TRY_CUDA("setup levels (latched error)", cudaGetLastError());
  const size_t nn0 = g->lev[0].nn;
  if (want32) { TRY(dalloc(&g->e32, nn0, "cudaMalloc(e32)")); TRY(dalloc(&g->r32, nn0, "cudaMalloc(r32)")); }
  if (want64) TRY(dalloc(&g->r64, nn0, "cudaMalloc(adjoint scratch)"));
  TRY(setup_direct_level(*g));
  TRY(setup_solver_state(g));
  if (want32 && g->dim == 2) TRY(setup_refine_residual(*g));
  // block work lists of every line smoother on every level, so that no later
  // call allocates
  TRY_CUDA("setup scratch (latched error)", cudaGetLastError());
  for (int l = 0; l < g->nlev; ++l)
    for (int wl = 0; wl < WL_COUNT; ++wl) {
      for (int prec = 0; prec < 2; ++prec)
        if (g->prec_mask & (prec == 0 ? 1 : 2)) TRY(build_worklists(*g, l, wl, prec));
      TRY_CUDA("setup work lists (latched error)", cudaGetLastError());
      TRY(build_tiles(*g, l, wl));
      TRY_CUDA("setup tiles (latched error)", cudaGetLastError());
      TRY(build_cluster_plans(*g, l, wl));
      TRY_CUDA("setup cluster plans (latched error)", cudaGetLastError());
    }
  if (g->tile_cap > 0) {
    // scratch of the tiled path, sized for FP64 (FP32 uses the first half)
    // rows (2 x 4 doubles per lane) followed by the (c', d') pairs of tile_couple
    TRY_CUDA("cudaMalloc(tile rows)", cudaMalloc(&g->tile_rows, g->tile_cap * 32 * 2 * 6 * sizeof(double)));
    TRY_CUDA("cudaMalloc(tile rhs)", cudaMalloc(&g->tile_d, g->tile_cap * 32 * 32 * sizeof(double)));
    TRY_CUDA("cudaMalloc(tile ends)", cudaMalloc(&g->tile_x, g->tile_cap * 32 * 2 * sizeof(double)));
    if (want32) TRY_CUDA("tile couple constants", setup_couple_consts(*g));
  }
  TRY_CUDA("setup (latched error)", cudaGetLastError());
  return MG_OK;
}

// ------------------------------------------------------------------ driver --

template <typename T> static T *level_u(Level &L);
template <typename T> static T *level_f(Level &L);
template <> double *level_u<double>(Level &L) { return L.u64; }
template <> double *level_f<double>(Level &L) { return L.f64; }
template <> float *level_u<float>(Level &L) { return L.u32; }
template <> float *level_f<float>(Level &L) { return L.f32; }

int wl_of(int smoother) {
  switch (smoother) {
    case MG_SMOOTH_ZEBRA_X: return WL_ZEBRA_X;
    case MG_SMOOTH_ZEBRA_Y: return WL_ZEBRA_Y;
    case MG_SMOOTH_TWEED: return WL_TWEED;
    case MG_SMOOTH_WIREFRAME: return WL_WIREFRAME;
  }
  return -1;
}

// The 4 timer events of this pass, or nullptr when level l is not timed.
static cudaEvent_t *timer_slot(Grid &g, int l) {
  if (!g.timer_ev || l != g.timer_level || g.timer_n >= g.timer_cap) return nullptr;
  return g.timer_ev + 4 * g.timer_n++;
}

template <typename T>
static mg_status colour_pass(Grid &g, int l, int smoother, int colour, T *u, const T *f, cudaStream_t s) {
  Level &L = g.lev[l];
  const int wl = smoother == MG_SMOOTH_CHECKERBOARD ? -2 : wl_of(smoother);
  if (wl == -1) return MG_ERR_INVALID_ARG;
  const int prec = sizeof(T) == 8 ? 0 : 1;
  if (wl >= 0) TRY(build_worklists(g, l, wl, prec));
  // path: the one set by mg_set_line_path / mg_autotune, else the warp path
  // where the level's blocks fit it, else the tiled path (large levels), else
  // the CTA line kernel
  const int chosen = wl >= 0 ? L.path[wl][prec] : MG_PATH_AUTO;
  const TileList *tl = wl >= 0 ? &L.tl[wl][colour] : nullptr;
  const bool has_tiles = tl && (tl->ntile > 0 || tl->nblock > 0);
  const bool warp = wl >= 0 && L.wp[wl][prec][colour].nwarp > 0 &&
                    (chosen == MG_PATH_AUTO || chosen == MG_PATH_WARP);
  const bool clustered = !warp && sizeof(T) == 4 && wl >= 0 && L.cp[wl][colour].ncta > 0 &&
                         chosen == MG_PATH_CLUSTER;
  const bool tiled = !warp && !clustered && has_tiles && (chosen == MG_PATH_AUTO || chosen == MG_PATH_TILED);
  cudaEvent_t *ev = timer_slot(g, l);
  if constexpr (sizeof(T) == 4) {
    if (clustered) {
      TRY_CUDA("cluster line pass", launch_cluster_pass(L, L.cp[wl][colour], u, f, s, ev));
      return MG_OK;
    }
  }
  if (tiled) {
    TRY_CUDA("tiled line pass", launch_tile_pass<T>(g, L, *tl, u, f, s, ev));
    return MG_OK;
  }
  // other passes: the whole pass falls in the third timer stage
  if (ev) for (int k = 0; k < 3; ++k) cudaEventRecord(ev[k], s);
  if (wl == -2) {
    TRY_CUDA("checker pass", launch_checker_pass<T>(L, colour, u, f, s));
  } else if (warp) {
    TRY_CUDA("warp line pass", launch_warp_pass<T>(L, L.wp[wl][prec][colour], u, f, s));
  } else {
    TRY_CUDA("line pass", launch_line_pass<T>(L, L.wl[wl][prec][colour][0], u, f, s));
    TRY_CUDA("line pass (large blocks)", launch_line_pass<T>(L, L.wl[wl][prec][colour][1], u, f, s));
  }
  if (ev) cudaEventRecord(ev[3], s);
  return MG_OK;
}

// One relaxation (red pass, then black pass; the alternating schemes run one
// relaxation of each of their two smoothers).
template <typename T>
static mg_status smooth(Grid &g, int l, int smoother, T *u, const T *f, cudaStream_t s) {
  if (smoother == MG_SMOOTH_ALT_ZEBRA) {
    TRY(smooth(g, l, MG_SMOOTH_ZEBRA_X, u, f, s));
    return smooth(g, l, MG_SMOOTH_ZEBRA_Y, u, f, s);
  }
  if (smoother == MG_SMOOTH_ALT_TW) {
    TRY(smooth(g, l, MG_SMOOTH_TWEED, u, f, s));
    return smooth(g, l, MG_SMOOTH_WIREFRAME, u, f, s);
  }
  TRY(colour_pass(g, l, smoother, 0, u, f, s));
  return colour_pass(g, l, smoother, 1, u, f, s);
}

// Sec. 4 steps (2)-(6) on level l; gamma = 1 (V) or 2 (W).
template <typename T>
static mg_status cycle_rec(Grid &g, const mg_params &p, int l, T *u, const T *f, cudaStream_t s) {
  if (g.dim == 3) return cycle3<T>(g, p, l, u, f, s);
  if constexpr (sizeof(T) == 4) {
    if (p.coarse_direct && l == g.fd_level) {
      TRY_CUDA("direct level solve", launch_direct_level(g, (float *)u, (const float *)f, s));
      return MG_OK;
    }
  }
  if (l == g.nlev - 1) {
    TRY_CUDA("coarse solve", launch_coarse_solve<T>(g, u, f, s));
    return MG_OK;
  }
  for (int k = 0; k < p.nu1; ++k) TRY(smooth(g, l, p.smoother, u, f, s));
  Level &F = g.lev[l], &C = g.lev[l + 1];
  T *uc = level_u<T>(C), *fc = level_f<T>(C);
  TRY_CUDA("residual+restrict", launch_residual_restrict<T>(F, C, p.restriction, u, f, fc, uc, s));
  for (int k = 0; k < p.cycle; ++k) TRY(cycle_rec<T>(g, p, l + 1, uc, fc, s));
  TRY_CUDA("prolong+correct", launch_prolong_add<T>(F, C, uc, u, s));
  for (int k = 0; k < p.nu2; ++k) TRY(smooth(g, l, p.smoother, u, f, s));
  return MG_OK;
}

// ncyc cycles (Sec. 4) on level 0 from (u, f).  The launch sequence of a
// cycle depends only on the grid, the parameters and the two arrays, so it is
// captured once into a CUDA graph and replayed: one submission instead of
// about a hundred launches, and shorter gaps between the kernels.  Direct
// launches while the pass timer runs (its events are per pass) or when the
// caller's stream is itself being captured.
constexpr size_t MAX_GRAPHS = 8;

template <typename T>
static mg_status run_cycles(Grid &g, const mg_params &p, int ncyc, T *u, const T *f, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TRY_CUDA("cudaStreamIsCapturing", cudaStreamIsCapturing(s, &cs));
  if (g.timer_ev || cs != cudaStreamCaptureStatusNone || !g.gs) {
    for (int k = 0; k < ncyc; ++k) TRY(cycle_rec<T>(g, p, 0, u, f, s));
    return MG_OK;
  }
  const int key[8] = {(int)sizeof(T), p.smoother, p.nu1, p.nu2, p.cycle, p.restriction, ncyc, p.coarse_direct};
  Grid::GraphEntry *ge = nullptr;
  for (auto &x : g.graphs)
    if (x.u == u && x.f == f && std::memcmp(x.key, key, sizeof(key)) == 0) { ge = &x; break; }
  if (!ge) {
    const unsigned long long l0 = g_launches.load();
    TRY_CUDA("cudaStreamBeginCapture", cudaStreamBeginCapture(g.gs, cudaStreamCaptureModeThreadLocal));
    mg_status st = MG_OK;
    for (int k = 0; k < ncyc && st == MG_OK; ++k) st = cycle_rec<T>(g, p, 0, u, f, g.gs);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(g.gs, &graph);
    const unsigned long long nl = g_launches.load() - l0;
    g_launches.fetch_sub(nl);  // counted again at every replay
    if (st != MG_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return st != MG_OK ? st : cuda_status("cudaStreamEndCapture", e);
    }
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_status("cudaGraphInstantiate", e);
    if (g.graphs.size() >= MAX_GRAPHS) {
      cudaGraphExecDestroy(g.graphs.front().exec);
      g.graphs.erase(g.graphs.begin());
    }
    Grid::GraphEntry ne;
    std::memcpy(ne.key, key, sizeof(key));
    ne.u = u; ne.f = f; ne.exec = ex; ne.launches = nl;
    g.graphs.push_back(ne);
    ge = &g.graphs.back();
  }
  TRY_CUDA("cudaEventRecord(fork)", cudaEventRecord(g.ev_fork, s));
  TRY_CUDA("cudaStreamWaitEvent(fork)", cudaStreamWaitEvent(g.gs, g.ev_fork, 0));
  TRY_CUDA("cudaGraphLaunch", cudaGraphLaunch(ge->exec, g.gs));
  count_launch(ge->launches);
  TRY_CUDA("cudaEventRecord(join)", cudaEventRecord(g.ev_join, g.gs));
  TRY_CUDA("cudaStreamWaitEvent(join)", cudaStreamWaitEvent(s, g.ev_join, 0));
  return MG_OK;
}

mg_status check_params(const Grid *g, const mg_params *p) {
  if (!p) return MG_ERR_INVALID_ARG;
  if (p->smoother < 0 || p->smoother > MG_SMOOTH_ALT_TW) return MG_ERR_INVALID_ARG;
  if (p->nu1 < 0 || p->nu2 < 0 || p->nu1 + p->nu2 > 64) return MG_ERR_INVALID_ARG;
  if (p->cycle != MG_CYCLE_V && p->cycle != MG_CYCLE_W) return MG_ERR_INVALID_ARG;
  if (p->restriction != MG_RESTRICT_HW && p->restriction != MG_RESTRICT_FW) return MG_ERR_INVALID_ARG;
  if (p->precision == MG_PREC_F64 && !(g->prec_mask & 1)) return MG_ERR_INVALID_ARG;
  if (p->precision == MG_PREC_F32_REFINE && !(g->prec_mask & 2)) return MG_ERR_INVALID_ARG;
  if (p->precision != MG_PREC_F64 && p->precision != MG_PREC_F32_REFINE) return MG_ERR_INVALID_ARG;
  if (!(p->tol >= 0.0) || p->max_cycles < 0 || p->max_outer < 0 || p->inner_cycles < 1) return MG_ERR_INVALID_ARG;
  if ((p->early_stop != 0 && p->early_stop != 1) || (p->coarse_direct != 0 && p->coarse_direct != 1))
    return MG_ERR_INVALID_ARG;
  if (g->dim == 3 && p->coarse_direct) return MG_ERR_UNSUPPORTED;
  // 3D grids: tweed, wireframe or both alternating, with full weighting (Sec. 7)
  if (g->dim == 3 && ((p->smoother != MG_SMOOTH_TWEED && p->smoother != MG_SMOOTH_WIREFRAME &&
                       p->smoother != MG_SMOOTH_ALT_TW) ||
                      p->restriction != MG_RESTRICT_FW))
    return MG_ERR_UNSUPPORTED;
  if (g->dim == 3 && p->smoother != MG_SMOOTH_TWEED)
    for (int l = 0; l + 1 < g->nlev; ++l)
      if (!g->g3->lev[l].wf_ok) return MG_ERR_UNSUPPORTED;
  return MG_OK;
}

static void record(mg_info *info, int k, double rel) {
  if (info && info->history && k < info->history_cap) {
    info->history[k] = rel;
    info->history_len = k + 1;
  }
}

static mg_status copy_norm(Grid &g, cudaStream_t s) {
  TRY_CUDA("cudaMemcpyAsync(norms)", cudaMemcpyAsync(g.hpinned, g.scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  return MG_OK;
}

mg_status enqueue(SolveState &q) {
  Grid &g = *q.g;
  const mg_params &p = q.p;
  const bool f64 = p.precision == MG_PREC_F64;
  const bool d3 = g.dim == 3;
  if (q.phase == 0) {
    if (q.info) { q.info->cycles = 0; q.info->outer_iters = 0; q.info->history_len = 0; q.info->rel_res = 0; q.info->conv_factor = 0; }
    if (!p.use_initial_guess) {
      if (d3) TRY(zero_interior3(g, q.u, q.s));
      else TRY_CUDA("zero u", launch_zero_interior<double>(g.lev[0], q.u, q.s));
    }
    // scale of the relative residual: ||f - B g||, the right-hand side of the
    // interior system (||f|| when the boundary data vanish)
    if (d3) {
      TRY(norms3(g, q.u, q.f, 1, nullptr, nullptr, q.s));
    } else if (!f64 && !p.use_initial_guess) {
      // the interior of u is zero: f - B g is also the first defect, so this
      // launch writes its FP32 copy and the next step starts the cycles
      TRY_CUDA("norm(f - B g) and first residual", launch_rhsnorm64(g, q.u, q.f, q.s, g.r32, g.e32));
      q.merged = true;
    } else {
      TRY_CUDA("norm(f - B g)", launch_rhsnorm64(g, q.u, q.f, q.s));
    }
  } else if (f64) {
    if (q.phase == 2) TRY(run_cycles<double>(g, p, 1, q.u, q.f, q.s));
    if (d3) TRY(norms3(g, q.u, q.f, 0, nullptr, nullptr, q.s));
    else TRY_CUDA("residual norm", launch_resnorm64(g, q.u, q.f, q.s));
  } else {
    // FP32 cycles on the correction equation L e = r (e zeroed by the
    // residual kernel), FP64 residual and update
    if (d3) {
      if (q.phase == 2) {
        TRY(run_cycles<float>(g, p, p.inner_cycles, g.e32, g.r32, q.s));
        TRY(ir_update3(g, q.u, g.e32, q.s));
      }
      TRY(norms3(g, q.u, q.f, 0, g.r32, g.e32, q.s));
    } else if (q.phase == 2) {
      // the update u + e and the next residual in one launch, into the other iterate
      TRY(run_cycles<float>(g, p, p.inner_cycles, g.e32, g.r32, q.s));
      double *cur = q.alt ? g.u2 : q.u, *nxt = q.alt ? q.u : g.u2;
      TRY_CUDA("refinement update and residual", launch_refine_residual(g, cur, g.e32, nxt, q.f, q.s));
      q.alt = !q.alt;
    } else {
      TRY_CUDA("refinement residual", launch_refine_residual(g, q.u, nullptr, nullptr, q.f, q.s));
    }
  }
  return copy_norm(g, q.s);
}

static void finish(SolveState &q) {
  q.done = true;
  if (q.st == MG_OK && !std::isfinite(q.rel)) q.st = MG_ERR_NONFINITE;
  if (!q.info) return;
  const int n = q.cycles;
  q.info->cycles = n;
  q.info->outer_iters = q.outer;
  q.info->rel_res = q.rel;
  q.info->conv_factor = (n > 0 && q.rel0 > 0 && q.rel > 0) ? std::pow(q.rel / q.rel0, 1.0 / n) : 0.0;
}

void consume(SolveState &q) { consume_value(q, q.g->hpinned[0]); }

void consume_value(SolveState &q, double v) {
  const mg_params &p = q.p;
  const bool f64 = p.precision == MG_PREC_F64;
  if (q.phase == 0) {
    q.fn = std::sqrt(v);
    q.phase = 1;
    if (!q.merged) return;
    q.merged = false;  // v is also the first residual's: on to the first step
  }
  if (q.phase == 1) {
    if (q.fn == 0.0) q.fn = std::sqrt(v) > 0.0 ? std::sqrt(v) : 1.0;
    q.rel = q.rel0 = std::sqrt(v) / q.fn;
    record(q.info, 0, q.rel);
    q.phase = 2;
  } else {
    if (f64) {
      q.cycles += 1;
    } else {
      q.cycles += p.inner_cycles;
      q.outer += 1;
    }
    q.prev = q.rel;
    q.rel = std::sqrt(v) / q.fn;
    record(q.info, f64 ? q.cycles : q.outer, q.rel);
  }
  if (q.rel <= p.tol) return finish(q);
  if (!std::isfinite(q.rel)) { q.st = MG_ERR_NONFINITE; return finish(q); }
  const bool limit = f64 ? q.cycles >= p.max_cycles : (q.outer >= p.max_outer || q.cycles >= p.max_cycles);
  if (limit || q.rel > 1e3 * q.rel0) { q.st = MG_ERR_NOT_CONVERGED; return finish(q); }
  // early stop: at the last step's rate the steps left under the caps fall short
  const int steps = f64 ? q.cycles : q.outer;
  if (p.early_stop && q.phase == 2) {
    const int left = steps_left(f64, p.max_cycles, p.max_outer, p.inner_cycles, q.cycles, q.outer);
    if (hopeless(steps, q.rel, q.prev, left, p.tol)) { q.st = MG_ERR_NOT_CONVERGED; return finish(q); }
  }
}

// A finished solve whose iterate ended in Grid::u2 copies its interior back
// into u (u keeps its own boundary: the data, corners included, which the
// five-point stencil never reads and the refinement never writes into u2).
mg_status finish_iterate(SolveState &q) {
  if (!q.alt) return MG_OK;
  q.alt = false;
  const Level &L = q.g->lev[0];
  const size_t pitch = (size_t)(L.nx + 1) * sizeof(double), first = (size_t)(L.nx + 1) + 1;
  TRY_CUDA("cudaMemcpy2DAsync(iterate)",
           cudaMemcpy2DAsync(q.u + first, pitch, q.g->u2 + first, pitch, (size_t)(L.nx - 1) * sizeof(double),
                             (size_t)(L.ny - 1), cudaMemcpyDeviceToDevice, q.s));
  return MG_OK;
}

static mg_status solve_impl(Grid &g, double *u, const double *f, const mg_params &p, mg_info *info,
                            cudaStream_t s) {
  SolveState q;
  q.g = &g; q.u = u; q.f = f; q.p = p; q.info = info; q.s = s;
  while (!q.done) {
    TRY(enqueue(q));
    TRY_CUDA("cudaStreamSynchronize", cudaStreamSynchronize(s));
    consume(q);
  }
  if (q.alt) {
    TRY(finish_iterate(q));
    TRY_CUDA("cudaStreamSynchronize", cudaStreamSynchronize(s));
  }
  return q.st;
}

}  // namespace tmg

using namespace tmg;

namespace tmg {

struct CheckReader {
  const char *tu;
  unsigned (*read)(unsigned *line);
};
static std::vector<CheckReader> &check_readers() {
  static std::vector<CheckReader> r;
  return r;
}
void register_check_reader(const char *tu, unsigned (*reader)(unsigned *line)) {
  check_readers().push_back({tu, reader});
}
unsigned check_words(std::string *where) {
  unsigned w = 0;
  for (const CheckReader &r : check_readers()) {
    unsigned line = 0;
    const unsigned v = r.read(&line);
    if (v != 0u && where && where->empty()) *where = std::string(r.tu) + ", line " + std::to_string(line);
    w |= v;
  }
  return w;
}

// In checked builds (-DMG_CHECK) every entry that launches kernels waits for
// them and turns a recorded out-of-range index into MG_ERR_INVALID_ARG.
mg_status checked(mg_status st) {
#ifdef MG_CHECK
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status("checked build: synchronize", e);
  std::string where;
  if (check_words(&where) != 0u) {
    set_error_text(("checked build: a kernel met an index out of its level's range (" + where + ")").c_str());
    return MG_ERR_INVALID_ARG;
  }
#endif
  return st;
}

}  // namespace tmg

extern "C" {

unsigned mg_check_word(void) {
#ifdef MG_CHECK
  cudaDeviceSynchronize();
  return check_words() | 0x80000000u;
#else
  return 0u;
#endif
}

void mg_default_params(mg_params *p) {
  if (!p) return;
  p->smoother = MG_SMOOTH_TWEED;
  p->nu1 = 2; p->nu2 = 2;
  p->cycle = MG_CYCLE_V;
  p->restriction = MG_RESTRICT_FW;
  p->precision = MG_PREC_F64;
  p->max_cycles = 100;
  p->max_outer = 8;
  p->inner_cycles = 3;
  p->use_initial_guess = 0;
  p->early_stop = 0;
  p->coarse_direct = 0;
  p->tol = 1e-10;
}

const char *mg_status_string(mg_status s) {
  switch (s) {
    case MG_OK: return "ok";
    case MG_ERR_INVALID_ARG: return "invalid argument";
    case MG_ERR_SIZE: return "unsupported size";
    case MG_ERR_CUDA: return "CUDA error";
    case MG_ERR_NOT_CONVERGED: return "not converged";
    case MG_ERR_NONFINITE: return "non-finite residual";
    case MG_ERR_TIMEOUT: return "device wait timed out";
    case MG_ERR_ALLOC: return "allocation failed";
    case MG_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char *mg_last_error(void) { return g_err; }

unsigned long long mg_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }


mg_status mg_setup_grid(mg_grid **out, int dim, const int64_t *n_intervals, const double *const *coords,
                        int precision_mask, void *stream) {
  (void)stream;
  if (!out || !n_intervals || !coords) return MG_ERR_INVALID_ARG;
  *out = nullptr;
  if (dim == 3) {
    for (int a = 0; a < 3; ++a) {
      if (n_intervals[a] < 2 || n_intervals[a] > 1020) return MG_ERR_SIZE;
      if (!coords[a]) return MG_ERR_INVALID_ARG;
      for (int64_t i = 0; i < n_intervals[a]; ++i)
        if (!(coords[a][i + 1] > coords[a][i])) return MG_ERR_SIZE;
    }
    mg_grid *g = new (std::nothrow) mg_grid();
    if (!g) return MG_ERR_ALLOC;
    g->prec_mask = (precision_mask & 3) ? (precision_mask & 3) : 3;
    mg_status st = setup3(*g, n_intervals, coords);
    if (st == MG_OK) st = setup_solver_state(g);
    if (st == MG_OK) st = cuda_status("3D setup (latched error)", cudaGetLastError());
    if (st != MG_OK) { free_grid(g); return st; }
    *out = g;
    return MG_OK;
  }
  if (dim != 2) return MG_ERR_INVALID_ARG;
  const int64_t nx = n_intervals[0], ny = n_intervals[1];
  if (nx < 2 || ny < 2 || nx > 32768 || ny > 32768) return MG_ERR_SIZE;
  if (!coords[0] || !coords[1]) return MG_ERR_INVALID_ARG;
  for (int64_t i = 0; i < nx; ++i)
    if (!(coords[0][i + 1] > coords[0][i])) return MG_ERR_SIZE;
  for (int64_t j = 0; j < ny; ++j)
    if (!(coords[1][j + 1] > coords[1][j])) return MG_ERR_SIZE;
  mg_grid *g = new (std::nothrow) mg_grid();
  if (!g) return MG_ERR_ALLOC;
  g->prec_mask = (precision_mask & 3) ? (precision_mask & 3) : 3;
  mg_status st = setup(g, (int)nx, (int)ny, coords[0], coords[1]);
  if (st != MG_OK) { free_grid(g); return st; }
  *out = g;
  return MG_OK;
}

void mg_destroy(mg_grid *g) { free_grid(g); }

int mg_num_levels(const mg_grid *g) { return g ? g->nlev : 0; }

mg_status mg_level_shape(const mg_grid *g, int level, int64_t *nx, int64_t *ny) {
  if (!g || !nx || !ny || level < 0 || level >= g->nlev) return MG_ERR_INVALID_ARG;
  if (g->dim == 3) {
    *nx = g->g3->lev[level].nx;
    *ny = g->g3->lev[level].ny;
    return MG_OK;
  }
  *nx = g->lev[level].nx;
  *ny = g->lev[level].ny;
  return MG_OK;
}

int mg_grid_dim(const mg_grid *g) { return g ? g->dim : 0; }

mg_status mg_level_dims(const mg_grid *g, int level, int64_t *dims) {
  if (!g || !dims || level < 0 || level >= g->nlev) return MG_ERR_INVALID_ARG;
  if (g->dim == 3) {
    const Level3 &L = g->g3->lev[level];
    dims[0] = L.nx; dims[1] = L.ny; dims[2] = L.nz;
  } else {
    dims[0] = g->lev[level].nx; dims[1] = g->lev[level].ny; dims[2] = 0;
  }
  return MG_OK;
}

static bool bad_level(const mg_grid *g, int level) { return !g || level < 0 || level >= g->nlev; }
static bool bad_dtype(const mg_grid *g, int dtype) {
  return !(dtype == MG_F64 && (g->prec_mask & 1)) && !(dtype == MG_F32 && (g->prec_mask & 2));
}

mg_status mg_colour_pass(mg_grid *g, int level, int smoother, int colour, void *u, const void *f, int dtype,
                         void *stream) {
  if (bad_level(g, level) || !u || !f || colour < 0 || colour > 1 || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  if (smoother == MG_SMOOTH_ALT_ZEBRA || smoother == MG_SMOOTH_ALT_TW || smoother < 0 || smoother > MG_SMOOTH_ALT_TW)
    return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (smoother != MG_SMOOTH_TWEED && smoother != MG_SMOOTH_WIREFRAME) return checked(MG_ERR_UNSUPPORTED);
    const int sm = smoother == MG_SMOOTH_WIREFRAME ? SM3_WIREFRAME : SM3_TWEED;
    if (dtype == MG_F64) return checked(colour_pass3<double>(*g, level, sm, colour, (double *)u, (const double *)f, s));
    return checked(colour_pass3<float>(*g, level, sm, colour, (float *)u, (const float *)f, s));
  }
  if (dtype == MG_F64) return checked(colour_pass<double>(*g, level, smoother, colour, (double *)u, (const double *)f, s));
  return checked(colour_pass<float>(*g, level, smoother, colour, (float *)u, (const float *)f, s));
}

mg_status mg_smooth(mg_grid *g, int level, int smoother, void *u, const void *f, int sweeps, int dtype,
                    void *stream) {
  if (bad_level(g, level) || !u || !f || sweeps < 0 || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  if (smoother < 0 || smoother > MG_SMOOTH_ALT_TW) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (smoother != MG_SMOOTH_TWEED && smoother != MG_SMOOTH_WIREFRAME && smoother != MG_SMOOTH_ALT_TW)
      return checked(MG_ERR_UNSUPPORTED);
    const int order[2] = {smoother == MG_SMOOTH_WIREFRAME ? MG_SMOOTH_WIREFRAME : MG_SMOOTH_TWEED,
                          smoother == MG_SMOOTH_ALT_TW ? MG_SMOOTH_WIREFRAME : -1};
    for (int k = 0; k < sweeps; ++k)
      for (int m = 0; m < 2 && order[m] >= 0; ++m)
        for (int c = 0; c < 2; ++c) {
          const mg_status st = mg_colour_pass(g, level, order[m], c, u, f, dtype, stream);
          if (st != MG_OK) return checked(st);
        }
    return checked(MG_OK);
  }
  for (int k = 0; k < sweeps; ++k) {
    mg_status st = dtype == MG_F64 ? smooth<double>(*g, level, smoother, (double *)u, (const double *)f, s)
                                   : smooth<float>(*g, level, smoother, (float *)u, (const float *)f, s);
    if (st != MG_OK) return checked(st);
  }
  return checked(MG_OK);
}

mg_status mg_smooth_tweed(mg_grid *g, int level, void *u, const void *f, int sweeps, int dtype, void *stream) {
  return mg_smooth(g, level, MG_SMOOTH_TWEED, u, f, sweeps, dtype, stream);
}

mg_status mg_smooth_wireframe(mg_grid *g, int level, void *u, const void *f, int sweeps, int dtype, void *stream) {
  return mg_smooth(g, level, MG_SMOOTH_WIREFRAME, u, f, sweeps, dtype, stream);
}

mg_status mg_residual_restrict(mg_grid *g, int level, int restriction, const void *u, const void *f, void *fc,
                               void *uc, int dtype, void *stream) {
  if (bad_level(g, level) || level + 1 >= g->nlev || !u || !f || !fc || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  if (restriction != MG_RESTRICT_HW && restriction != MG_RESTRICT_FW) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (restriction != MG_RESTRICT_FW) return checked(MG_ERR_UNSUPPORTED);
    if (dtype == MG_F64)
      return checked(residual_restrict3<double>(*g, level, (const double *)u, (const double *)f, (double *)fc, (double *)uc, s));
    return checked(residual_restrict3<float>(*g, level, (const float *)u, (const float *)f, (float *)fc, (float *)uc, s));
  }
  const Level &F = g->lev[level], &C = g->lev[level + 1];
  cudaError_t e = dtype == MG_F64
                      ? launch_residual_restrict<double>(F, C, restriction, (const double *)u, (const double *)f,
                                                         (double *)fc, (double *)uc, s)
                      : launch_residual_restrict<float>(F, C, restriction, (const float *)u, (const float *)f,
                                                        (float *)fc, (float *)uc, s);
  return checked(cuda_status("residual+restrict", e));
}

mg_status mg_prolong_add(mg_grid *g, int level, const void *uc, void *u, int dtype, void *stream) {
  if (bad_level(g, level) || level + 1 >= g->nlev || !u || !uc || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (dtype == MG_F64) return checked(prolong_add3<double>(*g, level, (const double *)uc, (double *)u, s));
    return checked(prolong_add3<float>(*g, level, (const float *)uc, (float *)u, s));
  }
  const Level &F = g->lev[level], &C = g->lev[level + 1];
  cudaError_t e = dtype == MG_F64 ? launch_prolong_add<double>(F, C, (const double *)uc, (double *)u, s)
                                  : launch_prolong_add<float>(F, C, (const float *)uc, (float *)u, s);
  return checked(cuda_status("prolong+correct", e));
}

mg_status mg_residual(mg_grid *g, int level, const void *u, const void *f, void *d, int dtype, void *stream) {
  if (bad_level(g, level) || !u || !f || !d || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (dtype == MG_F64) return checked(residual3<double>(*g, level, (const double *)u, (const double *)f, (double *)d, s));
    return checked(residual3<float>(*g, level, (const float *)u, (const float *)f, (float *)d, s));
  }
  const Level &L = g->lev[level];
  cudaError_t e = dtype == MG_F64 ? launch_residual<double>(L, (const double *)u, (const double *)f, (double *)d, s)
                                  : launch_residual<float>(L, (const float *)u, (const float *)f, (float *)d, s);
  return checked(cuda_status("residual", e));
}

mg_status mg_coarse_solve(mg_grid *g, void *u, const void *f, int dtype, void *stream) {
  if (!g || !u || !f || bad_dtype(g, dtype)) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (g->dim == 3) {
    if (dtype == MG_F64) return checked(coarse_solve3<double>(*g, (double *)u, (const double *)f, s));
    return checked(coarse_solve3<float>(*g, (float *)u, (const float *)f, s));
  }
  cudaError_t e = dtype == MG_F64 ? launch_coarse_solve<double>(*g, (double *)u, (const double *)f, s)
                                  : launch_coarse_solve<float>(*g, (float *)u, (const float *)f, s);
  return checked(cuda_status("coarse solve", e));
}

int mg_direct_level(const mg_grid *g) { return g && g->dim == 2 ? g->fd_level : -1; }

mg_status mg_direct_solve(mg_grid *g, void *u, const void *f, void *stream) {
  if (!g || !u || !f) return checked(MG_ERR_INVALID_ARG);
  if (g->dim != 2 || g->fd_level < 0) return checked(MG_ERR_UNSUPPORTED);
  return checked(cuda_status("direct level solve",
                     launch_direct_level(*g, (float *)u, (const float *)f, static_cast<cudaStream_t>(stream))));
}

mg_status mg_vcycle(mg_grid *g, void *u, const void *f, const mg_params *p, void *stream) {
  if (!g || !u || !f) return checked(MG_ERR_INVALID_ARG);
  mg_status st = check_params(g, p);
  if (st != MG_OK) return checked(st);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (p->precision == MG_PREC_F64) return checked(cycle_rec<double>(*g, *p, 0, (double *)u, (const double *)f, s));
  return checked(cycle_rec<float>(*g, *p, 0, (float *)u, (const float *)f, s));
}

mg_status mg_solve(mg_grid *g, double *u, const double *f, const mg_params *p, mg_info *info, void *stream) {
  if (!g || !u || !f) return checked(MG_ERR_INVALID_ARG);
  mg_status st = check_params(g, p);
  if (st != MG_OK) return checked(st);
  const auto t0 = std::chrono::steady_clock::now();
  st = solve_impl(*g, u, f, *p, info, static_cast<cudaStream_t>(stream));
  if (info) info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return checked(st);
}

mg_status mg_solve_adjoint(mg_grid *g, double *lambda, const double *rhs, const mg_params *p, mg_info *info,
                           void *stream) {
  if (!g || !lambda || !rhs) return checked(MG_ERR_INVALID_ARG);
  if (g->dim == 3) return checked(MG_ERR_UNSUPPORTED);
  mg_status st = check_params(g, p);
  if (st != MG_OK) return checked(st);
  if (!(g->prec_mask & 1)) return checked(MG_ERR_INVALID_ARG);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto t0 = std::chrono::steady_clock::now();
  if (!g->r64) return checked(MG_ERR_INVALID_ARG);  // allocated by mg_setup_grid with FP64 enabled
  // L^T = D L D^{-1} with D = diag(dx_i dy_j):  L mu = D^{-1} rhs, lambda = D mu
  cudaError_t e = launch_diag_scale(*g, g->r64, rhs, 1, s);
  if (e != cudaSuccess) return checked(cuda_status("adjoint scaling", e));
  mg_params q = *p;
  q.use_initial_guess = 0;
  e = launch_diag_scale(*g, lambda, lambda, 0, s);  // zero boundary (interior is reset by the solve)
  if (e != cudaSuccess) return checked(cuda_status("adjoint scaling", e));
  st = solve_impl(*g, lambda, g->r64, q, info, s);
  if (st != MG_OK && st != MG_ERR_NOT_CONVERGED) return checked(st);
  e = launch_diag_scale(*g, lambda, lambda, 0, s);
  if (e != cudaSuccess) return checked(cuda_status("adjoint scaling", e));
  if (info) info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return checked(st);
}

mg_status mg_boundary_adjoint(mg_grid *g, const double *lambda, const double *grad_u, double *grad_g,
                              void *stream) {
  if (!g || !lambda || !grad_u || !grad_g) return checked(MG_ERR_INVALID_ARG);
  if (g->dim == 3) return checked(MG_ERR_UNSUPPORTED);
  cudaError_t e = launch_boundary_adjoint(*g, lambda, grad_u, grad_g, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return checked(cuda_status("boundary adjoint", e));
  return checked(MG_OK);
}

mg_status mg_pass_timer_begin(mg_grid *g, int level, int max_passes) {
  if (bad_level(g, level) || max_passes < 1 || max_passes > (1 << 20) || g->timer_ev) return MG_ERR_INVALID_ARG;
  if (g->dim == 3) return MG_ERR_UNSUPPORTED;
  g->timer_ev = new (std::nothrow) cudaEvent_t[4 * (size_t)max_passes];
  if (!g->timer_ev) return MG_ERR_ALLOC;
  for (int k = 0; k < 4 * max_passes; ++k) {
    cudaError_t e = cudaEventCreate(&g->timer_ev[k]);
    if (e != cudaSuccess) {
      g->timer_cap = k / 4;
      for (int j = 4 * g->timer_cap; j < k; ++j) cudaEventDestroy(g->timer_ev[j]);
      destroy_timer(g);
      return cuda_status("cudaEventCreate(pass timer)", e);
    }
  }
  g->timer_cap = max_passes;
  g->timer_n = 0;
  g->timer_level = level;
  return MG_OK;
}

mg_status mg_pass_timer_end(mg_grid *g, int64_t *passes, double *stage_ms, double *pass_min_ms,
                            double *pass_max_ms) {
  if (!g || !g->timer_ev) return MG_ERR_INVALID_ARG;
  const int n = g->timer_n;
  double st[3] = {0.0, 0.0, 0.0}, mn = 0.0, mx = 0.0;
  mg_status rc = MG_OK;
  if (n > 0) {
    cudaError_t e = cudaEventSynchronize(g->timer_ev[4 * n - 1]);
    for (int p = 0; p < n && e == cudaSuccess; ++p) {
      double tot = 0.0;
      for (int k = 0; k < 3 && e == cudaSuccess; ++k) {
        float ms = 0.0f;
        e = cudaEventElapsedTime(&ms, g->timer_ev[4 * p + k], g->timer_ev[4 * p + k + 1]);
        st[k] += ms;
        tot += ms;
      }
      mn = p == 0 ? tot : std::min(mn, tot);
      mx = std::max(mx, tot);
    }
    if (e != cudaSuccess) rc = cuda_status("pass timer", e);
  }
  if (passes) *passes = n;
  if (stage_ms) for (int k = 0; k < 3; ++k) stage_ms[k] = st[k];
  if (pass_min_ms) *pass_min_ms = mn;
  if (pass_max_ms) *pass_max_ms = mx;
  destroy_timer(g);
  return rc;
}

}  // extern "C"
