// tune.cu -- choice of the line-solve path per level (mg_set_line_path,
// mg_get_line_path) and the autotuner that times the candidates
// (mg_autotune).  Every path solves every block exactly; only the layout of
// the work on the GPU differs.
#include <array>
#include <map>
#include <mutex>
#include <vector>

#include "mg_internal.h"

namespace tmg {
namespace {

bool has_tiles(const Level &L, int wl) {
  for (int c = 0; c < 2; ++c)
    if (L.tl[wl][c].ntile == 0 && L.tl[wl][c].nblock == 0) return false;
  return true;
}

bool has_cluster(const Level &L, int wl) { return L.cp[wl][0].ncta > 0 && L.cp[wl][1].ncta > 0; }

// Sets the path of (level, wl, prec); the caller has validated the arguments.
mg_status set_path(Grid &g, int level, int wl, int prec, int path, int k) {
  Level &L = g.lev[level];
  mg_status st = build_worklists(g, level, wl, prec);
  if (st != MG_OK) return st;
  if (path == MG_PATH_TILED && !has_tiles(L, wl)) return MG_ERR_UNSUPPORTED;
  if (path == MG_PATH_CLUSTER && (prec != 1 || !has_cluster(L, wl))) return MG_ERR_UNSUPPORTED;
  // the warp lists are rebuilt for the warp path, and back to the built-in
  // ones when leaving a warp path with another shape
  const bool rebuild = path == MG_PATH_WARP || L.kpref[wl][prec] != 0;
  if (rebuild) {
    WarpList fresh[2];
    const bool auto_rule = path != MG_PATH_WARP;
    if (!auto_rule || (L.nx < WARP_MAX_SIDE && L.ny < WARP_MAX_SIDE)) {
      st = build_warp_path(g, level, wl, prec, auto_rule ? 0 : k, fresh);
      if (st == MG_OK && !auto_rule && (fresh[0].nwarp == 0 || fresh[1].nwarp == 0)) st = MG_ERR_UNSUPPORTED;
      if (st != MG_OK) {
        free_warplist(fresh[0]);
        free_warplist(fresh[1]);
        return st;
      }
    }
    // kernels or graphs may still read the old lists
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("cudaDeviceSynchronize (line path)", e);
      free_warplist(fresh[0]);
      free_warplist(fresh[1]);
      return MG_ERR_CUDA;
    }
    for (int c = 0; c < 2; ++c) {
      free_warplist(L.wp[wl][prec][c]);
      L.wp[wl][prec][c] = fresh[c];
    }
  } else {
    const cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      set_error("cudaDeviceSynchronize (line path)", e);
      return MG_ERR_CUDA;
    }
  }
  L.path[wl][prec] = path;
  L.kpref[wl][prec] = path == MG_PATH_WARP ? (k > 0 ? k : WK_PREF) : 0;
  ++g.gen;
  drop_graphs(g);
  return MG_OK;
}

// The path colour 0 of (level, wl, prec) takes now.
int resolved(const Level &L, int wl, int prec) {
  const int p = L.path[wl][prec];
  if (p != MG_PATH_AUTO) return p;
  if (L.wp[wl][prec][0].nwarp > 0) return MG_PATH_WARP;
  const TileList &t = L.tl[wl][0];
  return (t.ntile > 0 || t.nblock > 0) ? MG_PATH_TILED : MG_PATH_CTA;
}

// Remembered choices: (nx, ny, wl, prec) -> (path, k, microseconds per pass).
struct Choice {
  int path, k;
  double us;
};
std::mutex g_tune_mu;
std::map<std::array<int, 4>, Choice> g_tuned;

}  // namespace
}  // namespace tmg

using namespace tmg;

namespace {

bool bad_args(const mg_grid *g, int level, int dtype) {
  if (!g || g->dim != 2 || level < 0 || level >= g->nlev) return true;
  return !(dtype == MG_F64 && (g->prec_mask & 1)) && !(dtype == MG_F32 && (g->prec_mask & 2));
}

// Average milliseconds per colour pass of `reps` passes (after 2 untimed).
mg_status time_passes(mg_grid *g, int level, int smoother, int dtype, int reps, void *u, const void *f,
                      cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double *ms) {
  for (int r = 0; r < 2; ++r) {
    const mg_status st = mg_colour_pass(g, level, smoother, r & 1, u, f, dtype, s);
    if (st != MG_OK) return st;
  }
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) {
    const mg_status st = mg_colour_pass(g, level, smoother, r & 1, u, f, dtype, s);
    if (st != MG_OK) return st;
  }
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e != cudaSuccess) {
    set_error("autotune timing", e);
    return MG_ERR_CUDA;
  }
  *ms = (double)t / reps;
  return MG_OK;
}

}  // namespace

extern "C" {

// 3D grids: tweed passes take the warp path or the 3D tiled path (both
// precisions alike); wireframe passes have the warp path alone.
static mg_status set_path3(mg_grid *g, int level, int smoother, int path) {
  if (level < 0 || level + 1 >= g->nlev || !(path == MG_PATH_AUTO || path == MG_PATH_WARP || path == MG_PATH_TILED))
    return MG_ERR_INVALID_ARG;
  if (smoother != MG_SMOOTH_TWEED) return smoother == MG_SMOOTH_WIREFRAME ? MG_ERR_UNSUPPORTED : MG_ERR_INVALID_ARG;
  Level3 &L = g->g3->lev[level];
  if (path == MG_PATH_TILED && !L.t3_ok) return MG_ERR_UNSUPPORTED;
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    set_error("cudaDeviceSynchronize (line path)", e);
    return MG_ERR_CUDA;
  }
  L.t3_path = path == MG_PATH_AUTO ? 0 : path == MG_PATH_WARP ? 1 : 2;
  ++g->gen;
  drop_graphs(*g);
  return MG_OK;
}

mg_status mg_set_line_path(mg_grid *g, int level, int smoother, int dtype, int path, int k) {
  if (g && g->dim == 3) return set_path3(g, level, smoother, path);
  if (bad_args(g, level, dtype) || path < MG_PATH_AUTO || path > MG_PATH_CLUSTER) return MG_ERR_INVALID_ARG;
  if (!(k == 0 || k == 1 || k == 2 || k == 4 || k == 8 || k == 16)) return MG_ERR_INVALID_ARG;
  const int wl = wl_of(smoother);
  if (wl < 0) return MG_ERR_INVALID_ARG;
  return set_path(*g, level, wl, dtype == MG_F64 ? 0 : 1, path, k);
}

mg_status mg_get_line_path(const mg_grid *g, int level, int smoother, int dtype, int *path, int *k, int *w) {
  if (g && g->dim == 3) {
    if (level < 0 || level + 1 >= g->nlev || (smoother != MG_SMOOTH_TWEED && smoother != MG_SMOOTH_WIREFRAME))
      return MG_ERR_INVALID_ARG;
    const Level3 &L = g->g3->lev[level];
    const bool tiled = smoother == MG_SMOOTH_TWEED && tiled3(L);
    const WarpList3 &wp = L.wp[smoother == MG_SMOOTH_TWEED ? SM3_TWEED : SM3_WIREFRAME][0];
    if (path) *path = tiled ? MG_PATH_TILED : MG_PATH_WARP;
    if (k) *k = tiled ? 0 : wp.K;
    if (w) *w = tiled ? 0 : wp.W;
    return MG_OK;
  }
  if (bad_args(g, level, dtype)) return MG_ERR_INVALID_ARG;
  const int wl = wl_of(smoother);
  if (wl < 0) return MG_ERR_INVALID_ARG;
  const int prec = dtype == MG_F64 ? 0 : 1;
  const Level &L = g->lev[level];
  const int p = resolved(L, wl, prec);
  const WarpList &wp = L.wp[wl][prec][0];
  if (path) *path = p;
  if (k) *k = p == MG_PATH_WARP ? wp.K : 0;
  if (w) *w = p == MG_PATH_WARP ? wp.W : 0;
  return MG_OK;
}

mg_status mg_autotune(mg_grid *g, int smoother, int dtype, int reps, double *times_us, void *stream) {
  if (bad_args(g, 0, dtype) || smoother < MG_SMOOTH_CHECKERBOARD || smoother > MG_SMOOTH_ALT_TW)
    return MG_ERR_INVALID_ARG;
  if (times_us)
    for (int l = 0; l < g->nlev; ++l) times_us[l] = 0.0;
  std::vector<int> smoothers;
  if (smoother == MG_SMOOTH_ALT_ZEBRA) smoothers = {MG_SMOOTH_ZEBRA_X, MG_SMOOTH_ZEBRA_Y};
  else if (smoother == MG_SMOOTH_ALT_TW) smoothers = {MG_SMOOTH_TWEED, MG_SMOOTH_WIREFRAME};
  else if (smoother != MG_SMOOTH_CHECKERBOARD) smoothers = {smoother};
  if (smoothers.empty()) return MG_OK;
  const int prec = dtype == MG_F64 ? 0 : 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t esz = dtype == MG_F64 ? sizeof(double) : sizeof(float);
  void *u = nullptr, *f = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  mg_status st = MG_OK;
  auto fail = [&](const char *where, cudaError_t e) {
    set_error(where, e);
    st = e == cudaErrorMemoryAllocation ? MG_ERR_ALLOC : MG_ERR_CUDA;
  };
  if (reps > 0) {
    const size_t bytes = esz * g->lev[0].nn;
    cudaError_t e = cudaMalloc(&u, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&f, bytes);
    if (e == cudaSuccess) e = cudaMemsetAsync(u, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, bytes, s);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) fail("autotune scratch", e);
  }
  for (size_t si = 0; si < smoothers.size() && st == MG_OK; ++si) {
    const int sm = smoothers[si], wl = wl_of(sm);
    for (int l = 0; l + 1 < g->nlev && st == MG_OK; ++l) {
      const Level &L = g->lev[l];
      const std::array<int, 4> key = {L.nx, L.ny, wl, prec};
      Choice known{-1, 0, 0.0};
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) known = it->second;
      }
      if (known.path >= 0) {
        st = set_path(*g, l, wl, prec, known.path, known.k);
        if (st == MG_OK && times_us) times_us[l] += known.us;
        continue;
      }
      if (reps <= 0) continue;
      // candidates: the warp path with each preferred k (distinct shapes
      // only), the cluster path, the tiled path, the CTA path
      Choice best{-1, 0, 0.0};
      std::vector<std::array<int, 2>> shapes;
      const int cand[8][2] = {{MG_PATH_WARP, 1}, {MG_PATH_WARP, 2}, {MG_PATH_WARP, 4}, {MG_PATH_WARP, 8},
                              {MG_PATH_WARP, 16}, {MG_PATH_CLUSTER, 0}, {MG_PATH_TILED, 0}, {MG_PATH_CTA, 0}};
      for (int c = 0; c < 8 && st == MG_OK; ++c) {
        const mg_status ps = set_path(*g, l, wl, prec, cand[c][0], cand[c][1]);
        if (ps == MG_ERR_UNSUPPORTED) continue;
        if (ps != MG_OK) { st = ps; break; }
        if (cand[c][0] == MG_PATH_WARP) {
          const std::array<int, 2> shape = {L.wp[wl][prec][0].K * 64 + L.wp[wl][prec][0].W,
                                            L.wp[wl][prec][1].K * 64 + L.wp[wl][prec][1].W};
          bool seen = false;
          for (auto &x : shapes) seen |= x == shape;
          if (seen) continue;
          shapes.push_back(shape);
        }
        double ms = 0.0;
        st = time_passes(g, l, sm, dtype, reps, u, f, s, e0, e1, &ms);
        if (st == MG_OK && (best.path < 0 || 1e3 * ms < best.us)) best = {cand[c][0], cand[c][1], 1e3 * ms};
      }
      if (st != MG_OK) break;
      st = set_path(*g, l, wl, prec, best.path, best.k);
      if (st != MG_OK) break;
      if (times_us) times_us[l] += best.us;
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tuned[key] = best;
    }
  }
  const cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess && st == MG_OK) fail("autotune", e);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(u);
  cudaFree(f);
  return st;
}

}  // extern "C"
