// mg_internal.h -- data layout shared by the host driver and the sm_103a
// kernels of tweedmg (not part of the public ABI; see include/mg.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/mg.h"

namespace tmg {

// ---------------------------------------------------------------------------
// Directions.  A "direction" d names the neighbour one step away:
//   0 = +x (coefficient E_i), 1 = -x (W_i), 2 = +y (N_j), 3 = -y (S_j);
// the opposite direction is d ^ 1.
// ---------------------------------------------------------------------------
enum { DIR_PX = 0, DIR_MX = 1, DIR_PY = 2, DIR_MY = 3 };

// Flag byte of a segment / chunk descriptor.
//   bits 0-1  dir       direction of travel along the run
//   bits 2-3  nextdir   direction from the run's last node to whatever follows
//                       it (the next run of the chain, or the junction)
//   bit  4    LP        the first node's predecessor (one step against dir)
//                       is an unknown of the same chain
//   bit  5    LN        the last node's successor (one step along nextdir) is
//                       an unknown of the same chain
//   bit  6    FJ        the first node is coupled to the block's junction,
//                       which sits one step against dir
//   bit  7    LJ        the last node is coupled to the junction, which sits
//                       one step along nextdir
enum : uint8_t { F_LP = 16, F_LN = 32, F_FJ = 64, F_LJ = 128 };

// A run of <= 32 consecutive chain nodes along one direction, solved by one
// thread.  Chunk c of a CTA owns the shared-memory slots [32c, 32c+32) (node q
// of the chunk in slot 32c + q).  Consecutive chunks of a chain are
// consecutive in the CTA's chunk list, so the reduced-system neighbours of
// chunk t are chunks t-1 (if LP) and t+1 (if LN).  junc = CTA-local index of
// the chain's junction, or 0xFFFF.
struct ChunkDesc {
  uint16_t i0, j0;
  uint8_t len, flags;
  uint16_t junc;
  uint16_t pad[4];
};
static_assert(sizeof(ChunkDesc) == 16, "ChunkDesc layout");

// A junction node: the branch point of a tweed star (Eq. mLThomas), the node
// where a wireframe ring is closed (Eq. CircTri), or a lone point block.
// row[e] = reduced-system row of the chain end attached to it; bits 2e..2e+1
// of dirs = direction from the junction to that chain end.
struct JuncDesc {
  uint16_t i, j;
  uint16_t row[4];
  uint8_t dirs, nend;
  uint8_t pad[2];
};
static_assert(sizeof(JuncDesc) == 16, "JuncDesc layout");

// Work of one CTA: whole blocks only (a block never spans two CTAs).
struct CtaWork {
  int chunk0, nchunk;
  int junc0, njunc;
  int nnode;  // unknowns of the CTA's chains (junctions excluded)
  int pad[3];
};
static_assert(sizeof(CtaWork) == 32, "CtaWork layout");

// Device-resident work list of one (level, smoother, colour, CTA shape).
struct WorkList {
  int ncta = 0;
  int nt = 0;           // threads per CTA = max chunks per CTA
  int total_nodes = 0;  // unknowns relaxed by this list (junctions included)
  void *mem = nullptr;  // one allocation behind the three arrays
  CtaWork *cta = nullptr;
  ChunkDesc *chunk = nullptr;
  JuncDesc *junc = nullptr;
};

// Shapes of the line-solve kernel: 32 nodes per chunk (one thread each);
// blocks of up to NT_SMALL*32 unknowns go to CTAs of NT_SMALL threads (two
// resident per SM), larger ones (wireframe rings) to CTAs of NT_LARGE.
constexpr int CMAX = 32;
constexpr int NT_SMALL = 256, NT_LARGE = 512;
constexpr int MAX_BLOCK_NODES = NT_LARGE * CMAX;

// Base smoothers that use line work lists.
enum { WL_ZEBRA_X = 0, WL_ZEBRA_Y = 1, WL_TWEED = 2, WL_WIREFRAME = 3, WL_COUNT = 4 };

struct Level {
  int nx = 0, ny = 0;
  size_t nn = 0;                     // (nx+1)*(ny+1)
  std::vector<double> hx, hy;        // host coordinates
  std::vector<double> hW, hE, hS, hN;
  double *W64 = nullptr, *E64 = nullptr, *S64 = nullptr, *N64 = nullptr;
  float *W32 = nullptr, *E32 = nullptr, *S32 = nullptr, *N32 = nullptr;
  double *xd = nullptr, *yd = nullptr;  // device copies of the coordinates
  void *dev_block = nullptr;            // one allocation behind the arrays above
  // workspaces of coarse levels (level 0 uses the caller's arrays)
  double *u64 = nullptr, *f64 = nullptr;
  float *u32 = nullptr, *f32 = nullptr;
  bool wl_built[WL_COUNT][2] = {};    // [smoother][precision 0=f64,1=f32]
  WorkList wl[WL_COUNT][2][2][2];     // [smoother][precision][colour][small, large]
};

struct Grid {
  int nlev = 0;
  int prec_mask = 3;
  std::vector<Level> lev;
  // coarsest level: dense inverse of the interior operator (FP64, row-major)
  int cn = 0;
  double *cinv = nullptr;
  // finest-level FP64/FP32 scratch for the refinement loop and norms
  double *r64 = nullptr;             // residual / scaled rhs scratch (finest)
  double *lam_tmp = nullptr;         // adjoint scratch (finest)
  float *e32 = nullptr, *r32 = nullptr;
  double *partial = nullptr;         // per-CTA partial sums (deterministic norm)
  double *hpinned = nullptr;         // pinned host mirror of the norm results
  int npartial = 0;
  double *scal = nullptr;            // device scalars (reduced norms)
};

// Kernels launched by this library in this process (mg_kernel_launches).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---- host helpers (setup.cu)
mg_status build_worklists(Grid &g, int level, int wl, int prec);
const char *set_error(const char *where, cudaError_t e);
void set_error_text(const char *msg);

// ---- kernel launchers (smooth.cu, transfer.cu).  All return cudaError_t of
// the launch (cudaGetLastError).
template <typename T>
cudaError_t launch_line_pass(const Level &L, const WorkList &w, T *u, const T *f, cudaStream_t s);
template <typename T>
cudaError_t launch_checker_pass(const Level &L, int colour, T *u, const T *f, cudaStream_t s);
template <typename T>
cudaError_t launch_residual(const Level &L, const T *u, const T *f, T *d, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_restrict(const Level &F, const Level &C, int kind, const T *u, const T *f,
                                     T *fc, T *uc, cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add(const Level &F, const Level &C, const T *uc, T *u, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve(const Grid &g, T *u, const T *f, cudaStream_t s);

// FP64 norms: out[0] = sum (f-Lu)^2 over interior, out[1] = max |f-Lu|,
// written to the device scalars g.scal[0..1] (u may be NULL: residual = f).
cudaError_t launch_resnorm64(const Grid &g, const double *u, const double *f, cudaStream_t s);
// Refinement: r32 = float(f - L u64) and the FP64 norms of f - L u64 into scal.
cudaError_t launch_ir_residual(const Grid &g, const double *u, const double *f, float *r32,
                               cudaStream_t s);
// u64 += e32 on interior nodes.
cudaError_t launch_ir_update(const Grid &g, double *u, const float *e, cudaStream_t s);
// a[interior] *= scale_x[i]*scale_y[j] (adjoint diagonal scalings), boundary := 0.
cudaError_t launch_diag_scale(const Grid &g, double *out, const double *in, int inverse,
                              cudaStream_t s);
// Zero the interior (and optionally boundary) of a level array.
template <typename T>
cudaError_t launch_zero_interior(const Level &L, T *a, cudaStream_t s);

}  // namespace tmg
