// packed.h -- per-problem kernel arguments for packed launches.  A packed
// launch serves a group of problems whose grids have the same shape (so the
// same blocks and work lists on every level): blockIdx.y or blockIdx.z (the
// launcher says which) selects problem q, whose arguments are tab[q]; a
// problem whose active[q] is 0 does nothing.  The arithmetic of each problem
// is exactly that of its unpacked launch.
#pragma once
#include "device_util.cuh"

namespace tmg {

template <typename T>
struct PassArgs {  // colour pass
  Coefs<T> c;
  T *u;
  const T *f;
};
template <typename T>
struct RRArgs {  // defect + restriction, fine level -> next level
  Coefs<T> c;
  const T *u, *f;
  T *fc, *uc;
};
template <typename T>
struct ProlongArgs {  // prolongation + correction
  const T *uc;
  T *u;
};
template <typename T>
struct CoarseArgs {  // direct solve of the coarsest level
  Coefs<double> c;
  const double *inv;
  T *u;
  const T *f;
};
struct NormArgs {  // FP64 norms (and refinement residual) of the finest level
  Coefs<double> c;
  const double *we;  // W_i + E_i per column
  const double *u, *f;
  double *part, *out;
  float *r32, *e32;  // the first refinement step of a zeroed guess (launch_norms_packed with_r32)
};
struct RefineArgs {  // refinement residual with the update fused (transfer.cu)
  Coefs<double> c;
  const double *cd;  // W_i + E_i + S_j + N_j per node (Grid::cd64)
  double *ua, *ub;   // the two FP64 iterates: read one, write the other
  const float *e;    // FP32 correction (NULL: residual of the iterate alone)
  const double *f;
  float *r32, *e32;
  double *part, *out;
};
struct UpdateArgs {  // u64 interior := 0 (e unused)
  double *u;
  const float *e;
};

// Host view of one packed launch: device tables, device active flags and the
// number of problems.
struct PackedLaunch {
  const void *tab;
  const int *active;
  int count;
};

// Packed launchers (the kernels' own translation units).
template <typename T>
cudaError_t launch_warp_pass_packed(const Level &L, const WarpList &w, const PackedLaunch &pk, cudaStream_t s);
template <typename T>
cudaError_t launch_residual_restrict_packed(const Level &F, const Level &C, int kind, const PackedLaunch &pk,
                                            cudaStream_t s);
template <typename T>
cudaError_t launch_prolong_add_packed(const Level &F, const Level &C, const PackedLaunch &pk, cudaStream_t s);
template <typename T>
cudaError_t launch_coarse_solve_packed(const Grid &g, const PackedLaunch &pk, cudaStream_t s);
// norms: bnd_only as launch_rhsnorm64; with_r32: the refinement residual
cudaError_t launch_norms_packed(const Grid &g, int bnd_only, const PackedLaunch &pk, cudaStream_t s,
                                bool with_r32 = false);
// The refinement residual of every active member (update: the FP32
// correction added first; active flag 1 reads ua and writes ub, 2 the
// reverse), its r32 and FP64 norm; then each member's e32 zeroed.
cudaError_t launch_refine_residual_packed(const Grid &g, bool update, const PackedLaunch &pk,
                                          float *const *e32s, cudaStream_t s);
cudaError_t launch_zero_interior_packed(const Grid &g, const PackedLaunch &pk, cudaStream_t s);

}  // namespace tmg
