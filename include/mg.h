/*
 * mg.h -- C ABI of tweedmg, a GB300 (sm_103a) geometric multigrid library for
 * the Dirichlet Poisson problem on stretched rectilinear grids, with the tweed
 * and wireframe smoothers of Bewley, Mashayek, Cavaglieri & Luchini,
 * "Tweed and wireframe: accelerated relaxation algorithms for multigrid
 * solution of elliptic PDEs on stretched structured grids" (arXiv:2110.08389).
 *
 * Problem (Sec. 2, Eq. prob:DP): on an (nx+1) x (ny+1) grid with coordinates
 * x_0 < ... < x_nx and y_0 < ... < y_ny, find u with
 *     W_i u_{i-1,j} + E_i u_{i+1,j} + S_j u_{i,j-1} + N_j u_{i,j+1} + C_ij u_ij = f_ij
 * at every interior node (0 < i < nx, 0 < j < ny), u given on the boundary,
 * where W_i = 1/(dx_i dx_{i-1/2}), E_i = 1/(dx_i dx_{i+1/2}) (same for S_j,
 * N_j in y), dx_{i-1/2} = x_i - x_{i-1}, dx_i = (x_{i+1} - x_{i-1})/2 and
 * C_ij = -(W_i + E_i + S_j + N_j).
 *
 * Conventions for every entry point:
 *   - Grid arrays (u, f, corrections) are dense, row-major, x fastest:
 *     element (i,j) of a level with nx, ny intervals is at a[j*(nx+1)+i].
 *     They are DEVICE pointers owned by the caller, 8-byte (double) or 4-byte
 *     (float) aligned, and must not alias each other.
 *   - u carries the Dirichlet data on its boundary nodes; kernels write only
 *     interior nodes.  f is read only at interior nodes.
 *   - Level 0 is the finest grid (the paper's Omega_p); level l+1 drops every
 *     other grid line of level l (Sec. 4).  Coarsening stops when a side is
 *     odd, a side would fall below 2 intervals, or max(nx,ny) <= 8; the
 *     coarsest level is solved directly.
 *   - All work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  Only mg_setup_grid, mg_solve, mg_solve_adjoint, mg_batch_solve,
 *     mg_set_line_path and mg_autotune synchronise (the solves read residual
 *     norms back to the host).  No entry point allocates device memory except
 *     mg_setup_grid, mg_batch_create, mg_set_line_path and mg_autotune.
 *   - Errors are returned as mg_status; nothing aborts or traps.  After
 *     MG_ERR_CUDA the message of the failing call is available from
 *     mg_last_error().  Calls on one grid must not run concurrently.
 */
#ifndef TWEEDMG_MG_H
#define TWEEDMG_MG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mg_grid mg_grid; /* opaque: level hierarchy, coefficients,
                                   block work lists and workspaces */

typedef enum {
  MG_OK = 0,
  MG_ERR_INVALID_ARG = 1,   /* NULL pointer, bad enum, bad level, ...           */
  MG_ERR_SIZE = 2,          /* nx, ny < 2, coordinates not increasing, a block  */
                            /* longer than the kernels support (16384 nodes)    */
  MG_ERR_CUDA = 3,          /* a CUDA runtime call failed (see mg_last_error)   */
  MG_ERR_NOT_CONVERGED = 4, /* tolerance not reached within the cycle cap, or  */
                            /* the defect grew 1e3-fold (info is still filled)  */
  MG_ERR_NONFINITE = 5,     /* a residual norm was NaN or infinite              */
  MG_ERR_TIMEOUT = 6,       /* reserved for bounded device-side waits           */
  MG_ERR_ALLOC = 7,         /* device or host allocation failed                 */
  MG_ERR_UNSUPPORTED = 8    /* valid request this library does not implement    */
} mg_status;

/* Smoothers (Sec. 2 and Sec. 3).  One "relaxation" of each is a red pass then
 * a black pass; the alternating schemes apply one step of each of their two
 * smoothers per relaxation.                                                   */
typedef enum {
  MG_SMOOTH_CHECKERBOARD = 0, /* red-black point Gauss-Seidel, red = (i+j) even */
  MG_SMOOTH_ZEBRA_X = 1,      /* lines along x, red = odd j                     */
  MG_SMOOTH_ZEBRA_Y = 2,      /* lines along y, red = odd i                     */
  MG_SMOOTH_ALT_ZEBRA = 3,    /* zebra x step, then zebra y step                */
  MG_SMOOTH_TWEED = 4,        /* branched lines, blocks = level sets of         */
                              /* max(dist to x-walls, dist to y-walls), Sec. 3  */
  MG_SMOOTH_WIREFRAME = 5,    /* concentric rings, level sets of the min, Sec. 3*/
  MG_SMOOTH_ALT_TW = 6        /* tweed step, then wireframe step                */
} mg_smoother;

typedef enum { MG_F64 = 0, MG_F32 = 1 } mg_dtype;
typedef enum { MG_PREC_F64 = 0, MG_PREC_F32_REFINE = 1 } mg_precision;
typedef enum { MG_CYCLE_V = 1, MG_CYCLE_W = 2 } mg_cycle;
typedef enum { MG_RESTRICT_HW = 0, MG_RESTRICT_FW = 1 } mg_restriction;

/* Solver parameters (Sec. 4).  mg_default_params() fills the defaults:
 * tweed, V(2,2), full weighting, FP64, tol 1e-10, 100 cycles, 8 outer
 * iterations, 3 inner cycles, zero initial guess, no early stop.             */
typedef struct {
  int smoother;          /* mg_smoother                                          */
  int nu1, nu2;          /* pre- / post-smoothing relaxations (>= 0)             */
  int cycle;             /* mg_cycle: 1 = V, 2 = W                               */
  int restriction;       /* mg_restriction (prolongation is always bilinear)     */
  int precision;         /* mg_precision                                         */
  int max_cycles;        /* cap on cycles (FP64) or on inner cycles (FP32+refine:*/
                         /* checked after each refinement step, which runs all  */
                         /* inner_cycles, so the count can end up to            */
                         /* inner_cycles - 1 past the cap)                       */
  int max_outer;         /* cap on refinement iterations (FP32+refine)           */
  int inner_cycles;      /* FP32 cycles per refinement iteration (default 3)     */
  int use_initial_guess; /* 0: interior of u is zeroed first; 1: u is the guess  */
  int early_stop;        /* 1: give up (MG_ERR_NOT_CONVERGED) once, from the 3rd */
                         /* cycle (FP64) or refinement iteration on, the last    */
                         /* step's reduction, kept for the steps left under the  */
                         /* caps, cannot reach tol (or the step did not reduce)  */
  int coarse_direct;     /* 1: the FP32 cycles solve the level mg_direct_level() */
                         /* names exactly (one kernel) instead of cycling below  */
                         /* it; FP64 cycles are not affected (default 0)         */
  double tol;            /* stop when ||f - L u||_2 / ||f||_2 <= tol (interior)   */
} mg_params;

/* Convergence record.  history is a caller-owned HOST buffer of history_cap
 * doubles (may be NULL): history[k] = ||f - L u||_2/||f||_2 after cycle k
 * (FP64) or after refinement iteration k (FP32+refine); history[0] is the
 * initial value.                                                             */
typedef struct {
  int cycles;            /* V/W cycles run (all precisions)                      */
  int outer_iters;       /* refinement iterations (FP32+refine), else 0          */
  double rel_res;        /* final ||f - L u||_2 / ||f||_2                         */
  double conv_factor;    /* (rho_K / rho_0)^(1/K) over the recorded history       */
  double ms;             /* wall time of the call, milliseconds                   */
  double *history;
  int history_cap;
  int history_len;
} mg_info;

/* Build the level hierarchy, the 1-D coefficient arrays of Sec. 2 on every
 * level (rediscretised on the subsampled coordinates, Sec. 4) and the device
 * workspaces.  dim 2: n_intervals = {nx, ny}; coords = {x, y}, HOST arrays of
 * nx+1 and ny+1 strictly increasing doubles (copied).
 * dim 3 (Sec. 7): n_intervals = {nx, ny, nz} (each 2 .. 1020), coords =
 * {x, y, z}; grid arrays are [nz+1][ny+1][nx+1], x fastest, and the operator
 * is the 7-point one with B_k, T_k over z built like S_j, N_j.  3D grids
 * offer the tweed smoother (blocks: the level sets of the two larger sorted
 * wall distances, lines perpendicular to the nearest wall, stars of up to six
 * legs), the wireframe smoother (level sets of the two smaller ones: rings on
 * the faces of concentric cuboids and each cuboid's twelve-edge skeleton),
 * both alternating (MG_SMOOTH_ALT_TW), full weighting and trilinear
 * prolongation (tensor products of the 1D factors of Sec. 4),
 * mg_colour_pass, mg_smooth(_tweed, _wireframe), mg_residual,
 * mg_residual_restrict, mg_prolong_add, mg_coarse_solve, mg_vcycle and
 * mg_solve in both precisions; other smoothers and the other entry points
 * return MG_ERR_UNSUPPORTED.  Sides that are odd on a smoothed level are
 * MG_ERR_UNSUPPORTED (their middle blocks would close loops).
 * precision_mask: bit 0 = FP64 workspaces, bit 1 = FP32 workspaces (0 means
 * both).  The block work lists of every smoother are built here too, and
 * with FP32 workspaces the part of the tiled line solves that only the
 * coefficients fix (the pivots of the reduced system each leg's 32-node
 * chunks form), which runs kernels on the device and waits for them.
 * On success *out owns device memory until mg_destroy.                       */
mg_status mg_setup_grid(mg_grid **out, int dim, const int64_t *n_intervals,
                        const double *const *coords, int precision_mask, void *stream);

/* Release everything owned by the grid (NULL is a no-op).                    */
void mg_destroy(mg_grid *grid);

/* Number of levels and the interval counts of one level (mg_level_shape:
 * nx, ny of either dimension; mg_level_dims: {nx, ny, nz}, nz = 0 in 2D) and
 * the grid's dimension (2 or 3).                                             */
int mg_num_levels(const mg_grid *grid);
mg_status mg_level_shape(const mg_grid *grid, int level, int64_t *nx, int64_t *ny);
mg_status mg_level_dims(const mg_grid *grid, int level, int64_t *dims);
int mg_grid_dim(const mg_grid *grid);

/* Relaxation on one level.  u, f: device arrays of that level's shape in
 * dtype (mg_dtype).  `sweeps` relaxations are applied in place on u.
 *   mg_smooth_tweed:     Sec. 3 tweed relaxation: each block (corner points,
 *                        L-shaped two-legged blocks, the centre cross or the two
 *                        T-blocks, straight lines in the middle of a
 *                        rectangle) is solved exactly, red blocks first.
 *   mg_smooth_wireframe: Sec. 3 wireframe relaxation: concentric rings
 *                        (circulant tridiagonal systems, Eq. CircTri) and the
 *                        centre point or centre x/y line.
 *   mg_smooth:           any mg_smoother.
 *   mg_colour_pass:      one colour (0 = red, 1 = black) of a base smoother
 *                        (not the alternating ones).                          */
mg_status mg_smooth_tweed(mg_grid *grid, int level, void *u, const void *f, int sweeps,
                          int dtype, void *stream);
mg_status mg_smooth_wireframe(mg_grid *grid, int level, void *u, const void *f, int sweeps,
                              int dtype, void *stream);
mg_status mg_smooth(mg_grid *grid, int level, int smoother, void *u, const void *f, int sweeps,
                    int dtype, void *stream);
mg_status mg_colour_pass(mg_grid *grid, int level, int smoother, int colour, void *u,
                         const void *f, int dtype, void *stream);

/* Sec. 4 step (3) fused: defect d = f - L u on `level`, restricted (half or
 * full weighting) into fc on level+1; uc (level+1, may be NULL) has its
 * interior zeroed, ready for the coarse correction.                          */
mg_status mg_residual_restrict(mg_grid *grid, int level, int restriction, const void *u,
                               const void *f, void *fc, void *uc, int dtype, void *stream);

/* Sec. 4 step (5) fused: u(level) += bilinear prolongation of uc(level+1).   */
mg_status mg_prolong_add(mg_grid *grid, int level, const void *uc, void *u, int dtype,
                         void *stream);

/* Defect d = f - L u on `level` (d is written on every node, 0 on the
 * boundary).                                                                 */
mg_status mg_residual(mg_grid *grid, int level, const void *u, const void *f, void *d,
                      int dtype, void *stream);

/* Direct solve of the coarsest level (dense LU, FP64 arithmetic for both
 * dtypes).  The boundary values of u enter the right-hand side.              */
mg_status mg_coarse_solve(mg_grid *grid, void *u, const void *f, int dtype, void *stream);

/* The level the FP32 cycles solve directly under mg_params.coarse_direct:
 * the finest level below the finest one with both sides at most 64
 * intervals, or -1 (no such level, a 3D grid, or no FP32 workspaces).       */
int mg_direct_level(const mg_grid *grid);

/* Direct solve of that level's interior system in FP32 (u, f: float arrays
 * of the level's shape; the boundary values of u enter the right-hand side)
 * by the fast diagonalisation of the operator's Kronecker-sum form: the 1D
 * factors, symmetrised by the diagonal D of Sec. 2's symmetry, are
 * eigen-decomposed once at setup; a solve is four dense products in one CTA.
 * MG_ERR_UNSUPPORTED when mg_direct_level() is -1.                          */
mg_status mg_direct_solve(mg_grid *grid, void *u, const void *f, void *stream);

/* One cycle (params->cycle: V or W) on the finest level, in the dtype of
 * params->precision (MG_PREC_F64 -> double arrays, MG_PREC_F32_REFINE ->
 * float arrays).  u holds the boundary data and the current iterate.         */
mg_status mg_vcycle(mg_grid *grid, void *u, const void *f, const mg_params *params,
                    void *stream);

/* Solve to params->tol: cycles (Sec. 4) until ||f - L u||_2 / ||f - B g||_2
 * <= tol over the interior nodes, where f - B g is the right-hand side of the
 * interior system (||f|| when the boundary data g vanish).  u, f: FP64 device
 * arrays of the finest level.  u holds g on its boundary (and the initial
 * guess when use_initial_guess).  MG_PREC_F64: FP64 cycles.
 * MG_PREC_F32_REFINE: FP32 smoothing, transfers and cycles on the correction
 * equation, FP64 residual, update and coarsest solve (iterative refinement).
 * info may be NULL.                                                          */
mg_status mg_solve(mg_grid *grid, double *u, const double *f, const mg_params *params,
                   mg_info *info, void *stream);

/* Adjoint solve L^T lambda = rhs with homogeneous boundary data, to the same
 * tolerance.  Uses D L = (D L)^T with D = diag(dx_i dy_j): lambda = D mu with
 * L mu = D^{-1} rhs, solved by the same multigrid.  lambda, rhs: FP64 device
 * arrays of the finest level; lambda's boundary is set to 0.                 */
mg_status mg_solve_adjoint(mg_grid *grid, double *lambda, const double *rhs,
                           const mg_params *params, mg_info *info, void *stream);

/* ---- batches of independent problems (the paper solves one problem at a
 * time; this serves many problems of different sizes and stretchings at
 * once).  A batch is a set of distinct grids (each problem needs its own
 * grid: grids hold per-solve scratch).  mg_batch_create creates up to 64
 * streams of the batch's own and the argument tables of its packed groups
 * (below; device and pinned host memory, about 1.5 KB per problem);
 * MG_ERR_INVALID_ARG if a grid repeats.  The grids stay owned by the caller
 * and must outlive the batch.                                                */
typedef struct mg_batch mg_batch;
mg_status mg_batch_create(mg_batch **out, int count, mg_grid *const *grids);
void mg_batch_destroy(mg_batch *batch);

/* Solves problem i (u[i], f[i]: FP64 device arrays of grid i, as in
 * mg_solve) for every i, with params[0] for all (nparams = 1) or params[i]
 * for problem i (nparams = count; e.g. tweed for wall-clustered and
 * wireframe for centre-clustered grids, Sec. 6).  Problems whose grids have
 * the same shape and whose parameters are equal (MG_PREC_F32_REFINE,
 * coarse_direct 0, every line pass on the warp path of mg_set_line_path)
 * form packed groups: each
 * kernel of their solve is one launch for the whole group, and the FP32
 * cycles of a refinement step are one CUDA graph per group (captured on the
 * first call and reused while the grids' line paths stay).  Groups and the
 * other problems run concurrently on the batch's streams; the host waits once
 * per cycle (FP64) or refinement step (FP32) for all of them, and each problem
 * stops at its own tolerance.  Results, infos[i] and status[i] (host arrays of
 * count entries, either may be NULL) are those mg_solve gives for the problem
 * alone, bit for bit.  Starts after the work already on `stream` and makes
 * `stream` wait for its end.  Returns MG_OK if every problem returned MG_OK,
 * else the first non-OK status in problem order.                            */
mg_status mg_batch_solve(mg_batch *batch, double *const *u, const double *const *f, const mg_params *params,
                         int nparams, mg_info *infos, int *status, void *stream);

/* Gradient with respect to the Dirichlet data (adjoint of the boundary
 * coupling; the paper has no adjoint, this serves differentiation through the
 * solve).  With u_int = A^{-1} (f - B g), where (B g)_p sums coef(p -> b) g_b
 * over the boundary neighbours b of interior node p, and lambda from
 * mg_solve_adjoint with rhs = dloss/du:
 *     grad_g[b] = grad_u[b] - sum_p coef(p -> b) lambda[p]   on boundary nodes,
 *     grad_g    = 0                                          at interior nodes
 * (dloss/df = lambda).  lambda, grad_u, grad_g: FP64 device arrays of the
 * finest level; grad_g must not alias the others.  Enqueued on `stream`.      */
mg_status mg_boundary_adjoint(mg_grid *grid, const double *lambda, const double *grad_u, double *grad_g,
                              void *stream);

/* Defaults for mg_params.                                                    */
void mg_default_params(mg_params *params);

/* Static description of a status code / the last CUDA error message.        */
const char *mg_status_string(mg_status status);
const char *mg_last_error(void);

/* Checked builds.  The library built with -DMG_CHECK (build.py --checked)
 * has every kernel validate the indices it decodes from its descriptors --
 * node positions, junctions, tiles, chunk runs, sequences -- against its
 * level before it uses them, in place of a memory checker (compute-sanitizer
 * is not available everywhere).  A bad index is recorded in a device word and
 * replaced by a safe one; every entry that launches kernels then waits for
 * them and returns MG_ERR_INVALID_ARG.  mg_check_word() waits for the device
 * and returns, and clears, the recorded bits: 0x80000000 marks a checked
 * build, bit 0 a bad index since the last call.  Other builds return 0
 * without waiting.  The paper has no counterpart; this is a test aid.       */
unsigned mg_check_word(void);

/* Residual norms for callers that cannot allocate device memory (the paper has
 * no counterpart; this is a deployment aid).  Some callers must not call
 * cudaMalloc at all -- code that runs inside a memory pool it does not own, a
 * process whose allocator is locked after start-up -- and so cannot create an
 * mg_grid either.  This entry point needs no grid and allocates nothing: from
 * caller-owned DEVICE arrays it computes, over the interior nodes,
 *   out[0] = sum (f - L u)^2,  out[1] = max |f - L u|,
 *   out[2] = sum f^2,          out[3] = max |f|          (out: 4 doubles),
 * with L the operator of Eq. (prob:DP) given by the coefficient arrays W, E
 * (nx+1 each) and S, N (ny+1 each), u and f of shape (ny+1) x (nx+1), FP64.
 * Its scratch is a static device array of 4 x 16384 doubles (one partial per
 * interior row), so ny - 1 may not exceed 16384: larger grids return
 * MG_ERR_SIZE with a message in mg_last_error().  Every call made outside a
 * stream capture looks up the array's device address (cudaGetSymbolAddress)
 * for the current device; a call made while `stream` is being captured uses
 * the address found by an earlier uncaptured call on that device, so make a
 * first call before any stream capture (and again after a cudaDeviceReset);
 * without one a captured call returns MG_ERR_INVALID_ARG.  All calls on a
 * device share the array: calls whose kernels overlap on the GPU (different
 * streams without ordering) race and give wrong results.  No entry needs
 * clearing: each call writes every partial it reads.  The maxima propagate
 * NaN, like the sums.  Enqueued on `stream`; no synchronisation.             */
mg_status mg_residual_norm_static(int64_t nx, int64_t ny, const double *W, const double *E,
                                  const double *S, const double *N, const double *u, const double *f,
                                  double *out, void *stream);

/* Number of CUDA kernels this library has launched in this process (all
 * grids, all streams; counted on the host at launch time).  For
 * instrumentation: the difference across a region counts its launches.      */
unsigned long long mg_kernel_launches(void);

/* Live timing of the colour passes (Sec. 3 relaxation, one colour) that run
 * on `level` from now on, up to `max_passes` (1 .. 2^20) of them: every such
 * pass records 4 CUDA events on its own stream -- before each of the three
 * kernels of the tiled line path (reduce, couple, expand) and after the last.
 * Passes that do not take the tiled path put all their time in the third
 * stage.  Creates the 4 x max_passes events on the host (no device memory);
 * MG_ERR_INVALID_ARG if a timer is already running on this grid.  The events
 * are not captured into CUDA graphs: do not begin a timer around a capture. */
mg_status mg_pass_timer_begin(mg_grid *g, int level, int max_passes);

/* Ends the timer: waits for the last recorded event, then writes the number
 * of passes timed (`passes`), the summed milliseconds of each stage
 * (`stage_ms`, 3 doubles: reduce, couple, expand) and the fastest and slowest
 * whole pass.  Any output pointer may be NULL.  Destroys the events.         */
mg_status mg_pass_timer_end(mg_grid *g, int64_t *passes, double *stage_ms, double *pass_min_ms,
                            double *pass_max_ms);

/* ---- line-solve paths and their autotuner.  A colour pass of a line
 * smoother (zebra, tweed, wireframe; Sec. 3) can be laid out on the GPU in
 * four ways; each solves every block of the colour exactly, they differ only
 * in how the work is spread over threads (and so in rounding order and
 * speed).  The paper's solver is serial; these have no counterpart there.    */
typedef enum {
  MG_PATH_AUTO = 0,  /* built-in rule: the warp path where every block of the
                        colour fits it and both sides are below 2048 intervals,
                        else the tiled path where it exists, else the CTA path */
  MG_PATH_WARP = 1,  /* blocks laid end to end in sequences of 32*W*K nodes, one
                        per CTA of W warps; K consecutive nodes per thread     */
  MG_PATH_TILED = 2, /* 32 x 32-node tiles of parallel legs: three kernels     */
  MG_PATH_CTA = 3,   /* whole blocks per CTA, 32-node chunks per thread         */
  MG_PATH_CLUSTER = 4 /* the tiles of the tiled path, each group of blocks on
                        one thread-block cluster, in one kernel with every
                        intermediate in shared memory (FP32 only; measured
                        slower than the tiled path on GB300, so never chosen
                        by the built-in rule)                                  */
} mg_line_path;

/* Sets the path of the colour passes of `smoother` (MG_SMOOTH_ZEBRA_X,
 * _ZEBRA_Y, _TWEED or _WIREFRAME) on `level` in `dtype` (mg_dtype).  k: for
 * MG_PATH_WARP the preferred nodes per thread (1, 2, 4, 8 or 16; 0 = 4), kept
 * while the largest block fits 8 warps (K doubles otherwise); ignored by the
 * other paths.  MG_ERR_UNSUPPORTED if the level's blocks do not fit the path:
 * the warp path takes blocks of up to 4096 nodes in FP32 and 2048 in FP64;
 * the tiled path exists for tweed and zebra on levels whose sides are both at
 * least 1024 intervals; the cluster path exists in FP32 where the tiled path
 * does, the device runs clusters of 8 CTAs, and every group of the tiled
 * path fits 8 CTAs of 16 tiles.  The previous choice then stays.  May allocate and
 * free device memory (work lists); synchronises the device and drops the
 * grid's captured cycle graphs.
 * On 3D grids (Sec. 7) the choice is for MG_SMOOTH_TWEED only, and for both
 * dtypes at once: MG_PATH_WARP, or MG_PATH_TILED on levels whose sides are
 * all at least 64 intervals (32 chunks of parallel legs per warp; the
 * built-in rule takes it where the sides are all at least 256); k is
 * ignored.  The 3D wireframe has the warp path alone (MG_ERR_UNSUPPORTED for
 * any other); the coarsest level has no passes (MG_ERR_INVALID_ARG).       */
mg_status mg_set_line_path(mg_grid *grid, int level, int smoother, int dtype, int path, int k);

/* The path the colour passes of (level, smoother, dtype) take now, resolved
 * (never MG_PATH_AUTO; where the two colours differ, that of colour 0) and,
 * for the warp path, its shape: *k nodes per thread and *w warps per
 * sequence (both 0 for the other paths).  Any output pointer may be NULL.   */
mg_status mg_get_line_path(const mg_grid *grid, int level, int smoother, int dtype, int *path, int *k,
                           int *w);

/* Autotuner.  For every level but the coarsest (which is solved directly),
 * times `reps` colour passes of `smoother` in `dtype` (alternating colours,
 * after 2 untimed ones; CUDA events on `stream`) with each path and warp
 * shape (k = 1, 2, 4, 8, 16) the level's blocks fit, and keeps the fastest
 * (mg_set_line_path).  The passes run on zeroed scratch arrays allocated
 * here, so no caller data is touched.  The alternating smoothers tune both of
 * their line smoothers; checkerboard has nothing to tune.  Choices are
 * remembered for the process by (level shape, line smoother, dtype): levels
 * of this or any later grid with a remembered shape take the remembered
 * choice without timing (with reps <= 0, only remembered choices are applied
 * and nothing is timed).  times_us: NULL or a HOST array of mg_num_levels
 * doubles, set to the chosen paths' microseconds per colour pass (summed over
 * the two line smoothers of an alternating smoother; 0 where nothing was
 * timed).  Synchronises; may allocate; drops the grid's captured graphs.     */
mg_status mg_autotune(mg_grid *grid, int smoother, int dtype, int reps, double *times_us, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TWEEDMG_MG_H */
