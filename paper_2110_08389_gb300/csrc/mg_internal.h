// mg_internal.h -- data layout shared by the host driver and the sm_103a
// kernels of tweedmg (not part of the public ABI; see include/mg.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
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
// thread.  Chunk c of a CTA owns 32 shared-memory slots (node q of the chunk
// in slot 32c + (q ^ (c % 32)), an XOR swizzle that keeps both "one thread per
// chunk" and "one lane per node" accesses free of bank conflicts).
// Consecutive chunks of a chain are consecutive in the CTA's chunk list, so
// the reduced-system neighbours of chunk t are chunks t-1 (if LP) and t+1 (if
// LN).  info: bits 0-9 = CTA-local index of the chain's junction (JNONE if
// none); bit 15 = the chunk is loaded and stored through a VGroup.
struct ChunkDesc {
  uint16_t i0, j0;
  uint8_t len, flags;
  uint16_t info;
};
static_assert(sizeof(ChunkDesc) == 8, "ChunkDesc layout");
constexpr uint16_t JNONE = 1023, GROUPED = 0x8000;

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
  int vg0, nvg;
  int nnode;  // unknowns of the CTA's chains (junctions excluded)
  int pad;
};

// Up to four vertical chunks of one CTA with the same rows and direction in
// same-colour columns i, i+2, i+4, i+6 (CTA-local chunk ids, 0xFFFF = none).
// The load / store phases read them with lanes spread over 8 rows x 4
// columns, so one warp access touches a few sectors instead of 32 rows.
struct VGroup {
  uint16_t c[4];
};
static_assert(sizeof(CtaWork) == 32, "CtaWork layout");

// Device-resident work list of one (level, smoother, colour, CTA shape).
struct WorkList {
  int ncta = 0;
  int nt = 0;           // threads per CTA = max chunks per CTA
  int total_nodes = 0;  // unknowns relaxed by this list (junctions included)
  void *mem = nullptr;  // one allocation behind the four arrays
  CtaWork *cta = nullptr;
  ChunkDesc *chunk = nullptr;
  JuncDesc *junc = nullptr;
  VGroup *vg = nullptr;
};

// ---------------------------------------------------------------------------
// Warp line path (small levels).  The blocks of one colour are concatenated,
// whole, into sequences of at most 32*K chain nodes, one sequence per warp;
// consecutive nodes of a sequence are coupled when they are consecutive nodes
// of one chain, so the sequence is one tridiagonal system with zero couplings
// between chains.  Lane l owns nodes l*K .. l*K+K-1; the last of them is the
// lane's separator.  A warp holds at most one junction node.
enum : uint32_t { WN_PRED = 1u << 2, WN_SUCC = 1u << 5, WN_JUNC = 1u << 8, WN_VALID = 1u << 9 };

// One node of a sequence: position, and the directions from it to its
// predecessor (bits 0-1, present if WN_PRED), successor (bits 3-4, WN_SUCC)
// and the junction (bits 6-7, WN_JUNC).  Unused slots have fl = 0.
struct WNode {
  uint16_t i, j;
  uint32_t fl;
};
static_assert(sizeof(WNode) == 8, "WNode layout");

// The junction of one warp (has_j = 0: none).  Attached node e (< natt) is
// node as[e] of the sequence, in direction (adirs >> 2e) & 3 from the
// junction.
struct WBlock {
  uint16_t ji, jj;
  uint8_t has_j, natt, adirs, pad;
  uint16_t as[4];
};
static_assert(sizeof(WBlock) == 16, "WBlock layout");

struct WarpList {
  int nwarp = 0;        // sequences (CTAs); 0: the level's blocks do not fit
  int K = 0;            // nodes per lane (power of two)
  int W = 1;            // warps per sequence (power of two)
  int total_nodes = 0;  // unknowns relaxed (junctions included)
  void *mem = nullptr;
  WNode *node = nullptr;   // 32*W*K per sequence
  WBlock *blk = nullptr;   // one per sequence
};
// Shapes of the warp path: K nodes per lane (register arrays of 4K values
// per thread) on W warps per sequence.  K is the smaller of WK_PREF and what
// the largest block needs on one warp, W what it then needs; when that is
// more than WW_MAX warps, K doubles up to WK_MAX.
constexpr int WK_PREF = 4, WK_MAX_F32 = 16, WK_MAX_F64 = 8, WW_MAX = 8;
// Levels with both sides below this use the warp path wherever the largest
// block fits it; larger levels use the tiled path.  Measured on GB300 (FP32
// tweed colour pass, 4097^2 wall grid): 1025^2 15 us (tiled: 39 us), 2049^2
// 43 us (tiled: 44 us, and the whole solve 0.3 ms faster with the tiled path).
constexpr int WARP_MAX_SIDE = 2048;

// ---------------------------------------------------------------------------
// 3D grids (Sec. 7): tweed and wireframe on the warp path.  Directions 0..5 =
// +x, -x, +y, -y, +z, -z (coefficients E_i, W_i, N_j, S_j, T_k, B_k); the
// opposite of d is d ^ 1.  A 3D node descriptor packs i | j << 10 | k << 20
// and the directions to its predecessor (bits 0-2, WN3_PRED), successor
// (bits 4-6, WN3_SUCC) and junction (bits 8-10, WN3_JUNC); bits 16-20 hold
// the index, within its sequence, of the junction of the node's block.
// Unused slots are zero.
enum : uint32_t { WN3_PRED = 1u << 3, WN3_SUCC = 1u << 7, WN3_JUNC = 1u << 11, WN3_VALID = 1u << 12 };
constexpr int WN3_JSHIFT = 16, WJ3_MAX = 32;  // at most 32 junctions per sequence
struct WNode3 {
  uint32_t ijk, fl;
};
static_assert(sizeof(WNode3) == 8, "WNode3 layout");
// A junction of a 3D sequence: the centre of a tweed star (natt = its legs)
// or the node that closes a wireframe ring (natt = 2, both ends of the ring's
// chain).  Attached node e (< natt <= 6) is node as[e] of the sequence, in
// direction (adirs >> 3e) & 7 from the junction.
struct WJunc3 {
  uint32_t ijk;
  uint8_t natt, pad[3];
  uint32_t adirs;
  uint16_t as[6];
  uint8_t pad2[8];
};
static_assert(sizeof(WJunc3) == 32, "WJunc3 layout");
// A wireframe edge skeleton (Sec. 7): the twelve edges of a concentric
// cuboid.  Corner c at cijk[c]; edge e runs from corner ea[e] towards corner
// eb[e] in direction ed[e], its interior nodes at scratch positions
// [eoff[e], eoff[e + 1]) in order from corner ea[e].
struct WSkel3 {
  uint32_t cijk[8];
  uint32_t eoff[13];
  uint8_t ea[12], eb[12], ed[12];
  uint8_t pad[8];
};
static_assert(sizeof(WSkel3) == 128, "WSkel3 layout");
struct WarpList3 {
  int nwarp = 0, K = 0, W = 1, total_nodes = 0;
  int nskel = 0, skel_nodes = 0;      // skeleton CTAs (launched first) and their interior edge nodes
  bool multi = false;                 // several junctions per sequence (wireframe lists)
  void *mem = nullptr;
  WNode3 *node = nullptr;
  WJunc3 *junc = nullptr;
  int *jofs = nullptr;                // multi: sequence w owns junctions [jofs[w], jofs[w + 1]);
                                      // otherwise junc[w] is sequence w's (natt = 0: none)
  WSkel3 *skel = nullptr;
};
enum { SM3_TWEED = 0, SM3_WIREFRAME = 1 };
// 3D tiled tweed path (tiles3.cu; layout by tile3_host.h): every 3D tweed
// block of a colour (Sec. 7) as straight legs plus at most one junction, the
// legs cut into 32-node chunks from their first node.  A tile holds 32 such
// chunks of parallel legs, one per lane, at the same 32 positions (same run
// direction and start); the chunks of one leg may sit in different tiles and
// lanes, so every leg lists its chunks' lane slots.  Runs along y and z have
// consecutive x across lanes where the blocks allow (coalesced); runs along
// x are read and written through a per-warp shared-memory transpose.  Lane
// flags are the 2D ones (TL_*): the node before the first / after the last
// is outside the block (its value is known), or the last node's successor is
// the junction.
struct Tile3Desc {
  uint16_t base;  // run coordinate of slot 0
  uint8_t dir;    // 0..5: +x, -x, +y, -y, +z, -z
  uint8_t pad;
};
static_assert(sizeof(Tile3Desc) == 4, "Tile3Desc layout");
struct Tile3Lane {
  uint16_t c1, c2;  // fixed coordinates of the run: (j, k) along x, (i, k) along y, (i, j) along z
  uint8_t q1;       // active slots [0, q1) (0: unused lane)
  uint8_t flags;    // TL_*
  uint16_t pad;
};
static_assert(sizeof(Tile3Lane) == 8, "Tile3Lane layout");
struct Block3Desc {
  uint16_t ji, jj, jk;   // junction node
  uint8_t nleg, junc;    // legs; 1 if the block has a junction
  uint32_t jdirs;        // 3 bits per leg: direction from the junction to the leg's last node
  uint32_t leg_slot0[6]; // chunk r of leg l is lane slot[leg_slot0[l] + r] (= tile * 32 + lane)
  uint16_t leg_len[6];
  uint8_t pad[16];
};
static_assert(sizeof(Block3Desc) == 64, "Block3Desc layout");
struct Tile3List {
  int ntile = 0, nblock = 0, ngroup = 0, nslot = 0, max_leg_chunks = 0;
  void *mem = nullptr;
  Tile3Desc *tile = nullptr;
  Tile3Lane *lane = nullptr;    // 32 per tile
  Block3Desc *block = nullptr;  // 32 per group (unused entries: nleg = junc = 0)
  uint32_t *slot = nullptr;     // the chunks of every leg, in order
  // FP32 grids: per lane slot (tile * 32 + lane), the couple's forward-sweep
  // constants of the reduced lo and hi rows, laid out as TileList.cconst
  // (a float4 per slot, then a float2 per slot); set at setup
  // (setup_couple_consts3).  nullptr otherwise.
  void *cconst = nullptr;
};
struct Level3 {
  int nx = 0, ny = 0, nz = 0;
  size_t nn = 0;
  std::vector<double> hx, hy, hz;
  std::vector<double> hc[6];          // host coefficients W, E, S, N, B, T
  double *c64[6] = {};                // device coefficients (same order)
  float *c32[6] = {};
  void *dev_block = nullptr;          // one allocation behind the coefficients
  double *u64 = nullptr, *f64 = nullptr;  // coarse-level workspaces
  float *u32 = nullptr, *f32 = nullptr;
  WarpList3 wp[2][2];                 // [SM3_*][colour]: shared by both precisions
  bool wf_ok = false;                 // wireframe blocks are all rings, lines, points and skeletons
  Tile3List t3[2];                    // tweed tiles per colour (t3_ok: built)
  bool t3_ok = false;
  int t3_path = 0;                    // 0: built-in rule, 1: warp path, 2: tiled path (mg_set_line_path)
};
struct Grid3 {
  std::vector<Level3> lev;
  int cn = 0;
  double *cinv = nullptr;             // dense inverse of the coarsest interior operator
  double *d64 = nullptr;              // defect scratch of the finest level's size
  float *d32 = nullptr;
  double *skel_scr = nullptr;         // skeleton edge scratch: 6 rows of skel_len values
  size_t skel_len = 0;
};

// ---------------------------------------------------------------------------
// Tiled line path (tweed and zebra on large levels).  Every block is a set of
// legs that each start at a wall, plus at most one junction node (the
// paper's m-legged form, Eq. mLThomas; m = 1 for a line from wall to wall).
// Legs are cut into chunks at absolute positions (every 32 nodes from the
// wall), so the legs of neighbouring same-colour blocks line up: a tile is
// one such 32-node stretch of 32 parallel legs, one warp per tile.
//   tile_reduce   per lane: right-hand side of the chunk and its two reduced
//                 rows (partition method) -> scratch
//   tile_couple   per leg: Thomas on the reduced rows towards the junction,
//                 the junction row, back-substitution -> chunk end values
//   tile_expand   per lane: interior of the chunk by Thomas -> u
enum : uint8_t { TL_FIRST = 1, TL_LAST_J = 2, TL_LAST_W = 4 };

struct TileLane {
  uint16_t line;   // fixed coordinate of the run (j for x-runs, i for y-runs)
  uint8_t q0, q1;  // active slots [q0, q1) of the tile (q1 = 0: unused lane)
  uint8_t flags;   // TL_FIRST: slot q0 is the leg's first node (its predecessor is a wall node);
                   // TL_LAST_J / TL_LAST_W: slot q1-1 is the leg's last node and its successor
                   // is the junction / a wall node
  uint8_t pad[3];
};
static_assert(sizeof(TileLane) == 8, "TileLane layout");

struct TileDesc {
  uint16_t base;   // run coordinate of slot 0
  uint8_t dir;     // run direction (DIR_*)
  uint8_t pad[5];
};
static_assert(sizeof(TileDesc) == 8, "TileDesc layout");

// One block for tile_couple: its legs are lane `lane` of the tiles
// leg_tile0[l] .. leg_tile0[l] + ceil(leg_len[l]/32) - 1.
struct BlockDesc {
  uint16_t ji, jj;        // junction node
  uint8_t nleg, junc;     // number of legs; 1 if the block has a junction
  uint8_t jdirs, lane;    // direction junction -> last node of leg l (2 bits each); tile lane
  uint32_t leg_tile0[4];
  uint16_t leg_len[4];
};
static_assert(sizeof(BlockDesc) == 32, "BlockDesc layout");

// Legs of at most this many chunks take the FP32 couple with precomputed
// pivots (tiles.cu, tile_couple_pc).
constexpr int TILE_PC_CHUNKS = 64;

struct TileList {
  int ntile = 0, nblock = 0, ngroup = 0;
  int max_leg_chunks = 0;       // longest leg, in chunks
  int total_nodes = 0;
  void *mem = nullptr;
  TileDesc *tile = nullptr;
  TileLane *lane = nullptr;     // 32 per tile
  BlockDesc *block = nullptr;   // 32 per group (unused entries have nleg = junc = 0)
  // FP32 grids with legs of at most TILE_PC_CHUNKS chunks: per lane and
  // chunk (index tile * 32 + lane), the couple's forward-sweep constants of
  // the reduced lo and hi rows: a float4 (pivot 1 / (1 - a c'_prev) and a
  // times it, lo then hi) for every lane chunk, followed by a float2 (c' of
  // lo and hi) for every lane chunk; set once at setup (setup_couple_consts).
  // nullptr otherwise.
  void *cconst = nullptr;
};

// Cluster pass (FP32 tweed and zebra on the tiled levels): the three stages of
// the tiled path in ONE kernel, the chunk right-hand sides and reduced rows
// kept in shared memory.  The tiles of a group of blocks are spread over the
// CTAs of one thread-block cluster, at most CL_TILES tiles per CTA; each CTA
//   1. computes its chunks' right-hand sides and reduced rows (partition
//      method, as tile_reduce) into shared memory;
//   2. after a cluster barrier, solves some of the group's blocks: Thomas on
//      the reduced rows of each leg from the wall to the junction, the
//      junction row, back-substitution (as tile_couple), reading and writing
//      the rows and chunk end values where they lie, in the shared memory of
//      the CTA that holds the chunk (DSMEM);
//   3. after a second cluster barrier, expands its chunks (Thomas between the
//      known end values) into u.
// Blocks are the paper's m-legged systems (Eq. mLThomas); the elimination is
// that of the tiled path.  A group of one block (the centre cross, the
// T-blocks of a rectangle) is laid out "compact": the lanes of a tile are 32
// consecutive chunks of one leg instead of 32 parallel legs.
constexpr int CL_TILES = 16;      // tiles (32 chunks each) per CTA
constexpr int CL_CTAS = 8;        // CTAs per cluster (portable maximum)
constexpr int CL_WARPS = 8;       // warps per CTA
constexpr int CL_MAXSEG = CL_CTAS;  // segments per leg (one per CTA of its group)
constexpr int CL_LEGROWS = 1536;    // (c', d') places of the legs one CTA solves

enum : uint8_t { CT_COMPACT = 1 };
struct CTile {
  uint16_t base;   // run coordinate of slot 0 (regular tiles)
  uint8_t dir;     // run direction (DIR_*)
  uint8_t kind;    // 0 or CT_COMPACT
  uint32_t pad;
};
static_assert(sizeof(CTile) == 8, "CTile layout");
struct CLane {
  uint16_t line;   // fixed coordinate of the run
  uint8_t q1;      // active slots [0, q1) (0: unused lane)
  uint8_t flags;   // TL_FIRST / TL_LAST_J / TL_LAST_W, as TileLane
  uint16_t cbase;  // compact tiles: run coordinate of the lane's slot 0
  uint16_t pad;
};
static_assert(sizeof(CLane) == 8, "CLane layout");
// One CTA: tiles [tile0, tile0 + ntile) of the plan, segments [seg0, seg0 +
// nseg); its group's CTAs are cluster ranks rank0 .. rank0 + ngr - 1 and this
// one is rank0 + grank.  group < 0: an idle CTA that only fills its cluster.
struct CCta {
  int32_t tile0, group, seg0;
  uint16_t nseg;
  uint8_t ntile, grank, rank0, ngr, nleg, pad;
};
static_assert(sizeof(CCta) == 20, "CCta layout");
// A segment: nchunk consecutive chunks of one leg held by one CTA, the first
// (nearest the wall) at CTA-local chunk slot slot0 = tile * 32 + lane, the
// next ones stride slots further (32 for regular tiles, 1 for compact ones).
// Each chunk has two reduced rows, but a last chunk of one node (one = 1)
// has one.
struct CSeg {
  uint16_t slot0, nchunk;
  uint8_t stride, one, pad[2];
};
static_assert(sizeof(CSeg) == 8, "CSeg layout");
// A block of a group: junction node, legs, and direction junction -> last
// node of leg l in bits 2l..2l+1 (as BlockDesc).
struct CBlock {
  uint16_t ji, jj;
  uint8_t nleg, junc, jdirs, pad;
};
static_assert(sizeof(CBlock) == 8, "CBlock layout");
// Leg l of block b of a group (record l * 32 + b): its segments from the wall
// to the junction, segment s held by cluster rank rank[s] as segment slot[s]
// of that CTA's list.
struct CChain {
  uint8_t nseg;
  uint8_t rank[CL_MAXSEG];
  uint8_t slot[CL_MAXSEG];
  uint8_t pad;
  uint16_t roff;   // first of its rows' places in the solving CTA's (c', d') store
  uint16_t nrow;   // reduced rows of the leg
  uint16_t pad2;
};
static_assert(sizeof(CChain) == 24, "CChain layout");
struct ClusterPlan {
  int ncta = 0;        // a multiple of CL_CTAS (0: the level has no cluster pass)
  int ntile = 0, nseg = 0, ngroup = 0;
  void *mem = nullptr;
  CTile *tile = nullptr;
  CLane *lane = nullptr;   // 32 per tile
  CCta *cta = nullptr;
  CSeg *seg = nullptr;
  CBlock *block = nullptr; // 32 per group
  CChain *chain = nullptr; // 128 per group
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
  double *WE64 = nullptr;               // W_i + E_i per column (the FP64 defect's diagonal part)
  void *dev_block = nullptr;            // one allocation behind the arrays above
  // workspaces of coarse levels (level 0 uses the caller's arrays)
  double *u64 = nullptr, *f64 = nullptr;
  float *u32 = nullptr, *f32 = nullptr;
  bool wl_built[WL_COUNT][2] = {};    // [smoother][precision 0=f64,1=f32]
  bool tl_built[WL_COUNT] = {};
  TileList tl[WL_COUNT][2];           // [smoother][colour]: tiled path (empty: use the work lists)
  ClusterPlan cp[WL_COUNT][2];        // [smoother][colour]: cluster pass (FP32; ncta = 0: none)
  WorkList wl[WL_COUNT][2][2][2];     // [smoother][precision][colour][small, large]
  WarpList wp[WL_COUNT][2][2];        // [smoother][precision][colour]: warp path (nwarp = 0: unused)
  int path[WL_COUNT][2] = {};         // [smoother][precision]: MG_PATH_* (0 = the built-in rule)
  int kpref[WL_COUNT][2] = {};        // nodes per lane asked of the warp path (0 = WK_PREF)
};

struct Grid {
  int dim = 2;
  Grid3 *g3 = nullptr;               // dim == 3: the 3D levels (lev then stays empty)
  int nlev = 0;
  int sms = 1;                       // multiprocessors of the device the grid was set up on
  bool cluster_ok = false;           // FP32 grid on a device that runs the cluster pass
  int prec_mask = 3;
  std::vector<Level> lev;
  // coarsest level: dense inverse of the interior operator (FP64, row-major)
  int cn = 0;
  double *cinv = nullptr;
  // level solved directly by the FP32 cycles when mg_params.coarse_direct is
  // set (fd.cu): -1 if none; its transforms (FP32)
  int fd_level = -1;
  float *fd_tr = nullptr;
  // finest-level FP64/FP32 scratch for the refinement loop and norms
  double *r64 = nullptr;             // adjoint scratch: the scaled right-hand side (finest)
  float *e32 = nullptr, *r32 = nullptr;
  // FP32+refine on 2D grids: the second FP64 iterate (the refinement writes
  // u + e here, then back, alternately), the diagonal W_i + E_i + S_j + N_j
  // per node, and the tiling of the fused residual kernel (rows per CTA, CTA
  // grid) with its own partial sums
  double *u2 = nullptr, *cd64 = nullptr, *rpart = nullptr;
  int rr_rows = 0, rr_gx = 0, rr_gy = 0;
  double *partial = nullptr;         // per-CTA partial sums (deterministic norm)
  double *hpinned = nullptr;         // pinned host mirror of the norm results
  int npartial = 0;
  double *scal = nullptr;            // device scalars (reduced norms)
  unsigned *dev_status = nullptr;    // bits set by kernels that found a fault (DEV_*); 0 when clean
  // scratch of the tiled line path, sized for the largest tile list
  size_t tile_cap = 0;               // tiles
  void *tile_rows = nullptr;         // 2 reduced rows per lane per tile (FP64 sized)
  void *tile_d = nullptr;            // 32 x 32 right-hand sides per tile (FP64 sized)
  void *tile_x = nullptr;            // 2 end values per lane per tile (FP64 sized)
  // live timing of one level's colour passes (mg_pass_timer_begin/end): 4
  // events per pass, recorded on the pass's stream before each of the three
  // tiled-path kernels and after the last
  int timer_level = -1, timer_cap = 0, timer_n = 0;
  cudaEvent_t *timer_ev = nullptr;
  // Captured cycle sequences (CUDA graphs), replayed on the grid's own stream
  // `gs`, ordered after / before the caller's stream by ev_fork / ev_join.
  struct GraphEntry {
    int key[8];
    const void *u, *f;
    cudaGraphExec_t exec;
    unsigned long long launches;  // kernels in the graph
  };
  std::vector<GraphEntry> graphs;
  cudaStream_t gs = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  unsigned long long gen = 0;        // bumped whenever a level's line path or warp lists change
};

// Levels whose sides are both at least this get tiled lists for tweed and
// zebra, used where the warp path is not (below it the CTA line kernel is
// faster than the tiled path: measured on GB300, 512^2: 29 vs 39 us per
// colour pass; 1024^2: 45 vs 41 us).
constexpr int TILE_MIN_SIDE = 1024;

// Checked builds (-DMG_CHECK): each translation unit with kernels registers,
// under its file name, a reader of its device check word and of the source
// line of its first failed check (device_util.cuh); check_words() ORs and
// clears them all (0 in other builds) and names the first site in *where.
void register_check_reader(const char *tu, unsigned (*reader)(unsigned *line));
unsigned check_words(std::string *where = nullptr);
// st, or in checked builds MG_ERR_INVALID_ARG once a kernel recorded a bad index
mg_status checked(mg_status st);

// Kernels launched by this library in this process (mg_kernel_launches).
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---- host helpers (api.cu): Sec. 2 coefficients of one axis; Gauss-Jordan
// inverse with partial pivoting (false if singular)
void axis_coefficients(const std::vector<double> &x, std::vector<double> &lo, std::vector<double> &hi);
bool invert(int n, std::vector<double> &A, std::vector<double> &inv);

// ---- direct level solve (fd.cu): levels with both sides at most this many
// intervals qualify; the finest such level below the finest one is chosen
constexpr int FD_MAX_SIDE = 64;
mg_status setup_direct_level(Grid &g);
cudaError_t launch_direct_level(const Grid &g, float *u, const float *f, cudaStream_t s);

// ---- 3D grids (grid3d.cu)
mg_status setup3(Grid &g, const int64_t *n, const double *const *coords);
void free3(Grid &g);
template <typename T>
mg_status colour_pass3(Grid &g, int l, int sm, int colour, T *u, const T *f, cudaStream_t s);  // sm: SM3_*
template <typename T>
mg_status cycle3(Grid &g, const mg_params &p, int l, T *u, const T *f, cudaStream_t s);
template <typename T>
mg_status residual3(Grid &g, int l, const T *u, const T *f, T *d, cudaStream_t s);
template <typename T>
mg_status residual_restrict3(Grid &g, int l, const T *u, const T *f, T *fc, T *uc, cudaStream_t s);
template <typename T>
mg_status prolong_add3(Grid &g, int l, const T *uc, T *u, cudaStream_t s);
template <typename T>
mg_status coarse_solve3(Grid &g, T *u, const T *f, cudaStream_t s);
// the FP64 steps of a solve: interior of u := 0; norms into g.scal[0]
// (bnd_only: ||f - B g||^2; with r32: the refinement residual, e32 := 0);
// u += e32
mg_status zero_interior3(Grid &g, double *u, cudaStream_t s);
mg_status norms3(Grid &g, const double *u, const double *f, int bnd_only, float *r32, float *e32, cudaStream_t s);
mg_status ir_update3(Grid &g, double *u, const float *e, cudaStream_t s);

// ---- host helpers (setup.cu)
mg_status build_worklists(Grid &g, int level, int wl, int prec);
// Warp lists of both colours of (level, smoother, precision) with kpref nodes
// per lane preferred (0 = WK_PREF); out[c].nwarp = 0 where a colour's blocks
// do not fit.  The caller owns (and frees) out.
mg_status build_warp_path(Grid &g, int level, int wl, int prec, int kpref, WarpList out[2]);
void free_warplist(WarpList &w);
// (api.cu) work-list index of a base line smoother (-1 otherwise); destroy
// the grid's captured cycle graphs (the caller has synchronised).
int wl_of(int smoother);
void drop_graphs(Grid &g);
const char *set_error(const char *where, cudaError_t e);
void set_error_text(const char *msg);

mg_status build_tiles(Grid &g, int level, int wl);
// (cluster_setup.cu) the cluster pass plans of both colours of a tiled level
// (none where a colour's groups do not fit a cluster, or on FP64-only grids)
mg_status build_cluster_plans(Grid &g, int level, int wl);
// Dynamic shared memory opt-in of the line kernels on the current device
// (called by mg_setup_grid).
cudaError_t prepare_line_kernels();
cudaError_t prepare_tile_kernels();
// The couple constants of every FP32 tile list of the grid (after its tiled
// scratch is allocated).
cudaError_t setup_couple_consts(Grid &g);
cudaError_t prepare_warp_kernels();
// ev: nullptr, or 4 events recorded before tile_reduce, tile_couple,
// tile_expand and after tile_expand
template <typename T>
cudaError_t launch_tile_pass(const Grid &g, const Level &L, const TileList &t, T *u, const T *f, cudaStream_t s,
                             cudaEvent_t *ev);
// The cluster pass (FP32) of one colour; ev as launch_tile_pass (ev[0] before
// the kernel, ev[1..3] after it).
cudaError_t launch_cluster_pass(const Level &L, const ClusterPlan &cp, float *u, const float *f, cudaStream_t s,
                                cudaEvent_t *ev);
cudaError_t prepare_cluster_kernel();
// Clusters of the cluster pass the current device holds at once (0: none).
int cluster_pass_capacity();
// 3D tiled tweed path (tiles3.cu): one colour pass, and the setup-time build
// of a level's tile lists from its tweed blocks (false in *ok if a block does
// not fit the layout; the level then keeps the warp path).
struct HBlock3;
template <typename T>
cudaError_t launch_tile3_pass(const Grid &g, const Level3 &L, const Tile3List &t, T *u, const T *f, cudaStream_t s);
mg_status build_tiles3(Grid &g, Level3 &L, const std::vector<HBlock3> &tweed_blocks, bool *ok);
// The couple constants of every FP32 3D tile list (after the tiled scratch
// and e32 are allocated).
cudaError_t setup_couple_consts3(Grid &g);
// Levels whose sides are all at least T3_MIN_SIDE intervals get 3D tile
// lists; the built-in rule takes the tiled path on those whose sides are all
// at least T3_AUTO_SIDE (measured on GB300, FP32 tweed relaxation: 257^3
// 0.29 ms tiled against 0.42 ms on the warp path; 129^3 0.089 against
// 0.056 ms; 65^3 0.064 against 0.017 ms).
constexpr int T3_MIN_SIDE = 64, T3_AUTO_SIDE = 256;
// The 3D tweed passes of a level take the tiled path (see T3_AUTO_SIDE).
inline bool tiled3(const Level3 &L) {
  return L.t3_ok && (L.t3_path == 2 || (L.t3_path == 0 && std::min(L.nx, std::min(L.ny, L.nz)) >= T3_AUTO_SIDE));
}

// ---- kernel launchers (smooth.cu, transfer.cu).  All return cudaError_t of
// the launch (cudaGetLastError).
template <typename T>
cudaError_t launch_line_pass(const Level &L, const WorkList &w, T *u, const T *f, cudaStream_t s);
template <typename T>
cudaError_t launch_warp_pass(const Level &L, const WarpList &w, T *u, const T *f, cudaStream_t s);
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
// ||f - B u_b||^2: the right-hand side of the interior system (u's interior
// taken as 0); with r32 and e32 also float(f - B u_b), the defect of a zero
// interior, and e32 = 0 (the first refinement step of a zeroed guess)
cudaError_t launch_rhsnorm64(const Grid &g, const double *u, const double *f, cudaStream_t s,
                             float *r32 = nullptr, float *e32 = nullptr);
// Refinement residual of the finest 2D level with the update fused: v = u + e
// (e NULL: v = u), r = f - L v in FP64, r32 = float(r), the FP64 norms of r
// into scal; with e, v goes to uo and e32 is zeroed afterwards, else e32 is
// zeroed in the kernel.  setup_refine_residual sizes its tiling and computes
// cd64 (setup time).
cudaError_t launch_refine_residual(const Grid &g, const double *u, const float *e, double *uo, const double *f,
                                   cudaStream_t s);
mg_status setup_refine_residual(Grid &g);
cudaError_t launch_boundary_adjoint(const Grid &g, const double *lam, const double *gu, double *gg, cudaStream_t s);
// a[interior] *= scale_x[i]*scale_y[j] (adjoint diagonal scalings), boundary := 0.
cudaError_t launch_diag_scale(const Grid &g, double *out, const double *in, int inverse,
                              cudaStream_t s);
// Zero the interior (and optionally boundary) of a level array.
template <typename T>
cudaError_t launch_zero_interior(const Level &L, T *a, cudaStream_t s);

}  // namespace tmg

// The opaque handle of the C ABI.
struct mg_grid : public tmg::Grid {};
