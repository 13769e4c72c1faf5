/*
 * mg_oracle3d.c -- plain, slow, FP64 CPU oracle for 3D tweed / wireframe multigrid
 * (Bewley, Mashayek, Cavaglieri & Luchini, arXiv:2110.08389, Sec. 7).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the tests and the benchmark's CPU-baseline leg use it.
 * It shares no code, header or table with the CUDA path, nor with the 2D
 * oracle.
 *
 * What it computes, in the paper's order:
 *   - the 7-point operator: Eq. (prob:DP) of Sec. 2 with a third axis
 *     (coefficients B_k, T_k over z built like S_j, N_j over y);
 *   - 3D tweed blocks (Sec. 7): starting from the eight corner points, legs
 *     perpendicular to the nearest wall, m = 2 or 3 legs per block, m = 6 at
 *     the centre of a cube;
 *   - 3D wireframe blocks (Sec. 7): the faces of concentric cuboids, as
 *     concentric rings on each face and the cuboid's edge skeleton;
 *   - 3D complementary wireframe blocks (Sec. 7): on the same cuboid faces,
 *     orthogonal to the wireframe, the corner points alone and lines that
 *     circle each cuboid's corners (six joined "+" shapes on a cube);
 *   - each block solved exactly (Sec. 3), here by Gaussian elimination on the
 *     block's tree (leaves first), which is the m-legged Thomas of
 *     Eq. (mLThomas) for a star, and by dense LU for blocks with loops (the
 *     rings of Eq. CircTri and the edge skeletons);
 *   - red pass, then black pass; V-cycle of Sec. 4 with a direct solve on the
 *     coarsest level.
 *
 * Readings where the paper is silent (it gives no 3D formulas):
 *   Q1  nodes 0-based, x fastest: a[(k*(ny+1) + j)*(nx+1) + i].
 *   Q2  with the index distances to the nearer wall d_x = min(i, nx-i),
 *       d_y, d_z sorted as d1 <= d2 <= d3, a tweed block is a connected set of
 *       interior nodes with equal (d2, d3); its lines run along the axis of
 *       d1, perpendicular to the nearest wall, as in 2D (Sec. 3).  Colour:
 *       red (relaxed first) when d2 + d3 is even, so that the eight corner
 *       points (d = 1, 1, 1) are red ("first relaxed", Sec. 7).  Adjacent
 *       nodes either share (d2, d3) or differ by one in d2 + d3, so blocks of
 *       one colour never touch.
 *   Q3  transfers are the tensor products of the 1D factors of the 2D rules
 *       of Sec. 4: full weighting with 1D weights (1/4, 1/2, 1/4) per axis
 *       (27 points), trilinear prolongation; coarse operators rediscretised
 *       on the subsampled coordinates.
 *   Q4  coarsening stops once max(nx, ny, nz) <= 8, or a side is odd or would
 *       drop below 2 intervals; the coarsest level is solved by dense LU.
 *   Q5  the stop test is that of the 2D solve: ||f - L u||_2 / ||f - B g||_2
 *       over interior nodes.
 *   Q6  a 3D wireframe block is a connected set of interior nodes with equal
 *       (d1, d2): for d1 < d2 a ring around the centre of a cuboid face (or a
 *       line or point where the face degenerates), for d1 = d2 the cuboid's
 *       twelve edges with its eight corners.  Red when d1 + d2 is even, so the
 *       outermost skeleton is red, as the outermost ring is in 2D (Sec. 3).
 *   Q7  a complementary wireframe block is a connected set of interior nodes
 *       with equal (d1, d3), red when d1 + d3 is even, so the corner points
 *       (d1 = d3 = 1) are red.  A step between neighbours changes exactly one
 *       of d1, d2, d3 when every side is even, so the three motifs share no
 *       wire and cover every wire.  The triplet step (Sec. 7) is one tweed,
 *       one wireframe and one complementary relaxation, in that order.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define O3_MAXLEV 16

typedef struct {
  int nx, ny, nz;
  double *x, *y, *z;
  double *W, *E, *S, *N, *B, *T; /* 0 at boundary indices */
} lev3_t;

/* one tweed block: nodes in breadth-first order from the root (the node
 * with most in-block neighbours), parent[] the index in node[] of each
 * node's parent (-1 for the root) */
typedef struct {
  int n, colour, maxdeg;
  int *node, *parent;
} blk3_t;

typedef struct {
  int built, nblock;
  blk3_t *blk;
  int *owner;
  int *pool;
} part3_t;

enum { O3_TWEED = 0, O3_WIREFRAME = 1, O3_COMPLEMENTARY = 2, O3_NMOTIF = 3 };
/* o3_smooth also takes the sequences of Sec. 7: */
enum { O3_ALT_TW = 3 /* tweed, then wireframe */, O3_TRIPLET = 4 /* tweed, wireframe, complementary */ };

typedef struct {
  int nlev;
  lev3_t lev[O3_MAXLEV];
  part3_t part[O3_MAXLEV][O3_NMOTIF];  /* [level][tweed, wireframe, complementary] */
  int cn;
  double *clu;
  int *cpiv;
  double *work[O3_MAXLEV][3];
} o3_problem;

static inline size_t I3(const lev3_t *L, int i, int j, int k) {
  return ((size_t)k * (L->ny + 1) + j) * (L->nx + 1) + i;
}
static inline size_t nn3(const lev3_t *L) { return (size_t)(L->nx + 1) * (L->ny + 1) * (L->nz + 1); }
static inline int imin3(int a, int b) { return a < b ? a : b; }
static inline int imax3(int a, int b) { return a > b ? a : b; }

/* Sec. 2 coefficients on one axis: lo_i = 1/(dx_i dx_{i-1/2}),
 * hi_i = 1/(dx_i dx_{i+1/2}), dx_i = (x_{i+1} - x_{i-1})/2.               */
static void coeff_axis(int n, const double *x, double *lo, double *hi) {
  for (int i = 0; i <= n; ++i) lo[i] = hi[i] = 0.0;
  for (int i = 1; i < n; ++i) {
    const double dm = x[i] - x[i - 1], dp = x[i + 1] - x[i], dc = 0.5 * (x[i + 1] - x[i - 1]);
    lo[i] = 1.0 / (dc * dm);
    hi[i] = 1.0 / (dc * dp);
  }
}

static double *dup(const double *a, int n) {
  double *b = malloc(sizeof(double) * n);
  memcpy(b, a, sizeof(double) * n);
  return b;
}

static void lev3_init(lev3_t *L, int nx, int ny, int nz, const double *x, const double *y, const double *z) {
  L->nx = nx; L->ny = ny; L->nz = nz;
  L->x = dup(x, nx + 1); L->y = dup(y, ny + 1); L->z = dup(z, nz + 1);
  L->W = malloc(sizeof(double) * (nx + 1)); L->E = malloc(sizeof(double) * (nx + 1));
  L->S = malloc(sizeof(double) * (ny + 1)); L->N = malloc(sizeof(double) * (ny + 1));
  L->B = malloc(sizeof(double) * (nz + 1)); L->T = malloc(sizeof(double) * (nz + 1));
  coeff_axis(nx, x, L->W, L->E);
  coeff_axis(ny, y, L->S, L->N);
  coeff_axis(nz, z, L->B, L->T);
}

/* the six neighbour steps: -x, +x, -y, +y, -z, +z */
static const int DI[6] = {-1, 1, 0, 0, 0, 0}, DJ[6] = {0, 0, -1, 1, 0, 0}, DK[6] = {0, 0, 0, 0, -1, 1};

/* coefficient of row (i,j,k) towards its neighbour in direction d */
static double coef6(const lev3_t *L, int i, int j, int k, int d) {
  switch (d) {
    case 0: return L->W[i];
    case 1: return L->E[i];
    case 2: return L->S[j];
    case 3: return L->N[j];
    case 4: return L->B[k];
    default: return L->T[k];
  }
}
static double centre3(const lev3_t *L, int i, int j, int k) {
  return -(L->W[i] + L->E[i] + L->S[j] + L->N[j] + L->B[k] + L->T[k]);
}
static int interior3(const lev3_t *L, int i, int j, int k) {
  return i > 0 && i < L->nx && j > 0 && j < L->ny && k > 0 && k < L->nz;
}

/* ------------------------------------------------------- operator, norms -- */

void o3_apply(o3_problem *P, int lev, const double *u, double *out) {
  const lev3_t *L = &P->lev[lev];
  memset(out, 0, sizeof(double) * nn3(L));
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) {
        double s = centre3(L, i, j, k) * u[I3(L, i, j, k)];
        for (int d = 0; d < 6; ++d) s += coef6(L, i, j, k, d) * u[I3(L, i + DI[d], j + DJ[d], k + DK[d])];
        out[I3(L, i, j, k)] = s;
      }
}

void o3_residual(o3_problem *P, int lev, const double *u, const double *f, double *d) {
  const lev3_t *L = &P->lev[lev];
  o3_apply(P, lev, u, d);
  for (int k = 0; k <= L->nz; ++k)
    for (int j = 0; j <= L->ny; ++j)
      for (int i = 0; i <= L->nx; ++i) {
        const size_t p = I3(L, i, j, k);
        d[p] = interior3(L, i, j, k) ? f[p] - d[p] : 0.0;
      }
}

static double sumsq_interior(const lev3_t *L, const double *a) {
  double s = 0.0;
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) s += a[I3(L, i, j, k)] * a[I3(L, i, j, k)];
  return s;
}

/* --------------------------------------------------------- tweed blocks -- */

/* block key of a node: (d2, d3) for tweed (Q2), (d1, d2) for wireframe (Q6),
   (d1, d3) for complementary wireframe (Q7) */
static void key3(const lev3_t *L, int sm, int i, int j, int k, int *k1, int *k2) {
  int a = imin3(i, L->nx - i), b = imin3(j, L->ny - j), c = imin3(k, L->nz - k), t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
  if (sm == O3_WIREFRAME) { *k1 = a; *k2 = b; }
  else if (sm == O3_COMPLEMENTARY) { *k1 = a; *k2 = c; }
  else { *k1 = b; *k2 = c; }
}

static int uf_find(int *par, int x) {
  while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
  return x;
}

static int build_part(o3_problem *P, int lev, int sm) {
  part3_t *T = &P->part[lev][sm];
  if (T->built) return 0;
  const lev3_t *L = &P->lev[lev];
  const size_t nn = nn3(L);
  int *par = malloc(sizeof(int) * nn);
  for (size_t p = 0; p < nn; ++p) par[p] = (int)p;
  /* union along grid edges between interior nodes of equal (d2, d3) */
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) {
        int a2, a3;
        key3(L, sm, i, j, k, &a2, &a3);
        for (int d = 1; d < 6; d += 2) {  /* +x, +y, +z */
          const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
          if (!interior3(L, ii, jj, kk)) continue;
          int b2, b3;
          key3(L, sm, ii, jj, kk, &b2, &b3);
          if (a2 == b2 && a3 == b3) {
            const int r1 = uf_find(par, (int)I3(L, i, j, k)), r2 = uf_find(par, (int)I3(L, ii, jj, kk));
            if (r1 != r2) par[r1] = r2;
          }
        }
      }
  T->owner = malloc(sizeof(int) * nn);
  for (size_t p = 0; p < nn; ++p) T->owner[p] = -1;
  int nb = 0;
  int *root_block = malloc(sizeof(int) * nn);
  for (size_t p = 0; p < nn; ++p) root_block[p] = -1;
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) {
        const int p = (int)I3(L, i, j, k), r = uf_find(par, p);
        if (root_block[r] < 0) root_block[r] = nb++;
        T->owner[p] = root_block[r];
      }
  T->nblock = nb;
  T->blk = calloc(nb, sizeof(blk3_t));
  int *count = calloc(nb, sizeof(int));
  for (size_t p = 0; p < nn; ++p)
    if (T->owner[p] >= 0) count[T->owner[p]]++;
  T->pool = malloc(sizeof(int) * 2 * (nn + 1));
  int off = 0;
  for (int b = 0; b < nb; ++b) {
    T->blk[b].node = T->pool + off;
    T->blk[b].parent = T->pool + nn + 1 + off;
    off += count[b];
  }
  /* per block: root = node with most in-block neighbours (first such in
     index order), then breadth-first order with parents */
  int *first = malloc(sizeof(int) * nb), *best = malloc(sizeof(int) * nb);
  for (int b = 0; b < nb; ++b) { first[b] = -1; best[b] = -1; }
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) {
        const int p = (int)I3(L, i, j, k), b = T->owner[p];
        int deg = 0;
        for (int d = 0; d < 6; ++d) {
          const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
          if (interior3(L, ii, jj, kk) && T->owner[I3(L, ii, jj, kk)] == b) ++deg;
        }
        if (best[b] < deg) { best[b] = deg; first[b] = p; }
      }
  char *seen = calloc(nn, 1);
  for (int b = 0; b < nb; ++b) {
    blk3_t *B = &T->blk[b];
    B->maxdeg = best[b];
    int head = 0, tail = 0;
    B->node[tail] = first[b]; B->parent[tail] = -1; ++tail;
    seen[first[b]] = 1;
    while (head < tail) {
      const int p = B->node[head];
      const int i = p % (L->nx + 1), j = (p / (L->nx + 1)) % (L->ny + 1), k = p / ((L->nx + 1) * (L->ny + 1));
      for (int d = 0; d < 6; ++d) {
        const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
        if (!interior3(L, ii, jj, kk)) continue;
        const int q = (int)I3(L, ii, jj, kk);
        if (T->owner[q] != b || seen[q]) continue;
        seen[q] = 1;
        B->node[tail] = q; B->parent[tail] = head; ++tail;
      }
      ++head;
    }
    B->n = tail;
    {
      const int p = B->node[0];
      const int i = p % (L->nx + 1), j = (p / (L->nx + 1)) % (L->ny + 1), k = p / ((L->nx + 1) * (L->ny + 1));
      int d2, d3;
      key3(L, sm, i, j, k, &d2, &d3);
      B->colour = ((d2 + d3) % 2 == 0) ? 0 : 1;
    }
  }
  free(seen); free(first); free(best); free(count); free(root_block); free(par);
  T->built = 1;
  return 0;
}

/* coefficient of row p towards its grid neighbour q */
static double coef_pq3(const lev3_t *L, int p, int q) {
  const int i = p % (L->nx + 1), j = (p / (L->nx + 1)) % (L->ny + 1), k = p / ((L->nx + 1) * (L->ny + 1));
  for (int d = 0; d < 6; ++d)
    if ((int)I3(L, i + DI[d], j + DJ[d], k + DK[d]) == q) return coef6(L, i, j, k, d);
  return 0.0;
}

static int lu3(int n, double *A, int *piv);
static void lu3_solve(int n, const double *A, const int *piv, double *b);

/* Exact solve of block b (Sec. 3: every node of the block at once, the
 * other nodes held fixed): right-hand sides with the neighbours outside the
 * block moved over, then Gaussian elimination on the tree from the leaves
 * to the root and substitution back.  Blocks that are not trees (the double
 * middle lines of a side with an odd number of intervals close loops) are
 * solved by dense LU instead. */
static int solve_block3(const lev3_t *L, const part3_t *T, int b, double *u, const double *f) {
  const blk3_t *B = &T->blk[b];
  const int n = B->n;
  int edges = 0;
  for (int s = 0; s < n; ++s) {
    const int p = B->node[s];
    const int i = p % (L->nx + 1), j = (p / (L->nx + 1)) % (L->ny + 1), k = p / ((L->nx + 1) * (L->ny + 1));
    for (int d = 1; d < 6; d += 2) {
      const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
      if (interior3(L, ii, jj, kk) && T->owner[I3(L, ii, jj, kk)] == b) ++edges;
    }
  }
  double *dg = malloc(sizeof(double) * n), *r = malloc(sizeof(double) * n);
  for (int s = 0; s < n; ++s) {
    const int p = B->node[s];
    const int i = p % (L->nx + 1), j = (p / (L->nx + 1)) % (L->ny + 1), k = p / ((L->nx + 1) * (L->ny + 1));
    dg[s] = centre3(L, i, j, k);
    double v = f[p];
    for (int d = 0; d < 6; ++d) {
      const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
      const size_t q = I3(L, ii, jj, kk);
      if (interior3(L, ii, jj, kk) && T->owner[q] == b) continue;
      v -= coef6(L, i, j, k, d) * u[q];
    }
    r[s] = v;
  }
  if (edges != n - 1) {
    /* dense: A x = r over the block's nodes in breadth-first order */
    double *A = calloc((size_t)n * n, sizeof(double));
    int *piv = malloc(sizeof(int) * n);
    for (int s = 0; s < n; ++s) {
      A[(size_t)s * n + s] = dg[s];
      for (int t = 0; t < n; ++t)
        if (t != s) A[(size_t)s * n + t] = coef_pq3(L, B->node[s], B->node[t]);
    }
    const int rc = lu3(n, A, piv);
    if (!rc) {
      lu3_solve(n, A, piv, r);
      for (int s = 0; s < n; ++s) u[B->node[s]] = r[s];
    }
    free(A); free(piv); free(dg); free(r);
    return rc;
  }
  /* leaves first: fold node s into its parent */
  for (int s = n - 1; s > 0; --s) {
    const int ps = B->parent[s], p = B->node[s], q = B->node[ps];
    const double a_sp = coef_pq3(L, p, q), a_ps = coef_pq3(L, q, p);
    dg[ps] -= a_ps * a_sp / dg[s];
    r[ps] -= a_ps * r[s] / dg[s];
  }
  double *x = malloc(sizeof(double) * n);
  x[0] = r[0] / dg[0];
  for (int s = 1; s < n; ++s) {
    const int ps = B->parent[s], p = B->node[s], q = B->node[ps];
    x[s] = (r[s] - coef_pq3(L, p, q) * x[ps]) / dg[s];
  }
  for (int s = 0; s < n; ++s) u[B->node[s]] = x[s];
  free(dg); free(r); free(x);
  return 0;
}

int o3_colour_pass(o3_problem *P, int lev, int sm, int colour, double *u, const double *f) {
  if (sm < 0 || sm >= O3_NMOTIF) return -1;
  if (build_part(P, lev, sm)) return -1;
  const part3_t *T = &P->part[lev][sm];
  /* the blocks of one colour are decoupled: any order, or at once */
  int bad = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
#endif
  for (int b = 0; b < T->nblock; ++b)
    if (T->blk[b].colour == colour && solve_block3(&P->lev[lev], T, b, u, f)) bad |= 1;
  return bad ? -1 : 0;
}

/* one relaxation: red pass, black pass; O3_ALT_TW is the alternating scheme
   of Sec. 3 applied in 3D (a tweed relaxation, then a wireframe one) and
   O3_TRIPLET the triplet of Sec. 7 (tweed, wireframe, complementary) */
int o3_smooth(o3_problem *P, int lev, int sm, double *u, const double *f) {
  if (sm == O3_ALT_TW) return o3_smooth(P, lev, O3_TWEED, u, f) || o3_smooth(P, lev, O3_WIREFRAME, u, f);
  if (sm == O3_TRIPLET)
    return o3_smooth(P, lev, O3_TWEED, u, f) || o3_smooth(P, lev, O3_WIREFRAME, u, f) ||
           o3_smooth(P, lev, O3_COMPLEMENTARY, u, f);
  return o3_colour_pass(P, lev, sm, 0, u, f) || o3_colour_pass(P, lev, sm, 1, u, f);
}

/* ------------------------------------------------------------ transfers -- */

static const double W1[3] = {0.25, 0.5, 0.25};

void o3_restrict(o3_problem *P, int lev, const double *d, double *fc) {
  const lev3_t *F = &P->lev[lev], *C = &P->lev[lev + 1];
  memset(fc, 0, sizeof(double) * nn3(C));
  for (int K = 1; K < C->nz; ++K)
    for (int J = 1; J < C->ny; ++J)
      for (int I = 1; I < C->nx; ++I) {
        double v = 0.0;
        for (int c = -1; c <= 1; ++c)
          for (int b = -1; b <= 1; ++b)
            for (int a = -1; a <= 1; ++a)
              v += W1[a + 1] * W1[b + 1] * W1[c + 1] * d[I3(F, 2 * I + a, 2 * J + b, 2 * K + c)];
        fc[I3(C, I, J, K)] = v;
      }
}

void o3_prolong_add(o3_problem *P, int lev, const double *uc, double *u) {
  const lev3_t *F = &P->lev[lev], *C = &P->lev[lev + 1];
  for (int k = 1; k < F->nz; ++k)
    for (int j = 1; j < F->ny; ++j)
      for (int i = 1; i < F->nx; ++i) {
        /* 1D: even index -> the coarse node, weight 1; odd -> its two
           coarse neighbours, weight 1/2 each */
        int ci[2], cj[2], ck[2], ni, nj, nk;
        double wi, wj, wk;
        if (i % 2 == 0) { ci[0] = i / 2; ni = 1; wi = 1.0; } else { ci[0] = (i - 1) / 2; ci[1] = (i + 1) / 2; ni = 2; wi = 0.5; }
        if (j % 2 == 0) { cj[0] = j / 2; nj = 1; wj = 1.0; } else { cj[0] = (j - 1) / 2; cj[1] = (j + 1) / 2; nj = 2; wj = 0.5; }
        if (k % 2 == 0) { ck[0] = k / 2; nk = 1; wk = 1.0; } else { ck[0] = (k - 1) / 2; ck[1] = (k + 1) / 2; nk = 2; wk = 0.5; }
        double v = 0.0;
        for (int c = 0; c < nk; ++c)
          for (int b = 0; b < nj; ++b)
            for (int a = 0; a < ni; ++a) v += uc[I3(C, ci[a], cj[b], ck[c])];
        u[I3(F, i, j, k)] += wi * wj * wk * v;
      }
}

/* ------------------------------------------------------ direct solvers --- */

static int lu3(int n, double *A, int *piv) {
  for (int c = 0; c < n; ++c) {
    int m = c;
    for (int r = c + 1; r < n; ++r) if (fabs(A[(size_t)r * n + c]) > fabs(A[(size_t)m * n + c])) m = r;
    if (A[(size_t)m * n + c] == 0.0) return -1;
    piv[c] = m;
    if (m != c)
      for (int q = 0; q < n; ++q) { double t = A[(size_t)c * n + q]; A[(size_t)c * n + q] = A[(size_t)m * n + q]; A[(size_t)m * n + q] = t; }
    for (int r = c + 1; r < n; ++r) {
      const double l = A[(size_t)r * n + c] / A[(size_t)c * n + c];
      A[(size_t)r * n + c] = l;
      for (int q = c + 1; q < n; ++q) A[(size_t)r * n + q] -= l * A[(size_t)c * n + q];
    }
  }
  return 0;
}
static void lu3_solve(int n, const double *A, const int *piv, double *b) {
  for (int c = 0; c < n; ++c) { const int m = piv[c]; if (m != c) { double t = b[c]; b[c] = b[m]; b[m] = t; } }
  for (int r = 0; r < n; ++r) for (int q = 0; q < r; ++q) b[r] -= A[(size_t)r * n + q] * b[q];
  for (int r = n - 1; r >= 0; --r) { for (int q = r + 1; q < n; ++q) b[r] -= A[(size_t)r * n + q] * b[q]; b[r] /= A[(size_t)r * n + r]; }
}

/* the interior system of a level, dense; unknown index
   ((k-1)(ny-1) + (j-1))(nx-1) + (i-1); boundary values move to rhs */
static void assemble3(const lev3_t *L, double *A, const double *u, const double *f, double *rhs) {
  const int mx = L->nx - 1, my = L->ny - 1, mz = L->nz - 1, n = mx * my * mz;
  if (A) memset(A, 0, sizeof(double) * (size_t)n * n);
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) {
        const int r = ((k - 1) * my + (j - 1)) * mx + (i - 1);
        if (A) A[(size_t)r * n + r] = centre3(L, i, j, k);
        double v = f ? f[I3(L, i, j, k)] : 0.0;
        for (int d = 0; d < 6; ++d) {
          const int ii = i + DI[d], jj = j + DJ[d], kk = k + DK[d];
          const double c = coef6(L, i, j, k, d);
          if (interior3(L, ii, jj, kk)) {
            if (A) A[(size_t)r * n + ((kk - 1) * my + (jj - 1)) * mx + (ii - 1)] = c;
          } else if (f) {
            v -= c * u[I3(L, ii, jj, kk)];
          }
        }
        if (rhs) rhs[r] = v;
      }
}

int o3_direct_solve(o3_problem *P, int lev, double *u, const double *f) {
  const lev3_t *L = &P->lev[lev];
  const int mx = L->nx - 1, my = L->ny - 1, mz = L->nz - 1, n = mx * my * mz;
  double *A = malloc(sizeof(double) * (size_t)n * n), *b = malloc(sizeof(double) * n);
  int *piv = malloc(sizeof(int) * n);
  assemble3(L, A, u, f, b);
  int rc = lu3(n, A, piv);
  if (!rc) {
    lu3_solve(n, A, piv, b);
    for (int k = 1; k < L->nz; ++k)
      for (int j = 1; j < L->ny; ++j)
        for (int i = 1; i < L->nx; ++i) u[I3(L, i, j, k)] = b[((k - 1) * my + (j - 1)) * mx + (i - 1)];
  }
  free(A); free(b); free(piv);
  return rc;
}

static int coarse3(o3_problem *P, double *u, const double *f) {
  const lev3_t *L = &P->lev[P->nlev - 1];
  const int mx = L->nx - 1, my = L->ny - 1, mz = L->nz - 1, n = mx * my * mz;
  if (!P->clu) {
    P->cn = n;
    P->clu = malloc(sizeof(double) * (size_t)n * n);
    P->cpiv = malloc(sizeof(int) * n);
    assemble3(L, P->clu, NULL, NULL, NULL);
    if (lu3(n, P->clu, P->cpiv)) return -1;
  }
  double *b = malloc(sizeof(double) * n);
  assemble3(L, NULL, u, f, b);
  lu3_solve(n, P->clu, P->cpiv, b);
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) u[I3(L, i, j, k)] = b[((k - 1) * my + (j - 1)) * mx + (i - 1)];
  free(b);
  return 0;
}

/* ---------------------------------------------------------- hierarchy --- */

o3_problem *o3_create(int nx, int ny, int nz, const double *x, const double *y, const double *z) {
  if (nx < 2 || ny < 2 || nz < 2) return NULL;
  o3_problem *P = calloc(1, sizeof(o3_problem));
  lev3_init(&P->lev[0], nx, ny, nz, x, y, z);
  int l = 0;
  while (l + 1 < O3_MAXLEV) {
    const lev3_t *F = &P->lev[l];
    if (F->nx % 2 || F->ny % 2 || F->nz % 2 || F->nx / 2 < 2 || F->ny / 2 < 2 || F->nz / 2 < 2 ||
        imax3(F->nx, imax3(F->ny, F->nz)) <= 8)
      break;
    const int cx = F->nx / 2, cy = F->ny / 2, cz = F->nz / 2;
    double *xc = malloc(sizeof(double) * (cx + 1)), *yc = malloc(sizeof(double) * (cy + 1)),
           *zc = malloc(sizeof(double) * (cz + 1));
    for (int i = 0; i <= cx; ++i) xc[i] = F->x[2 * i];
    for (int j = 0; j <= cy; ++j) yc[j] = F->y[2 * j];
    for (int k = 0; k <= cz; ++k) zc[k] = F->z[2 * k];
    lev3_init(&P->lev[l + 1], cx, cy, cz, xc, yc, zc);
    free(xc); free(yc); free(zc);
    ++l;
  }
  P->nlev = l + 1;
  for (int k = 0; k < P->nlev; ++k)
    for (int s = 0; s < 3; ++s) P->work[k][s] = calloc(nn3(&P->lev[k]), sizeof(double));
  return P;
}

void o3_destroy(o3_problem *P) {
  if (!P) return;
  for (int k = 0; k < O3_MAXLEV; ++k) {
    lev3_t *L = &P->lev[k];
    free(L->x); free(L->y); free(L->z); free(L->W); free(L->E); free(L->S); free(L->N); free(L->B); free(L->T);
    for (int sm = 0; sm < O3_NMOTIF; ++sm) { free(P->part[k][sm].blk); free(P->part[k][sm].owner); free(P->part[k][sm].pool); }
    for (int s = 0; s < 3; ++s) free(P->work[k][s]);
  }
  free(P->clu); free(P->cpiv);
  free(P);
}

int o3_num_levels(o3_problem *P) { return P->nlev; }
void o3_level_shape(o3_problem *P, int lev, int *nx, int *ny, int *nz) {
  *nx = P->lev[lev].nx; *ny = P->lev[lev].ny; *nz = P->lev[lev].nz;
}
void o3_level_coeffs(o3_problem *P, int lev, double *W, double *E, double *S, double *N, double *B, double *T) {
  const lev3_t *L = &P->lev[lev];
  memcpy(W, L->W, sizeof(double) * (L->nx + 1)); memcpy(E, L->E, sizeof(double) * (L->nx + 1));
  memcpy(S, L->S, sizeof(double) * (L->ny + 1)); memcpy(N, L->N, sizeof(double) * (L->ny + 1));
  memcpy(B, L->B, sizeof(double) * (L->nz + 1)); memcpy(T, L->T, sizeof(double) * (L->nz + 1));
}

/* block owner of every node (-1 off the interior) and the colour of every
   block; returns the number of blocks */
int o3_partition(o3_problem *P, int lev, int sm, int *owner, int *colour, int max_blocks) {
  if (sm < 0 || sm >= O3_NMOTIF) return -1;
  if (build_part(P, lev, sm)) return -1;
  const part3_t *T = &P->part[lev][sm];
  memcpy(owner, T->owner, sizeof(int) * nn3(&P->lev[lev]));
  for (int b = 0; b < T->nblock && b < max_blocks; ++b) colour[b] = T->blk[b].colour;
  return T->nblock;
}

int o3_block_solve(o3_problem *P, int lev, int sm, int b, double *u, const double *f) {
  if (sm < 0 || sm >= O3_NMOTIF) return -1;
  if (build_part(P, lev, sm)) return -1;
  if (b < 0 || b >= P->part[lev][sm].nblock) return -1;
  return solve_block3(&P->lev[lev], &P->part[lev][sm], b, u, f);
}

/* --------------------------------------------------------------- cycles -- */

static int cycle3(o3_problem *P, int sm, int nu1, int nu2, int lev, double *u, const double *f) {
  if (lev == P->nlev - 1) return coarse3(P, u, f);
  for (int s = 0; s < nu1; ++s) if (o3_smooth(P, lev, sm, u, f)) return -1;
  double *d = P->work[lev][2], *uc = P->work[lev + 1][0], *fc = P->work[lev + 1][1];
  o3_residual(P, lev, u, f, d);
  o3_restrict(P, lev, d, fc);
  memset(uc, 0, sizeof(double) * nn3(&P->lev[lev + 1]));
  if (cycle3(P, sm, nu1, nu2, lev + 1, uc, fc)) return -1;
  o3_prolong_add(P, lev, uc, u);
  for (int s = 0; s < nu2; ++s) if (o3_smooth(P, lev, sm, u, f)) return -1;
  return 0;
}

int o3_cycle(o3_problem *P, int sm, int nu1, int nu2, double *u, const double *f) {
  return cycle3(P, sm, nu1, nu2, 0, u, f);
}

/* V(nu1, nu2) cycles from u until ||f - L u|| / ||f - B g|| <= tol (Q5) or
   max_cycles; hist[k] = that ratio after cycle k (hist[0] before the first).
   Returns the number of cycles, -1 on failure. */
int o3_solve(o3_problem *P, int sm, int nu1, int nu2, double tol, int max_cycles, double *u, const double *f,
             double *hist, int cap) {
  const lev3_t *L = &P->lev[0];
  const size_t nn = nn3(L);
  double *d = malloc(sizeof(double) * nn), *g = malloc(sizeof(double) * nn);
  for (size_t p = 0; p < nn; ++p) g[p] = u[p];
  for (int k = 1; k < L->nz; ++k)
    for (int j = 1; j < L->ny; ++j)
      for (int i = 1; i < L->nx; ++i) g[I3(L, i, j, k)] = 0.0;
  o3_residual(P, 0, g, f, d);
  double fn = sqrt(sumsq_interior(L, d));
  o3_residual(P, 0, u, f, d);
  double s = sumsq_interior(L, d);
  if (fn == 0.0) fn = sqrt(s) > 0.0 ? sqrt(s) : 1.0;
  double rel = sqrt(s) / fn;
  if (cap > 0) hist[0] = rel;
  int k = 0;
  while (rel > tol && k < max_cycles) {
    if (o3_cycle(P, sm, nu1, nu2, u, f)) { free(d); free(g); return -1; }
    ++k;
    o3_residual(P, 0, u, f, d);
    rel = sqrt(sumsq_interior(L, d)) / fn;
    if (k < cap) hist[k] = rel;
    if (!isfinite(rel)) break;
  }
  free(d); free(g);
  return k;
}
