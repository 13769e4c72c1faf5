/*
 * mg_oracle.c -- plain, slow, FP64 CPU oracle for tweed / wireframe multigrid
 * (Bewley, Mashayek, Cavaglieri & Luchini, "Tweed and wireframe: accelerated
 * relaxation algorithms for multigrid solution of elliptic PDEs on stretched
 * structured grids", arXiv:2110.08389).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may link, load or
 * call this file; only the tests, the package smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header or table with the
 * CUDA path.
 *
 * Everything is written from the paper's definitions, in the paper's order:
 *   - operator and coefficients ............ Sec. 2, Eq. (prob:DP) and the W/E/S/N
 *                                            definitions that follow it
 *   - block partitions ...................... Sec. 3 (tweed: Fig. 4/6 text;
 *                                            wireframe: Fig. 5/7 text), Sec. 2
 *                                            (checkerboard, zebra, alt-zebra)
 *   - block solvers ......................... Sec. 3: Thomas, m-legged Thomas
 *                                            (Eq. mLThomas), circulant Thomas
 *                                            (Eq. CircTri), pointwise relaxation
 *   - restriction / prolongation ............ Sec. 4 (half weighting, full
 *                                            weighting, bilinear interpolation)
 *   - V-cycle, steps (1)-(6) ................ Sec. 4
 *   - two-grid operator ..................... Sec. 5, Eq. (Mh2h)
 *
 * Readings where the paper is silent or garbled:
 *   R1  nodes are 0-based, i = 0..nx, j = 0..ny, boundary at 0 and nx / ny;
 *       x is the fast index of every array: a[j*(nx+1)+i].
 *   R2  the S-term of Eq. (prob:DP) is S_j u_{i,j-1} (the printed "u_{j-1,j}"
 *       is a typo).
 *   R3  tweed block = connected set of interior nodes with equal
 *       max(d_x, d_y), d_x = min(i, nx-i), d_y = min(j, ny-j); wireframe block
 *       = connected set with equal min(d_x, d_y); colour red when that
 *       distance is odd (corners red, outer ring red).
 *   R4  checkerboard red = (i+j) even; zebra red = odd line index; red is
 *       relaxed first; alt-zebra = x-zebra step then y-zebra step; alt
 *       tweed/wireframe = tweed step then wireframe step; post-smoothing uses
 *       the same order as pre-smoothing.
 *   R5  coarsening stops once max(nx,ny) <= 8 (or a side is odd or would drop
 *       below 2 intervals); the coarsest level is solved by dense LU.
 *   R6  the restriction/prolongation weights are the index-based ones printed
 *       in Sec. 4, applied to the pointwise defect; coarse operators are
 *       rediscretised on the subsampled coordinates.
 *   R11 the stop test of Sec. 4 step (6) ("sufficiently small") is
 *       ||f - L u||_2 / ||f - B g||_2 <= tol over interior nodes, f - B g the
 *       right-hand side of the interior system (f when the boundary data g
 *       vanish).
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXLEV 32

enum { SM_CHECKER = 0, SM_ZEBRA_X = 1, SM_ZEBRA_Y = 2, SM_ALT_ZEBRA = 3,
       SM_TWEED = 4, SM_WIREFRAME = 5, SM_ALT_TW = 6 };
enum { BT_POINT = 0, BT_PATH = 1, BT_CYCLE = 2, BT_STAR = 3 };
enum { RS_HW = 0, RS_FW = 1 };

typedef struct {
  int nx, ny;
  double *x, *y;           /* coordinates, nx+1 and ny+1 entries            */
  double *W, *E, *S, *N;   /* Sec. 2 coefficients (0 at boundary indices)   */
} level_t;

typedef struct {
  int type, colour, n;     /* n nodes in node[], in solve order             */
  int *node;
  int nleg;                /* star: node[0] is the junction; leg l occupies  */
  int leg_off[8], leg_len[8]; /* node[leg_off..], ordered tip -> junction   */
} block_t;

typedef struct {
  int built, nblock;
  block_t *blk;
  int *owner;              /* block index of every node, -1 on the boundary */
  int *pool;               /* storage behind every block's node[]           */
} partition_t;

typedef struct {
  int nlev;
  level_t lev[OR_MAXLEV];            /* lev[0] is the finest grid           */
  partition_t part[OR_MAXLEV][7];    /* only base smoothers 0,1,2,4,5 used  */
  /* dense LU of the coarsest level (partial pivoting)                       */
  int cn; double *clu; int *cpiv;
  /* banded LU of level 1 for the exact-coarse-solve two-grid operator      */
  int bn, bw; double *band;
  double *work[OR_MAXLEV][3];        /* per-level scratch: u, f, defect     */
} or_problem;

static inline int ID(const level_t *L, int i, int j) { return j * (L->nx + 1) + i; }
static inline int imin(int a, int b) { return a < b ? a : b; }
static inline int imax(int a, int b) { return a > b ? a : b; }

/* ---------------------------------------------------------------- grid --- */

/* Sec. 2: W_i = 1/(dx_i dx_{i-1/2}), E_i = 1/(dx_i dx_{i+1/2}) with
 * dx_{i-1/2} = x_i - x_{i-1} and dx_i = (x_{i+1} - x_{i-1})/2.             */
static void coeff_1d(int n, const double *x, double *lo, double *hi) {
  for (int i = 0; i <= n; ++i) { lo[i] = 0.0; hi[i] = 0.0; }
  for (int i = 1; i < n; ++i) {
    double dm = x[i] - x[i - 1];
    double dp = x[i + 1] - x[i];
    double dc = 0.5 * (x[i + 1] - x[i - 1]);
    lo[i] = 1.0 / (dc * dm);
    hi[i] = 1.0 / (dc * dp);
  }
}

static void level_init(level_t *L, int nx, int ny, const double *x, const double *y) {
  L->nx = nx; L->ny = ny;
  L->x = malloc(sizeof(double) * (nx + 1)); L->y = malloc(sizeof(double) * (ny + 1));
  memcpy(L->x, x, sizeof(double) * (nx + 1)); memcpy(L->y, y, sizeof(double) * (ny + 1));
  L->W = malloc(sizeof(double) * (nx + 1)); L->E = malloc(sizeof(double) * (nx + 1));
  L->S = malloc(sizeof(double) * (ny + 1)); L->N = malloc(sizeof(double) * (ny + 1));
  coeff_1d(nx, x, L->W, L->E);
  coeff_1d(ny, y, L->S, L->N);
}

/* Operator coefficient in row p=(i,j) for the neighbour one step away in
 * direction (di,dj): W_i, E_i, S_j or N_j.                                  */
static double coef_dir(const level_t *L, int i, int j, int di, int dj) {
  if (di == -1) return L->W[i];
  if (di == +1) return L->E[i];
  if (dj == -1) return L->S[j];
  return L->N[j];
}
static double coef_centre(const level_t *L, int i, int j) {
  return -(L->W[i] + L->E[i] + L->S[j] + L->N[j]);
}

/* ------------------------------------------------------- operator, norms -- */

/* (L u)_{ij} of Eq. (prob:DP) at interior nodes; 0 on the boundary.         */
void or_apply(or_problem *P, int lev, const double *u, double *out) {
  level_t *L = &P->lev[lev];
  int nx = L->nx, ny = L->ny;
  memset(out, 0, sizeof(double) * (nx + 1) * (ny + 1));
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i)
      out[ID(L, i, j)] = L->W[i] * u[ID(L, i - 1, j)] + L->E[i] * u[ID(L, i + 1, j)] +
                         L->S[j] * u[ID(L, i, j - 1)] + L->N[j] * u[ID(L, i, j + 1)] +
                         coef_centre(L, i, j) * u[ID(L, i, j)];
}

/* Defect d = f - L u at interior nodes (Sec. 4 step (3)); 0 on the boundary. */
void or_residual(or_problem *P, int lev, const double *u, const double *f, double *d) {
  level_t *L = &P->lev[lev];
  or_apply(P, lev, u, d);
  for (int j = 0; j <= L->ny; ++j)
    for (int i = 0; i <= L->nx; ++i) {
      int p = ID(L, i, j);
      d[p] = (i == 0 || j == 0 || i == L->nx || j == L->ny) ? 0.0 : f[p] - d[p];
    }
}

/* Sum of squares and max-abs over interior nodes.                            */
void or_norms(or_problem *P, int lev, const double *a, double *sumsq, double *maxabs) {
  level_t *L = &P->lev[lev];
  double s = 0.0, m = 0.0;
  for (int j = 1; j < L->ny; ++j)
    for (int i = 1; i < L->nx; ++i) {
      double v = a[ID(L, i, j)];
      s += v * v;
      if (fabs(v) > m) m = fabs(v);
    }
  *sumsq = s; *maxabs = m;
}

/* --------------------------------------------------------- partitions ---- */

/* Block key and colour of interior node (i,j) for a base smoother (R3, R4).
 * colour 0 = red (relaxed first), 1 = black.                                */
static int block_key(const level_t *L, int sm, int i, int j, int *colour) {
  int dx = imin(i, L->nx - i), dy = imin(j, L->ny - j), k;
  switch (sm) {
    case SM_CHECKER: *colour = ((i + j) % 2 == 0) ? 0 : 1; return ID(L, i, j);
    case SM_ZEBRA_X: *colour = (j % 2 == 1) ? 0 : 1; return j;
    case SM_ZEBRA_Y: *colour = (i % 2 == 1) ? 0 : 1; return i;
    case SM_TWEED:   k = imax(dx, dy); *colour = (k % 2 == 1) ? 0 : 1; return k;
    case SM_WIREFRAME: k = imin(dx, dy); *colour = (k % 2 == 1) ? 0 : 1; return k;
  }
  return -1;
}

static const int DI[4] = {-1, 1, 0, 0}, DJ[4] = {0, 0, -1, 1};

static int in_block_nbrs(const level_t *L, const int *owner, int p, int b, int *nb) {
  int nx = L->nx, i = p % (nx + 1), j = p / (nx + 1), c = 0;
  for (int d = 0; d < 4; ++d) {
    int q = ID(L, i + DI[d], j + DJ[d]);
    if (owner[q] == b) nb[c++] = q;
  }
  return c;
}

/* Connected components of equal key (4-neighbour adjacency), then the shape
 * of each component: point, path, closed cycle or star (one branch node).   */
static int build_partition(or_problem *P, int lev, int sm) {
  partition_t *T = &P->part[lev][sm];
  if (T->built) return 0;
  level_t *L = &P->lev[lev];
  int nx = L->nx, ny = L->ny, nn = (nx + 1) * (ny + 1);
  int *key = malloc(sizeof(int) * nn), *col = malloc(sizeof(int) * nn);
  T->owner = malloc(sizeof(int) * nn);
  T->pool = malloc(sizeof(int) * nn);
  int *queue = malloc(sizeof(int) * nn), *deg = malloc(sizeof(int) * nn);
  for (int p = 0; p < nn; ++p) { T->owner[p] = -1; key[p] = -1; col[p] = -1; }
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i) key[ID(L, i, j)] = block_key(L, sm, i, j, &col[ID(L, i, j)]);
  int cap = 64, nb = 0, used = 0;
  T->blk = malloc(sizeof(block_t) * cap);
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      int s = ID(L, i, j);
      if (T->owner[s] >= 0) continue;
      if (nb == cap) { cap *= 2; T->blk = realloc(T->blk, sizeof(block_t) * cap); }
      int head = 0, tail = 0;
      queue[tail++] = s; T->owner[s] = nb;
      while (head < tail) {
        int p = queue[head++], pi = p % (nx + 1), pj = p / (nx + 1);
        for (int d = 0; d < 4; ++d) {
          int qi = pi + DI[d], qj = pj + DJ[d];
          if (qi < 1 || qj < 1 || qi >= nx || qj >= ny) continue;
          int q = ID(L, qi, qj);
          if (T->owner[q] < 0 && key[q] == key[s]) { T->owner[q] = nb; queue[tail++] = q; }
        }
      }
      block_t *B = &T->blk[nb];
      memset(B, 0, sizeof(*B));
      B->n = tail; B->colour = col[s]; B->node = T->pool + used; used += tail;
      /* shape analysis */
      int nb_[4], n1 = 0, n3 = 0, hub = -1;
      for (int t = 0; t < tail; ++t) {
        deg[queue[t]] = in_block_nbrs(L, T->owner, queue[t], nb, nb_);
        if (deg[queue[t]] == 1) ++n1;
        if (deg[queue[t]] >= 3) { ++n3; hub = queue[t]; }
      }
      if (tail == 1) { B->type = BT_POINT; B->node[0] = s; }
      else if (n3 == 0 && n1 == 2) {                 /* path: walk from an end */
        int start = -1;
        for (int t = 0; t < tail; ++t) if (deg[queue[t]] == 1 && (start < 0 || queue[t] < start)) start = queue[t];
        B->type = BT_PATH;
        int prev = -1, cur = start;
        for (int t = 0; t < tail; ++t) {
          B->node[t] = cur;
          int c = in_block_nbrs(L, T->owner, cur, nb, nb_), nxt = -1;
          for (int e = 0; e < c; ++e) if (nb_[e] != prev) nxt = nb_[e];
          prev = cur; cur = nxt;
        }
      } else if (n3 == 0 && n1 == 0) {               /* closed cycle */
        int start = queue[0];
        for (int t = 0; t < tail; ++t) if (queue[t] < start) start = queue[t];
        B->type = BT_CYCLE;
        int c = in_block_nbrs(L, T->owner, start, nb, nb_);
        int nxt = nb_[0];                 /* first step: smaller-index neighbour */
        for (int e = 1; e < c; ++e) if (nb_[e] < nxt) nxt = nb_[e];
        int prev = start, cur = nxt;
        B->node[0] = start;
        for (int t = 1; t < tail; ++t) {
          B->node[t] = cur;
          int c2 = in_block_nbrs(L, T->owner, cur, nb, nb_), n2 = -1;
          for (int e = 0; e < c2; ++e) if (nb_[e] != prev) n2 = nb_[e];
          prev = cur; cur = n2;
        }
      } else if (n3 == 1) {                          /* star: legs into hub */
        B->type = BT_STAR;
        B->node[0] = hub;
        int c = in_block_nbrs(L, T->owner, hub, nb, nb_), pos = 1;
        B->nleg = c;
        for (int l = 0; l < c; ++l) {
          /* walk from the hub outward, then store reversed (tip -> hub) */
          int tmp0 = pos, prev = hub, cur = nb_[l], len = 0;
          while (cur >= 0) {
            B->node[pos + len++] = cur;
            int nb2[4], c2 = in_block_nbrs(L, T->owner, cur, nb, nb2), nxt = -1;
            for (int e = 0; e < c2; ++e) if (nb2[e] != prev) nxt = nb2[e];
            if (deg[cur] == 1) nxt = -1;
            prev = cur; cur = nxt;
          }
          for (int a = 0, z = len - 1; a < z; ++a, --z) {
            int t = B->node[tmp0 + a]; B->node[tmp0 + a] = B->node[tmp0 + z]; B->node[tmp0 + z] = t;
          }
          B->leg_off[l] = tmp0; B->leg_len[l] = len; pos += len;
        }
        if (pos != tail) { fprintf(stderr, "oracle: malformed star block\n"); return -1; }
      } else {
        fprintf(stderr, "oracle: unsupported block shape (n=%d, ends=%d, branches=%d)\n", tail, n1, n3);
        return -1;
      }
      ++nb;
    }
  T->nblock = nb; T->built = 1;
  free(key); free(col); free(queue); free(deg);
  return 0;
}

/* ------------------------------------------------------ block solvers ---- */

/* In-block coefficient between two adjacent nodes p -> q (row p).          */
static double coef_pq(const level_t *L, int p, int q) {
  int nx = L->nx, pi = p % (nx + 1), pj = p / (nx + 1), qi = q % (nx + 1), qj = q / (nx + 1);
  return coef_dir(L, pi, pj, qi - pi, qj - pj);
}

/* Right-hand side of row p inside block b: f_p minus every neighbour that is
 * not an unknown of the block, at its current value (Sec. 3: "solved exactly
 * ... while holding the values of the unknowns at the [other] points fixed").*/
static double block_rhs(const level_t *L, const int *owner, int b, int p,
                        const double *u, const double *f) {
  int nx = L->nx, i = p % (nx + 1), j = p / (nx + 1);
  double r = f[p];
  for (int d = 0; d < 4; ++d) {
    int q = ID(L, i + DI[d], j + DJ[d]);
    if (owner[q] != b) r -= coef_dir(L, i, j, DI[d], DJ[d]) * u[q];
  }
  return r;
}

static int adjacent(const level_t *L, int p, int q) {
  int nx = L->nx, pi = p % (nx + 1), pj = p / (nx + 1), qi = q % (nx + 1), qj = q / (nx + 1);
  return abs(pi - qi) + abs(pj - qj) == 1;
}

/* Thomas algorithm (Sec. 3): a_t x_{t-1} + b_t x_t + c_t x_{t+1} = r_t.
 * Forward elimination then back substitution; a_0 and c_{m-1} are unused. */
static void thomas(int m, const double *a, const double *b, const double *c, const double *r,
                   double *x, double *cp, double *rp) {
  cp[0] = c[0] / b[0];
  rp[0] = r[0] / b[0];
  for (int t = 1; t < m; ++t) {
    double den = b[t] - a[t] * cp[t - 1];
    cp[t] = c[t] / den;
    rp[t] = (r[t] - a[t] * rp[t - 1]) / den;
  }
  x[m - 1] = rp[m - 1];
  for (int t = m - 2; t >= 0; --t) x[t] = rp[t] - cp[t] * x[t + 1];
}

typedef struct { double *a, *b, *c, *r, *x, *cp, *rp, *z; int cap; } scratch_t;
static void scratch_need(scratch_t *s, int m) {
  if (m <= s->cap) return;
  s->cap = m;
  s->a = realloc(s->a, sizeof(double) * m); s->b = realloc(s->b, sizeof(double) * m);
  s->c = realloc(s->c, sizeof(double) * m); s->r = realloc(s->r, sizeof(double) * m);
  s->x = realloc(s->x, sizeof(double) * m); s->cp = realloc(s->cp, sizeof(double) * m);
  s->rp = realloc(s->rp, sizeof(double) * m); s->z = realloc(s->z, sizeof(double) * m);
}
/* one scratch per thread: the blocks of a colour pass may be solved by
 * several threads (OpenMP builds); the arithmetic of each block is the same */
static _Thread_local scratch_t g_scr;

/* Exact solve of one block, written into u (Sec. 3).                        */
static void solve_block(const level_t *L, const partition_t *T, int b, double *u, const double *f) {
  const block_t *B = &T->blk[b];
  const int *nd = B->node;
  int m = B->n;
  scratch_need(&g_scr, m + 2);
  double *a = g_scr.a, *bb = g_scr.b, *c = g_scr.c, *r = g_scr.r, *x = g_scr.x;
  int nx = L->nx;
  if (B->type == BT_POINT) {                       /* pointwise relaxation */
    int p = nd[0];
    u[p] = block_rhs(L, T->owner, b, p, u, f) / coef_centre(L, p % (nx + 1), p / (nx + 1));
    return;
  }
  if (B->type == BT_PATH) {                        /* Thomas along the path */
    for (int t = 0; t < m; ++t) {
      int p = nd[t];
      a[t] = t > 0 ? coef_pq(L, p, nd[t - 1]) : 0.0;
      c[t] = t < m - 1 ? coef_pq(L, p, nd[t + 1]) : 0.0;
      bb[t] = coef_centre(L, p % (nx + 1), p / (nx + 1));
      r[t] = block_rhs(L, T->owner, b, p, u, f);
    }
    thomas(m, a, bb, c, r, x, g_scr.cp, g_scr.rp);
    for (int t = 0; t < m; ++t) u[nd[t]] = x[t];
    return;
  }
  if (B->type == BT_CYCLE) {
    /* Circulant tridiagonal system, Eq. (CircTri): row t couples x_{t-1} and
     * x_{t+1} cyclically.  Solved as in the periodic Thomas method: x_{m-1}
     * is kept as a parameter, the open chain x_0..x_{m-2} is solved for two
     * right-hand sides (the actual one, and the response to x_{m-1} = 1), and
     * the last row fixes x_{m-1}.                                           */
    for (int t = 0; t < m; ++t) {
      int p = nd[t];
      a[t] = coef_pq(L, p, nd[(t + m - 1) % m]);
      c[t] = coef_pq(L, p, nd[(t + 1) % m]);
      bb[t] = coef_centre(L, p % (nx + 1), p / (nx + 1));
      r[t] = block_rhs(L, T->owner, b, p, u, f);
    }
    int k = m - 1;                                  /* open chain length */
    double *y = x, *z = g_scr.z;
    double *rr = malloc(sizeof(double) * k), *ww = malloc(sizeof(double) * k);
    for (int t = 0; t < k; ++t) { rr[t] = r[t]; ww[t] = 0.0; }
    ww[0] -= a[0];                                  /* coupling of row 0 to x_{m-1}   */
    ww[k - 1] -= c[k - 1];                          /* coupling of row m-2 to x_{m-1} */
    thomas(k, a, bb, c, rr, y, g_scr.cp, g_scr.rp);
    thomas(k, a, bb, c, ww, z, g_scr.cp, g_scr.rp);
    double xl = (r[k] - c[k] * y[0] - a[k] * y[k - 1]) / (bb[k] + c[k] * z[0] + a[k] * z[k - 1]);
    for (int t = 0; t < k; ++t) u[nd[t]] = y[t] + xl * z[t];
    u[nd[k]] = xl;
    free(rr); free(ww);
    return;
  }
  /* BT_STAR: m-legged Thomas, Eq. (mLThomas).  Each leg is swept from its tip
   * towards the branch point, the branch-point row is solved, and the legs
   * are back-substituted outward.                                          */
  int hub = nd[0], hi = hub % (nx + 1), hj = hub / (nx + 1);
  double num = block_rhs(L, T->owner, b, hub, u, f);   /* r_centre          */
  double den = coef_centre(L, hi, hj);                 /* d_{m+1}           */
  double *cp = g_scr.cp, *rp = g_scr.rp;
  for (int l = 0; l < B->nleg; ++l) {
    int off = B->leg_off[l], len = B->leg_len[l];
    for (int t = 0; t < len; ++t) {
      int p = nd[off + t];
      double at = t > 0 ? coef_pq(L, p, nd[off + t - 1]) : 0.0;
      int nxt = t < len - 1 ? nd[off + t + 1] : hub;   /* c_p couples x_centre */
      double ct = coef_pq(L, p, nxt);
      double bt = coef_centre(L, p % (nx + 1), p / (nx + 1));
      double rt = block_rhs(L, T->owner, b, p, u, f);
      double dd = t > 0 ? bt - at * cp[off + t - 1] : bt;
      cp[off + t] = ct / dd;
      rp[off + t] = (t > 0 ? rt - at * rp[off + t - 1] : rt) / dd;
    }
    int pl = nd[off + len - 1];                        /* x_p of this leg   */
    double dl = coef_pq(L, hub, pl);                   /* d_l               */
    num -= dl * rp[off + len - 1];
    den -= dl * cp[off + len - 1];
  }
  double xc = num / den;
  u[hub] = xc;
  for (int l = 0; l < B->nleg; ++l) {
    int off = B->leg_off[l], len = B->leg_len[l];
    double xn = xc;
    for (int t = len - 1; t >= 0; --t) {
      xn = rp[off + t] - cp[off + t] * xn;
      u[nd[off + t]] = xn;
    }
  }
}

/* ------------------------------------------------------------ smoothers -- */

static int base_pass(or_problem *P, int lev, int sm, int colour, double *u, const double *f) {
  if (build_partition(P, lev, sm)) return -1;
  partition_t *T = &P->part[lev][sm];
  /* the blocks of one colour are decoupled (Sec. 3): each reads only nodes of
     the other colour and writes only its own, so they may run in any order
     or at once, with the same result */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16)
#endif
  for (int b = 0; b < T->nblock; ++b)
    if (T->blk[b].colour == colour) solve_block(&P->lev[lev], T, b, u, f);
  return 0;
}

/* One colour pass of a base smoother (colour 0 = red, 1 = black).           */
int or_colour_pass(or_problem *P, int lev, int sm, int colour, double *u, const double *f) {
  return base_pass(P, lev, sm, colour, u, f);
}

/* One relaxation step: red pass then black pass (R4); the alternating
 * schemes do one step of each of their two smoothers.                      */
int or_smooth(or_problem *P, int lev, int sm, double *u, const double *f) {
  if (sm == SM_ALT_ZEBRA) return or_smooth(P, lev, SM_ZEBRA_X, u, f) || or_smooth(P, lev, SM_ZEBRA_Y, u, f);
  if (sm == SM_ALT_TW) return or_smooth(P, lev, SM_TWEED, u, f) || or_smooth(P, lev, SM_WIREFRAME, u, f);
  return base_pass(P, lev, sm, 0, u, f) || base_pass(P, lev, sm, 1, u, f);
}

/* ------------------------------------------------------------ transfers -- */

/* Sec. 4 restriction of the defect d (level lev) to f (level lev+1).        */
void or_restrict(or_problem *P, int lev, int kind, const double *d, double *fc) {
  level_t *F = &P->lev[lev], *C = &P->lev[lev + 1];
  memset(fc, 0, sizeof(double) * (C->nx + 1) * (C->ny + 1));
  for (int J = 1; J < C->ny; ++J)
    for (int I = 1; I < C->nx; ++I) {
      int i = 2 * I, j = 2 * J;
      double edge = d[ID(F, i - 1, j)] + d[ID(F, i, j - 1)] + d[ID(F, i + 1, j)] + d[ID(F, i, j + 1)];
      double v;
      if (kind == RS_HW) {
        v = 0.5 * d[ID(F, i, j)] + 0.125 * edge;
      } else {
        double corner = d[ID(F, i - 1, j - 1)] + d[ID(F, i + 1, j - 1)] +
                        d[ID(F, i - 1, j + 1)] + d[ID(F, i + 1, j + 1)];
        v = 0.25 * d[ID(F, i, j)] + 0.125 * edge + 0.0625 * corner;
      }
      fc[ID(C, I, J)] = v;
    }
}

/* Sec. 4 bilinear prolongation of the coarse correction uc (level lev+1),
 * added to u at the interior nodes of level lev (step (5)).                 */
void or_prolong_add(or_problem *P, int lev, const double *uc, double *u) {
  level_t *F = &P->lev[lev], *C = &P->lev[lev + 1];
  for (int j = 1; j < F->ny; ++j)
    for (int i = 1; i < F->nx; ++i) {
      double v;
      if (i % 2 == 0 && j % 2 == 0) v = uc[ID(C, i / 2, j / 2)];
      else if (i % 2 == 0) v = 0.5 * (uc[ID(C, i / 2, (j - 1) / 2)] + uc[ID(C, i / 2, (j + 1) / 2)]);
      else if (j % 2 == 0) v = 0.5 * (uc[ID(C, (i - 1) / 2, j / 2)] + uc[ID(C, (i + 1) / 2, j / 2)]);
      else v = 0.25 * (uc[ID(C, (i - 1) / 2, (j - 1) / 2)] + uc[ID(C, (i + 1) / 2, (j - 1) / 2)] +
                       uc[ID(C, (i - 1) / 2, (j + 1) / 2)] + uc[ID(C, (i + 1) / 2, (j + 1) / 2)]);
      u[ID(F, i, j)] += v;
    }
}

/* ------------------------------------------------------ direct solvers --- */

/* Assemble the interior system of level lev densely (unknown index
 * (j-1)(nx-1)+(i-1)); boundary values of u move to the right-hand side.     */
static void assemble_dense(const level_t *L, double *A, const double *u, const double *f, double *rhs) {
  int nx = L->nx, ny = L->ny, n = (nx - 1) * (ny - 1);
  memset(A, 0, sizeof(double) * n * n);
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      int row = (j - 1) * (nx - 1) + (i - 1);
      A[row * n + row] = coef_centre(L, i, j);
      if (rhs) rhs[row] = f[ID(L, i, j)];
      for (int d = 0; d < 4; ++d) {
        int qi = i + DI[d], qj = j + DJ[d];
        double cf = coef_dir(L, i, j, DI[d], DJ[d]);
        if (qi < 1 || qj < 1 || qi >= nx || qj >= ny) { if (rhs) rhs[row] -= cf * u[ID(L, qi, qj)]; }
        else A[row * n + (qj - 1) * (nx - 1) + (qi - 1)] = cf;
      }
    }
}

/* Gaussian elimination with partial pivoting, in place.                    */
static int lu_factor(int n, double *A, int *piv) {
  for (int k = 0; k < n; ++k) {
    int p = k; double mx = fabs(A[k * n + k]);
    for (int r = k + 1; r < n; ++r) if (fabs(A[r * n + k]) > mx) { mx = fabs(A[r * n + k]); p = r; }
    if (mx == 0.0) return -1;
    piv[k] = p;
    if (p != k) for (int c = 0; c < n; ++c) { double t = A[k * n + c]; A[k * n + c] = A[p * n + c]; A[p * n + c] = t; }
    for (int r = k + 1; r < n; ++r) {
      double l = A[r * n + k] / A[k * n + k];
      A[r * n + k] = l;
      for (int c = k + 1; c < n; ++c) A[r * n + c] -= l * A[k * n + c];
    }
  }
  return 0;
}
static void lu_solve(int n, const double *A, const int *piv, double *b) {
  for (int k = 0; k < n; ++k) { int p = piv[k]; if (p != k) { double t = b[k]; b[k] = b[p]; b[p] = t; } }
  for (int r = 1; r < n; ++r) for (int c = 0; c < r; ++c) b[r] -= A[r * n + c] * b[c];
  for (int r = n - 1; r >= 0; --r) { for (int c = r + 1; c < n; ++c) b[r] -= A[r * n + c] * b[c]; b[r] /= A[r * n + r]; }
}

/* Direct solution of the whole level-lev system by dense LU (used as the
 * reference "plain definition" on small grids and at the coarsest level).  */
int or_direct_solve(or_problem *P, int lev, double *u, const double *f) {
  level_t *L = &P->lev[lev];
  int nx = L->nx, ny = L->ny, n = (nx - 1) * (ny - 1);
  if (n <= 0) return 0;
  double *A = malloc(sizeof(double) * n * n), *b = malloc(sizeof(double) * n);
  int *piv = malloc(sizeof(int) * n);
  assemble_dense(L, A, u, f, b);
  int rc = lu_factor(n, A, piv);
  if (!rc) {
    lu_solve(n, A, piv, b);
    for (int j = 1; j < ny; ++j) for (int i = 1; i < nx; ++i) u[ID(L, i, j)] = b[(j - 1) * (nx - 1) + (i - 1)];
  }
  free(A); free(b); free(piv);
  return rc;
}

static int coarse_solve(or_problem *P, double *u, const double *f) {
  int lev = P->nlev - 1;
  level_t *L = &P->lev[lev];
  int nx = L->nx, ny = L->ny, n = (nx - 1) * (ny - 1);
  if (n <= 0) return 0;
  if (!P->clu) {
    P->cn = n; P->clu = malloc(sizeof(double) * n * n); P->cpiv = malloc(sizeof(int) * n);
    assemble_dense(L, P->clu, u, f, NULL);
    if (lu_factor(n, P->clu, P->cpiv)) return -1;
  }
  double *b = malloc(sizeof(double) * n);
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      int row = (j - 1) * (nx - 1) + (i - 1);
      b[row] = f[ID(L, i, j)];
      if (i == 1) b[row] -= L->W[i] * u[ID(L, 0, j)];
      if (i == nx - 1) b[row] -= L->E[i] * u[ID(L, nx, j)];
      if (j == 1) b[row] -= L->S[j] * u[ID(L, i, 0)];
      if (j == ny - 1) b[row] -= L->N[j] * u[ID(L, i, ny)];
    }
  lu_solve(n, P->clu, P->cpiv, b);
  for (int j = 1; j < ny; ++j) for (int i = 1; i < nx; ++i) u[ID(L, i, j)] = b[(j - 1) * (nx - 1) + (i - 1)];
  free(b);
  return 0;
}

/* Banded LU (no pivoting; -L is a diagonally dominant M-matrix) of level 1,
 * used for the exact coarse solve of the two-grid operator (Sec. 5).        */
static int band_factor(or_problem *P) {
  level_t *L = &P->lev[1];
  int nx = L->nx, ny = L->ny, n = (nx - 1) * (ny - 1), w = nx - 1, ld = 2 * w + 1;
  P->bn = n; P->bw = w;
  P->band = calloc((size_t)n * ld, sizeof(double));
#define BA(r, c) P->band[(size_t)(r) * ld + ((c) - (r) + w)]
  for (int j = 1; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      int row = (j - 1) * (nx - 1) + (i - 1);
      BA(row, row) = coef_centre(L, i, j);
      for (int d = 0; d < 4; ++d) {
        int qi = i + DI[d], qj = j + DJ[d];
        if (qi < 1 || qj < 1 || qi >= nx || qj >= ny) continue;
        BA(row, (qj - 1) * (nx - 1) + (qi - 1)) = coef_dir(L, i, j, DI[d], DJ[d]);
      }
    }
  for (int k = 0; k < n; ++k) {
    double pv = BA(k, k);
    if (pv == 0.0) return -1;
    for (int r = k + 1; r <= imin(n - 1, k + w); ++r) {
      double l = BA(r, k) / pv;
      if (l == 0.0) continue;
      BA(r, k) = l;
      for (int c = k + 1; c <= imin(n - 1, k + w); ++c) BA(r, c) -= l * BA(k, c);
    }
  }
  return 0;
}
static void band_solve(or_problem *P, double *b) {
  int n = P->bn, w = P->bw, ld = 2 * w + 1;
  for (int r = 1; r < n; ++r) for (int c = imax(0, r - w); c < r; ++c) b[r] -= BA(r, c) * b[c];
  for (int r = n - 1; r >= 0; --r) {
    for (int c = r + 1; c <= imin(n - 1, r + w); ++c) b[r] -= BA(r, c) * b[c];
    b[r] /= BA(r, r);
  }
#undef BA
}

/* ---------------------------------------------------------------- setup -- */

/* R5: coarsen by dropping every other grid line while both sides are even,
 * stay >= 2 intervals, and max(nx,ny) > 8.                                  */
or_problem *or_create(int nx, int ny, const double *x, const double *y) {
  if (nx < 2 || ny < 2) return NULL;
  or_problem *P = calloc(1, sizeof(or_problem));
  level_init(&P->lev[0], nx, ny, x, y);
  int l = 0;
  while (l + 1 < OR_MAXLEV) {
    level_t *F = &P->lev[l];
    if (F->nx % 2 || F->ny % 2 || F->nx / 2 < 2 || F->ny / 2 < 2 || imax(F->nx, F->ny) <= 8) break;
    int cx = F->nx / 2, cy = F->ny / 2;
    double *xc = malloc(sizeof(double) * (cx + 1)), *yc = malloc(sizeof(double) * (cy + 1));
    for (int i = 0; i <= cx; ++i) xc[i] = F->x[2 * i];
    for (int j = 0; j <= cy; ++j) yc[j] = F->y[2 * j];
    level_init(&P->lev[l + 1], cx, cy, xc, yc);
    free(xc); free(yc);
    ++l;
  }
  P->nlev = l + 1;
  for (int k = 0; k < P->nlev; ++k) {
    size_t nn = (size_t)(P->lev[k].nx + 1) * (P->lev[k].ny + 1);
    for (int s = 0; s < 3; ++s) P->work[k][s] = calloc(nn, sizeof(double));
  }
  return P;
}

void or_destroy(or_problem *P) {
  if (!P) return;
  for (int k = 0; k < OR_MAXLEV; ++k) {
    level_t *L = &P->lev[k];
    free(L->x); free(L->y); free(L->W); free(L->E); free(L->S); free(L->N);
    for (int s = 0; s < 7; ++s) { free(P->part[k][s].blk); free(P->part[k][s].owner); free(P->part[k][s].pool); }
    for (int s = 0; s < 3; ++s) free(P->work[k][s]);
  }
  free(P->clu); free(P->cpiv); free(P->band);
  free(P);
}

int or_num_levels(or_problem *P) { return P->nlev; }

/* Threads of the colour passes in OpenMP builds (1 in plain builds); n <= 0
 * keeps the current count.  Returns the count in effect.                    */
int or_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}
void or_level_shape(or_problem *P, int lev, int *nx, int *ny) { *nx = P->lev[lev].nx; *ny = P->lev[lev].ny; }
void or_level_coeffs(or_problem *P, int lev, double *W, double *E, double *S, double *N) {
  level_t *L = &P->lev[lev];
  memcpy(W, L->W, sizeof(double) * (L->nx + 1)); memcpy(E, L->E, sizeof(double) * (L->nx + 1));
  memcpy(S, L->S, sizeof(double) * (L->ny + 1)); memcpy(N, L->N, sizeof(double) * (L->ny + 1));
}

/* --------------------------------------------------------------- cycles -- */

typedef struct {
  int smoother, nu1, nu2, gamma, restriction;
} or_cycle_t;

/* Sec. 4 steps (2)-(6) at level lev; gamma = 1 is the V-cycle, gamma = 2 the
 * W-cycle ("other cycling strategies").  u already holds the boundary data. */
static int cycle_rec(or_problem *P, const or_cycle_t *c, int lev, double *u, const double *f) {
  if (lev == P->nlev - 1) return coarse_solve(P, u, f);
  for (int s = 0; s < c->nu1; ++s) if (or_smooth(P, lev, c->smoother, u, f)) return -1;
  double *d = P->work[lev][2];
  or_residual(P, lev, u, f, d);
  double *uc = P->work[lev + 1][0], *fc = P->work[lev + 1][1];
  level_t *C = &P->lev[lev + 1];
  or_restrict(P, lev, c->restriction, d, fc);
  memset(uc, 0, sizeof(double) * (C->nx + 1) * (C->ny + 1));
  for (int g = 0; g < c->gamma; ++g) if (cycle_rec(P, c, lev + 1, uc, fc)) return -1;
  or_prolong_add(P, lev, uc, u);
  for (int s = 0; s < c->nu2; ++s) if (or_smooth(P, lev, c->smoother, u, f)) return -1;
  return 0;
}

int or_cycle(or_problem *P, int smoother, int nu1, int nu2, int gamma, int restriction,
             double *u, const double *f) {
  or_cycle_t c = {smoother, nu1, nu2, gamma, restriction};
  return cycle_rec(P, &c, 0, u, f);
}

/* Repeat cycles from the given u until ||f - L u||_2 / ||f||_2 <= tol or
 * max_cycles (Sec. 4 step (6)).  hist[k] = relative 2-norm after cycle k
 * (hist[0] = before the first cycle), hmax[k] = max-norm of the defect over
 * the initial max-norm (the quantity plotted in the paper's histories).
 * Returns the number of cycles done, or -1 on failure.                      */
int or_solve(or_problem *P, int smoother, int nu1, int nu2, int gamma, int restriction,
             double tol, int max_cycles, double *u, const double *f,
             double *hist, double *hmax, int cap) {
  level_t *L = &P->lev[0];
  size_t nn = (size_t)(L->nx + 1) * (L->ny + 1);
  double *d = malloc(sizeof(double) * nn), fs, fm, s, m, m0;
  /* scale of the relative residual: the right-hand side of the interior
     system, f - B g = the residual of u with its interior set to zero (equal
     to f when the boundary data g vanish) */
  for (size_t k = 0; k < nn; ++k) d[k] = u[k];
  for (int j = 1; j < L->ny; ++j)
    for (int i = 1; i < L->nx; ++i) d[ID(L, i, j)] = 0.0;
  double *b = malloc(sizeof(double) * nn);
  or_residual(P, 0, d, f, b);
  or_norms(P, 0, b, &fs, &fm);
  free(b);
  double fn = sqrt(fs);
  or_residual(P, 0, u, f, d);
  or_norms(P, 0, d, &s, &m0);
  if (fn == 0.0) fn = sqrt(s) > 0 ? sqrt(s) : 1.0;
  if (cap > 0) { hist[0] = sqrt(s) / fn; hmax[0] = 1.0; }
  int k = 0;
  double rel = sqrt(s) / fn;
  while (rel > tol && k < max_cycles) {
    if (or_cycle(P, smoother, nu1, nu2, gamma, restriction, u, f)) { free(d); return -1; }
    ++k;
    or_residual(P, 0, u, f, d);
    or_norms(P, 0, d, &s, &m);
    rel = sqrt(s) / fn;
    if (k < cap) { hist[k] = rel; hmax[k] = m0 > 0 ? m / m0 : 0.0; }
    if (!isfinite(rel)) break;
  }
  free(d);
  return k;
}

/* ------------------------------------------------------ two-grid operator -- */

/* e <- M e with M = S^nu2 (I - P L1^{-1} R L0) S^nu1, Eq. (Mh2h): the
 * two-grid cycle for f = 0 with an exact solve on level 1 (Sec. 5).  e has
 * zero boundary values on entry and exit.                                  */
int or_twogrid_apply(or_problem *P, int smoother, int restriction, int nu1, int nu2, double *e) {
  if (P->nlev < 2) return -1;
  if (!P->band && band_factor(P)) return -1;
  level_t *F = &P->lev[0], *C = &P->lev[1];
  size_t nf = (size_t)(F->nx + 1) * (F->ny + 1);
  double *zero = P->work[0][1], *d = P->work[0][2], *fc = P->work[1][1], *uc = P->work[1][0];
  memset(zero, 0, sizeof(double) * nf);
  for (int s = 0; s < nu1; ++s) if (or_smooth(P, 0, smoother, e, zero)) return -1;
  or_residual(P, 0, e, zero, d);
  or_restrict(P, 0, restriction, d, fc);
  int cn = C->nx - 1;
  double *b = malloc(sizeof(double) * P->bn);
  for (int J = 1; J < C->ny; ++J) for (int I = 1; I < C->nx; ++I) b[(J - 1) * cn + (I - 1)] = fc[ID(C, I, J)];
  band_solve(P, b);
  memset(uc, 0, sizeof(double) * (C->nx + 1) * (C->ny + 1));
  for (int J = 1; J < C->ny; ++J) for (int I = 1; I < C->nx; ++I) uc[ID(C, I, J)] = b[(J - 1) * cn + (I - 1)];
  free(b);
  or_prolong_add(P, 0, uc, e);
  for (int s = 0; s < nu2; ++s) if (or_smooth(P, 0, smoother, e, zero)) return -1;
  return 0;
}

/* ------------------------------------------------- inspection for tests -- */

/* Partition summary of a base smoother on level lev: number of blocks and,
 * per block, (type, colour, size, number of legs).  out must hold 4*max
 * ints; returns the number of blocks (or -1).                               */
int or_partition_info(or_problem *P, int lev, int sm, int *out, int max) {
  if (build_partition(P, lev, sm)) return -1;
  partition_t *T = &P->part[lev][sm];
  for (int b = 0; b < T->nblock && b < max; ++b) {
    out[4 * b + 0] = T->blk[b].type; out[4 * b + 1] = T->blk[b].colour;
    out[4 * b + 2] = T->blk[b].n; out[4 * b + 3] = T->blk[b].nleg;
  }
  return T->nblock;
}

/* Block index of every node (-1 on the boundary).                           */
int or_partition_owner(or_problem *P, int lev, int sm, int *owner) {
  if (build_partition(P, lev, sm)) return -1;
  level_t *L = &P->lev[lev];
  memcpy(owner, P->part[lev][sm].owner, sizeof(int) * (L->nx + 1) * (L->ny + 1));
  return 0;
}

/* Nodes of block b in solve order (star: junction first, then each leg
 * tip -> junction).  Returns the count.                                    */
int or_block_nodes(or_problem *P, int lev, int sm, int b, int *nodes) {
  if (build_partition(P, lev, sm)) return -1;
  block_t *B = &P->part[lev][sm].blk[b];
  memcpy(nodes, B->node, sizeof(int) * B->n);
  return B->n;
}

/* Dense assembly of block b's system in the order of or_block_nodes:
 * A (n x n, row-major) and rhs, given the current u and f.                  */
int or_block_dense(or_problem *P, int lev, int sm, int b, const double *u, const double *f,
                   double *A, double *rhs) {
  if (build_partition(P, lev, sm)) return -1;
  level_t *L = &P->lev[lev];
  partition_t *T = &P->part[lev][sm];
  block_t *B = &T->blk[b];
  int n = B->n, nx = L->nx;
  memset(A, 0, sizeof(double) * n * n);
  for (int r = 0; r < n; ++r) {
    int p = B->node[r];
    A[r * n + r] = coef_centre(L, p % (nx + 1), p / (nx + 1));
    rhs[r] = block_rhs(L, T->owner, b, p, u, f);
    for (int c = 0; c < n; ++c)
      if (c != r && adjacent(L, p, B->node[c])) A[r * n + c] = coef_pq(L, p, B->node[c]);
  }
  return n;
}

/* Exact solve of the single block b in place in u (for block-level tests).  */
int or_block_solve(or_problem *P, int lev, int sm, int b, double *u, const double *f) {
  if (build_partition(P, lev, sm)) return -1;
  solve_block(&P->lev[lev], &P->part[lev][sm], b, u, f);
  return 0;
}

/* Dense LU solve of an n x n system (A overwritten; b becomes x).           */
int or_dense_solve(int n, double *A, double *b) {
  int *piv = malloc(sizeof(int) * n);
  int rc = lu_factor(n, A, piv);
  if (!rc) lu_solve(n, A, piv, b);
  free(piv);
  return rc;
}
