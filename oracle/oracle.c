/*
 * oracle.c -- plain FP64 CPU oracle for the black-box FMM (Laplace 1/r,
 * potentials and forces) of Agullo et al., "Pipelining the Fast Multipole
 * Method over a Runtime System" (2012).
 *
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline).  It is written to be read against the paper, not to be fast:
 * every operator is the formula of Sec. 2 evaluated with plain loops in
 * double precision.  Compile with -ffp-contract=off so that the Morton
 * quantisation is the IEEE operation sequence stated below.
 *
 * Paper references:
 *   eq. 1  pairwise summation f_i = sum_j P(x_i, y_j) w_j          (Sec. 2)
 *   eq. 2  P = 1/|x-y|, F = (x-y)/|x-y|^3                          (Sec. 2.1)
 *   eq. 3  P ~ sum_m S_m(x) sum_n P(xbar_m, ybar_n) S_n(y); F moves the
 *          gradient onto S_m(x)                                     (Sec. 2.1)
 *   eq. 4  S_m(x) = S_m1(x1) S_m2(x2) S_m3(x3)                      (Sec. 2.1.1)
 *   eq. 5  S(xbar, x) = 1/l + 2/l sum_{n=1}^{l-1} T_n(xbar) T_n(x),
 *          xbar the Chebyshev roots                                 (Sec. 2.1.1)
 *   Sec. 2.1.2  M2L over the children of the parent's neighbours that are not
 *          neighbours themselves (at most 189), 316 distinct transfer
 *          vectors, computed once thanks to the homogeneity of 1/r.
 *   Sec. 2.2  the method needs kernel values only: ofmm_set_kernel selects
 *          (|x-y|^2 + kc^2)^(-ks/2); kc = 0 is homogeneous (one operator set,
 *          scaled per level), kc > 0 (multiquadrics) gets a set per level.
 *   Sec. 3.2  bottom-up P2M, M2M; top-down M2L, L2L, L2P; P2P at the leaves.
 *   Sec. 4.2  cells in Morton order.
 *
 * Pins: each function is checked against closed forms, invariants or brute
 * force in tests/test_oracle.py (no function is left unpinned).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXH 12
#define MAXP 12

struct ofmm {
  int height, order, leaf, ncoef;
  int64_t n;
  double lo[3], width;
  int64_t* perm;   /* Morton rank -> input index */
  double* x;       /* [n][3], Morton order */
  double* q;       /* [n], Morton order */
  int64_t ncell[MAXH];
  uint64_t* key[MAXH];   /* sorted non-empty cell keys per level */
  int64_t* first[MAXH];  /* leaf level: first particle; else first child */
  int64_t* count[MAXH];  /* leaf level: particle count; else child count */
  int64_t* parent[MAXH]; /* index of the parent cell (level - 1) */
  double* M[MAXH];       /* multipole expansions [ncell][ncoef] */
  double* L[MAXH];       /* local expansions [ncell][ncoef] */
  double xbar[MAXP];     /* Chebyshev roots */
  double ks;             /* kernel exponent: P(x, y) = (|x - y|^2 + kc^2)^(-ks/2) */
  double kc;             /* kernel offset c (0: |x - y|^-ks; ks = 1, kc = 0: Laplace) */
  double* K;             /* M2L operators for unit half-width, see m2l_operators() */
  double* Kl[MAXH];      /* kc > 0: the operators of each level, at its half-width */
  /* SVD-compressed M2L (Sec. 2.1.2, "Improved M2L operator"); svd_eps > 0
   * selects it.  For the 16 canonical transfer vectors: rank, U_k Sigma_k
   * [C][rank] and V_k [C][rank]. */
  double svd_eps;
  int svd_rank[16];
  double* svd_US[16];
  double* svd_V[16];
};

/* ------------------------------------------------------------------------ */
/* Chebyshev interpolation, eq. 5                                            */
/* ------------------------------------------------------------------------ */

void ofmm_cheb_nodes(int order, double* xbar) {
  /* Roots of T_order: cos((2k+1) pi / (2 order)).  The upper half is taken
   * as the exact negation of the lower half and the middle root of an odd
   * order is exactly 0, so the node set is symmetric bit for bit. */
  for (int k = 0; k < order; ++k) xbar[k] = 0.0;
  for (int k = 0; 2 * k + 1 < order; ++k) {
    xbar[k] = cos((2.0 * k + 1.0) * M_PI / (2.0 * order));
    xbar[order - 1 - k] = -xbar[k];
  }
}

/* T_0..T_{p-1} at x by the three-term recurrence. */
static void cheb_T(int p, double x, double* T) {
  T[0] = 1.0;
  if (p > 1) T[1] = x;
  for (int n = 2; n < p; ++n) T[n] = 2.0 * x * T[n - 1] - T[n - 2];
}

/* dT_n/dx = n U_{n-1}(x) for n = 0..p-1. */
static void cheb_dT(int p, double x, double* dT) {
  double U[MAXP];
  U[0] = 1.0;
  if (p > 1) U[1] = 2.0 * x;
  for (int k = 2; k < p; ++k) U[k] = 2.0 * x * U[k - 1] - U[k - 2];
  dT[0] = 0.0;
  for (int n = 1; n < p; ++n) dT[n] = n * U[n - 1];
}

double ofmm_cheb_S(int p, double xbar, double xi) {
  double Tb[MAXP], Tx[MAXP], s = 0.0;
  cheb_T(p, xbar, Tb);
  cheb_T(p, xi, Tx);
  for (int n = 1; n < p; ++n) s += Tb[n] * Tx[n];
  return 1.0 / p + 2.0 / p * s;
}

double ofmm_cheb_dS(int p, double xbar, double xi) {
  double Tb[MAXP], dTx[MAXP], s = 0.0;
  cheb_T(p, xbar, Tb);
  cheb_dT(p, xi, dTx);
  for (int n = 1; n < p; ++n) s += Tb[n] * dTx[n];
  return 2.0 / p * s;
}

/* ------------------------------------------------------------------------ */
/* Root cube, Morton keys, sort (Sec. 3.2 subdivision; Sec. 4.2 Morton order) */
/* ------------------------------------------------------------------------ */

void ofmm_bounding_cube(int64_t n, const double* xyz, double* lo, double* width) {
  double hi[3];
  if (n <= 0) {
    lo[0] = lo[1] = lo[2] = 0.0;
    *width = 1.0;
    return;
  }
  for (int d = 0; d < 3; ++d) lo[d] = hi[d] = xyz[d];
  for (int64_t i = 1; i < n; ++i)
    for (int d = 0; d < 3; ++d) {
      double v = xyz[3 * i + d];
      if (v < lo[d]) lo[d] = v;
      if (v > hi[d]) hi[d] = v;
    }
  double w = 0.0;
  for (int d = 0; d < 3; ++d)
    if (hi[d] - lo[d] > w) w = hi[d] - lo[d];
  *width = (w > 0.0) ? w : 1.0;
}

/* Integer cell coordinate along one axis at the leaf level:
 * floor(((x - lo) / W) * 2^leaf), clamped to [0, 2^leaf - 1].  The product by
 * a power of two is exact, so the only roundings are the IEEE subtraction and
 * division. */
static int64_t leaf_coord(double x, double lo, double width, int leaf) {
  double t = (x - lo) / width;
  double u = ldexp(t, leaf);
  int64_t i = (int64_t)floor(u);
  int64_t top = ((int64_t)1 << leaf) - 1;
  if (i < 0) i = 0;
  if (i > top) i = top;
  return i;
}

static uint64_t morton_encode(int64_t ix, int64_t iy, int64_t iz, int bits) {
  uint64_t k = 0;
  for (int b = 0; b < bits; ++b) {
    k |= (uint64_t)((ix >> b) & 1) << (3 * b + 2);
    k |= (uint64_t)((iy >> b) & 1) << (3 * b + 1);
    k |= (uint64_t)((iz >> b) & 1) << (3 * b);
  }
  return k;
}

static void morton_decode(uint64_t k, int bits, int64_t* c) {
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < bits; ++b) {
    c[0] |= (int64_t)((k >> (3 * b + 2)) & 1) << b;
    c[1] |= (int64_t)((k >> (3 * b + 1)) & 1) << b;
    c[2] |= (int64_t)((k >> (3 * b)) & 1) << b;
  }
}

void ofmm_keys(int64_t n, const double* xyz, const double* lo, double width, int leaf,
               uint64_t* keys) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    int64_t c[3];
    for (int d = 0; d < 3; ++d) c[d] = leaf_coord(xyz[3 * i + d], lo[d], width, leaf);
    keys[i] = morton_encode(c[0], c[1], c[2], leaf);
  }
}

typedef struct {
  uint64_t key;
  int64_t idx;
} keyed;

static int cmp_keyed(const void* a, const void* b) {
  const keyed* x = (const keyed*)a;
  const keyed* y = (const keyed*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
  return 0;
}

/* Index of `k` among the sorted keys of a level, or -1. */
static int64_t find_cell(const ofmm* c, int level, uint64_t k) {
  int64_t a = 0, b = c->ncell[level] - 1;
  const uint64_t* keys = c->key[level];
  while (a <= b) {
    int64_t m = a + (b - a) / 2;
    if (keys[m] == k) return m;
    if (keys[m] < k) a = m + 1;
    else b = m - 1;
  }
  return -1;
}

static void cell_coords(const ofmm* c, int level, int64_t cell, int64_t* ic) {
  morton_decode(c->key[level][cell], level, ic);
}

/* Centre and half-width of a cell: the root cube halved `level` times. */
static void cell_geometry(const ofmm* c, int level, int64_t cell, double* centre, double* a) {
  int64_t ic[3];
  cell_coords(c, level, cell, ic);
  double w = ldexp(c->width, -level);
  for (int d = 0; d < 3; ++d) centre[d] = c->lo[d] + ((double)ic[d] + 0.5) * w;
  *a = 0.5 * w;
}

/* M2L operator for transfer vector t (in cell widths, |t|_inf in {2, 3}) and
 * unit half-width: K_t[m][n] = 1 / |2t + xbar_n - xbar_m|.  With cell
 * half-width a the operator is K_t / a (1/r is homogeneous of degree -1,
 * Sec. 2.1.2), because the target node is c_T + a xbar_m, the source node is
 * c_S + a xbar_n and c_S - c_T = 2 a t. */
static int tslot(int tx, int ty, int tz) { return ((tx + 3) * 7 + (ty + 3)) * 7 + (tz + 3); }

/* (r^2 + kc^2)^(-s/2) from r^2 (s = 1, kc = 0: the Laplace kernel, kept as
 * 1 / sqrt). */
static double kernel_of_r2(double r2, double s, double kc) {
  if (kc == 0.0) return s == 1.0 ? 1.0 / sqrt(r2) : pow(r2, -0.5 * s);
  return pow(r2 + kc * kc, -0.5 * s);
}

/* The factor a^-s that scales the unit-half-width operators to half-width a
 * (P is homogeneous of degree -s); s = 1 divides by a as before. */
static double scale_a(double x, double a, double s) { return s == 1.0 ? x / a : x * pow(a, -s); }

/* K_t[m][n] = P(xbar_m, 2 a t + a xbar_n) over the 343 slots of t in
 * [-3, 3]^3 (only the far ones are filled) for half-width a. */
static double* operators_at(const ofmm* c, double a, double kc) {
  int p = c->order, C = c->ncoef;
  double* Kall = (double*)calloc((size_t)343 * C * C, sizeof(double));
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < 343; ++s) {
    int t[3] = {s / 49 - 3, (s / 7) % 7 - 3, s % 7 - 3};
    int far = abs(t[0]) >= 2 || abs(t[1]) >= 2 || abs(t[2]) >= 2;
    if (!far) continue;
    double* K = Kall + (size_t)s * C * C;
    for (int m = 0; m < C; ++m) {
      int mi[3] = {m / (p * p), (m / p) % p, m % p};
      for (int nn = 0; nn < C; ++nn) {
        int ni[3] = {nn / (p * p), (nn / p) % p, nn % p};
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          double r = a * (2.0 * t[d] + c->xbar[ni[d]] - c->xbar[mi[d]]);
          r2 += r * r;
        }
        K[(size_t)m * C + nn] = kernel_of_r2(r2, c->ks, kc);
      }
    }
  }
  return Kall;
}

/* Homogeneous kernels (kc = 0): one set at unit half-width, scaled per level
 * (Sec. 2.1.2).  kc > 0 is not homogeneous: every level l gets its own set,
 * the kernel evaluated at the level's own node positions (half-width
 * a_l = W / 2^(l+1)), which the M2L applies unscaled. */
static void m2l_operators(ofmm* c) {
  if (c->kc == 0.0) {
    c->K = operators_at(c, 1.0, 0.0);
    return;
  }
  for (int l = 2; l <= c->leaf; ++l) c->Kl[l] = operators_at(c, ldexp(c->width, -l - 1), c->kc);
}

static void free_operators(ofmm* c) {
  free(c->K);
  c->K = NULL;
  for (int l = 0; l < MAXH; ++l) {
    free(c->Kl[l]);
    c->Kl[l] = NULL;
  }
}

ofmm* ofmm_create(int64_t n, const double* xyz, const double* q, int height, int order) {
  if (height < 1 || height > MAXH || order < 2 || order > MAXP || n < 0) return NULL;
  for (int64_t i = 0; i < n; ++i) {
    if (!isfinite(q[i])) return NULL;
    for (int d = 0; d < 3; ++d)
      if (!isfinite(xyz[3 * i + d])) return NULL;
  }
  ofmm* c = (ofmm*)calloc(1, sizeof(ofmm));
  c->height = height;
  c->order = order;
  c->ks = 1.0;
  c->leaf = height - 1;
  c->ncoef = order * order * order;
  c->n = n;
  ofmm_cheb_nodes(order, c->xbar);
  ofmm_bounding_cube(n, xyz, c->lo, &c->width);

  /* keys and the stable sort: ties keep input order */
  uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (n ? n : 1));
  ofmm_keys(n, xyz, c->lo, c->width, c->leaf, keys);
  keyed* kv = (keyed*)malloc(sizeof(keyed) * (n ? n : 1));
  for (int64_t i = 0; i < n; ++i) {
    kv[i].key = keys[i];
    kv[i].idx = i;
  }
  qsort(kv, (size_t)n, sizeof(keyed), cmp_keyed);
  c->perm = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  c->x = (double*)malloc(sizeof(double) * 3 * (n ? n : 1));
  c->q = (double*)malloc(sizeof(double) * (n ? n : 1));
  for (int64_t r = 0; r < n; ++r) {
    int64_t i = kv[r].idx;
    c->perm[r] = i;
    for (int d = 0; d < 3; ++d) c->x[3 * r + d] = xyz[3 * i + d];
    c->q[r] = q[i];
  }

  /* leaf level: runs of equal keys */
  int Lf = c->leaf;
  int64_t nl = 0;
  for (int64_t r = 0; r < n; ++r)
    if (r == 0 || kv[r].key != kv[r - 1].key) ++nl;
  c->ncell[Lf] = nl;
  c->key[Lf] = (uint64_t*)malloc(sizeof(uint64_t) * (nl ? nl : 1));
  c->first[Lf] = (int64_t*)malloc(sizeof(int64_t) * (nl ? nl : 1));
  c->count[Lf] = (int64_t*)calloc(nl ? nl : 1, sizeof(int64_t));
  int64_t li = -1;
  for (int64_t r = 0; r < n; ++r) {
    if (r == 0 || kv[r].key != kv[r - 1].key) {
      ++li;
      c->key[Lf][li] = kv[r].key;
      c->first[Lf][li] = r;
    }
    c->count[Lf][li]++;
  }
  /* coarser levels: parent key = child key >> 3 */
  for (int l = Lf - 1; l >= 0; --l) {
    int64_t nc = c->ncell[l + 1], np = 0;
    for (int64_t i = 0; i < nc; ++i)
      if (i == 0 || (c->key[l + 1][i] >> 3) != (c->key[l + 1][i - 1] >> 3)) ++np;
    c->ncell[l] = np;
    c->key[l] = (uint64_t*)malloc(sizeof(uint64_t) * (np ? np : 1));
    c->first[l] = (int64_t*)malloc(sizeof(int64_t) * (np ? np : 1));
    c->count[l] = (int64_t*)calloc(np ? np : 1, sizeof(int64_t));
    c->parent[l + 1] = (int64_t*)malloc(sizeof(int64_t) * (nc ? nc : 1));
    int64_t pi = -1;
    for (int64_t i = 0; i < nc; ++i) {
      uint64_t pk = c->key[l + 1][i] >> 3;
      if (i == 0 || pk != (c->key[l + 1][i - 1] >> 3)) {
        ++pi;
        c->key[l][pi] = pk;
        c->first[l][pi] = i;
      }
      c->count[l][pi]++;
      c->parent[l + 1][i] = pi;
    }
  }
  c->parent[0] = (int64_t*)calloc(c->ncell[0] ? c->ncell[0] : 1, sizeof(int64_t));
  for (int l = 0; l <= Lf; ++l) {
    size_t sz = (size_t)(c->ncell[l] ? c->ncell[l] : 1) * c->ncoef;
    c->M[l] = (double*)calloc(sz, sizeof(double));
    c->L[l] = (double*)calloc(sz, sizeof(double));
  }
  free(keys);
  free(kv);
  if (Lf >= 2) m2l_operators(c);
  return c;
}

void ofmm_destroy(ofmm* c) {
  if (!c) return;
  for (int l = 0; l <= c->leaf; ++l) {
    free(c->key[l]);
    free(c->first[l]);
    free(c->count[l]);
    free(c->parent[l]);
    free(c->M[l]);
    free(c->L[l]);
  }
  free(c->perm);
  free(c->x);
  free(c->q);
  free_operators(c);
  for (int k = 0; k < 16; ++k) {
    free(c->svd_US[k]);
    free(c->svd_V[k]);
  }
  free(c);
}

void ofmm_box(const ofmm* c, double* lo, double* width) {
  for (int d = 0; d < 3; ++d) lo[d] = c->lo[d];
  *width = c->width;
}

int64_t ofmm_level_size(const ofmm* c, int level) {
  if (level < 0 || level > c->leaf) return -1;
  return c->ncell[level];
}

void ofmm_level_keys(const ofmm* c, int level, uint64_t* keys) {
  memcpy(keys, c->key[level], sizeof(uint64_t) * c->ncell[level]);
}

void ofmm_level_ranges(const ofmm* c, int level, int64_t* first, int64_t* count) {
  memcpy(first, c->first[level], sizeof(int64_t) * c->ncell[level]);
  memcpy(count, c->count[level], sizeof(int64_t) * c->ncell[level]);
}

void ofmm_perm(const ofmm* c, int64_t* perm) { memcpy(perm, c->perm, sizeof(int64_t) * c->n); }

void ofmm_expansion(const ofmm* c, int level, int which, double* out) {
  const double* src = which ? c->L[level] : c->M[level];
  memcpy(out, src, sizeof(double) * c->ncell[level] * c->ncoef);
}

/* ------------------------------------------------------------------------ */
/* Interaction lists (Sec. 2.1.2, Sec. 3.3)                                  */
/* ------------------------------------------------------------------------ */

/* Near field of a leaf: the existing leaves whose coordinates differ from the
 * target's by at most 1 on every axis (the target itself included). */
static int near_list(const ofmm* c, int64_t cell, int64_t* src) {
  int Lf = c->leaf, ns = 0;
  int64_t ic[3], top = ((int64_t)1 << Lf) - 1;
  cell_coords(c, Lf, cell, ic);
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int64_t s[3] = {ic[0] + dx, ic[1] + dy, ic[2] + dz};
        if (s[0] < 0 || s[1] < 0 || s[2] < 0 || s[0] > top || s[1] > top || s[2] > top) continue;
        int64_t j = find_cell(c, Lf, morton_encode(s[0], s[1], s[2], Lf));
        if (j >= 0) src[ns++] = j;
      }
  return ns;
}

/* Far field of a cell at `level`: the existing children of the parent's
 * neighbours (the parent included) that are not neighbours of the cell.
 * Returns the count; src[] the cells, t[] their transfer vectors
 * (source minus target coordinates). */
static int far_list(const ofmm* c, int level, int64_t cell, int64_t* src, int* t) {
  int nf = 0;
  if (level < 2) return 0;
  int64_t ic[3], pc[3], ptop = ((int64_t)1 << (level - 1)) - 1;
  cell_coords(c, level, cell, ic);
  for (int d = 0; d < 3; ++d) pc[d] = ic[d] >> 1;
  for (int dx = -1; dx <= 1; ++dx)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dz = -1; dz <= 1; ++dz) {
        int64_t pn[3] = {pc[0] + dx, pc[1] + dy, pc[2] + dz};
        if (pn[0] < 0 || pn[1] < 0 || pn[2] < 0 || pn[0] > ptop || pn[1] > ptop || pn[2] > ptop)
          continue;
        for (int ch = 0; ch < 8; ++ch) {
          int64_t s[3] = {2 * pn[0] + ((ch >> 2) & 1), 2 * pn[1] + ((ch >> 1) & 1),
                          2 * pn[2] + (ch & 1)};
          int64_t tv[3] = {s[0] - ic[0], s[1] - ic[1], s[2] - ic[2]};
          if (llabs(tv[0]) <= 1 && llabs(tv[1]) <= 1 && llabs(tv[2]) <= 1) continue;
          int64_t j = find_cell(c, level, morton_encode(s[0], s[1], s[2], level));
          if (j < 0) continue;
          src[nf] = j;
          t[3 * nf + 0] = (int)tv[0];
          t[3 * nf + 1] = (int)tv[1];
          t[3 * nf + 2] = (int)tv[2];
          ++nf;
        }
      }
  return nf;
}

/* ------------------------------------------------------------------------ */
/* Operators (Sec. 2.1, eq. 3-5)                                             */
/* ------------------------------------------------------------------------ */

/* P2M: M_m = sum_j q_j S_m((y_j - c)/a), S_m the tensor product of eq. 4. */
void ofmm_p2m(ofmm* c) {
  int p = c->order, C = c->ncoef, Lf = c->leaf;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t cell = 0; cell < c->ncell[Lf]; ++cell) {
    double ctr[3], a, S[3][MAXP];
    cell_geometry(c, Lf, cell, ctr, &a);
    double* M = c->M[Lf] + (size_t)cell * C;
    for (int m = 0; m < C; ++m) M[m] = 0.0;
    for (int64_t r = c->first[Lf][cell]; r < c->first[Lf][cell] + c->count[Lf][cell]; ++r) {
      for (int d = 0; d < 3; ++d) {
        double xi = (c->x[3 * r + d] - ctr[d]) / a;
        for (int k = 0; k < p; ++k) S[d][k] = ofmm_cheb_S(p, c->xbar[k], xi);
      }
      for (int m = 0; m < C; ++m)
        M[m] += c->q[r] * S[0][m / (p * p)] * S[1][(m / p) % p] * S[2][m % p];
    }
  }
}

/* 1-D interpolation weights between a child and its parent along axis d:
 * A[m][m'] = S(xbar_m, (c_child + a_child xbar_m' - c_parent) / a_parent). */
static void child_weights(const ofmm* c, const double* cc, double ac, const double* cp, double ap,
                          double A[3][MAXP][MAXP]) {
  int p = c->order;
  for (int d = 0; d < 3; ++d)
    for (int m = 0; m < p; ++m)
      for (int mm = 0; mm < p; ++mm)
        A[d][m][mm] = ofmm_cheb_S(p, c->xbar[m], (cc[d] + ac * c->xbar[mm] - cp[d]) / ap);
}

/* M2M: the parent's multipole expansion interpolates its children's at the
 * parent's nodes: M_P[m] = sum_children sum_m' S_m(xi_P(child node m')) M_C[m']. */
void ofmm_m2m(ofmm* c) {
  int p = c->order, C = c->ncoef;
  for (int l = c->leaf - 1; l >= 2; --l) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t P = 0; P < c->ncell[l]; ++P) {
      double cp[3], ap, cc[3], ac, A[3][MAXP][MAXP];
      cell_geometry(c, l, P, cp, &ap);
      double* MP = c->M[l] + (size_t)P * C;
      for (int m = 0; m < C; ++m) MP[m] = 0.0;
      for (int64_t ch = c->first[l][P]; ch < c->first[l][P] + c->count[l][P]; ++ch) {
        cell_geometry(c, l + 1, ch, cc, &ac);
        child_weights(c, cc, ac, cp, ap, A);
        const double* MC = c->M[l + 1] + (size_t)ch * C;
        for (int m = 0; m < C; ++m) {
          int mx = m / (p * p), my = (m / p) % p, mz = m % p;
          double s = 0.0;
          for (int mm = 0; mm < C; ++mm)
            s += A[0][mx][mm / (p * p)] * A[1][my][(mm / p) % p] * A[2][mz][mm % p] * MC[mm];
          MP[m] += s;
        }
      }
    }
  }
}

/* M2L at one cell: L_T[m] = sum_{S in far field} sum_n P(xbar^T_m, ybar^S_n) M_S[n],
 * with P(xbar^T_m, ybar^S_n) = K_t[m][n] / a. */
static void m2l_cell(ofmm* c, int l, int64_t T, int64_t* src, int* tv) {
  int C = c->ncoef;
  double a = ldexp(c->width, -l - 1);
  double* LT = c->L[l] + (size_t)T * C;
  const double* Kset = c->kc == 0.0 ? c->K : c->Kl[l];
  for (int m = 0; m < C; ++m) LT[m] = 0.0;
  int nf = far_list(c, l, T, src, tv);
  for (int k = 0; k < nf; ++k) {
    const double* K = Kset + (size_t)tslot(tv[3 * k], tv[3 * k + 1], tv[3 * k + 2]) * C * C;
    const double* MS = c->M[l] + (size_t)src[k] * C;
    for (int m = 0; m < C; ++m) {
      double s = 0.0;
      for (int nn = 0; nn < C; ++nn) s += K[(size_t)m * C + nn] * MS[nn];
      LT[m] += c->kc == 0.0 ? scale_a(s, a, c->ks) : s;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* SVD-compressed M2L (Sec. 2.1.2, "Improved M2L operator", Table 1)         */
/* ------------------------------------------------------------------------ */

/* Symmetries of the cube.  A symmetry sigma permutes the axes and flips
 * signs: (sigma v)_d = sign[d] * v[axis[d]].  Every far transfer vector t is
 * sigma(that) for the canonical that = |t| sorted ascending (16 distinct
 * vectors); axis[d] is the position of |t_d| in that ordering (ties by axis
 * order) and sign[d] = -1 where t_d < 0, else +1. */
void ofmm_transfer_symmetry(const int* t, int* that, int* axis, int* sign) {
  int used[3] = {0, 0, 0};
  int a[3] = {abs(t[0]), abs(t[1]), abs(t[2])};
  int s[3] = {a[0], a[1], a[2]};
  /* ascending sort of three values */
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (s[j] < s[i]) {
        int x = s[i];
        s[i] = s[j];
        s[j] = x;
      }
  for (int d = 0; d < 3; ++d) {
    that[d] = s[d];
    sign[d] = t[d] < 0 ? -1 : 1;
    for (int j = 0; j < 3; ++j)
      if (!used[j] && s[j] == a[d]) {
        axis[d] = j;
        used[j] = 1;
        break;
      }
  }
}

/* Position of a canonical vector (0 <= a <= b <= c <= 3, c >= 2) in the
 * lexicographic list (0,0,2), (0,0,3), (0,1,2), ..., (3,3,3); -1 otherwise. */
int ofmm_canonical_index(const int* that) {
  int k = 0;
  for (int a = 0; a <= 3; ++a)
    for (int b = a; b <= 3; ++b)
      for (int cc = b; cc <= 3; ++cc) {
        if (cc < 2) continue;
        if (that[0] == a && that[1] == b && that[2] == cc) return k;
        ++k;
      }
  return -1;
}

/* Node multi-index map of a symmetry: sigma maps the node xbar_m to the node
 * xbar_{sm[m]}, because the roots are symmetric (xbar_{p-1-j} = -xbar_j):
 * (sigma.m)_d = m_{axis[d]}, or p-1-m_{axis[d]} where sign[d] = -1. */
void ofmm_node_permutation(int order, const int* axis, const int* sign, int32_t* sm) {
  int p = order, C = p * p * p;
  for (int m = 0; m < C; ++m) {
    int mi[3] = {m / (p * p), (m / p) % p, m % p}, r[3];
    for (int d = 0; d < 3; ++d) r[d] = sign[d] > 0 ? mi[axis[d]] : p - 1 - mi[axis[d]];
    sm[m] = (r[0] * p + r[1]) * p + r[2];
  }
}

/* One-sided Jacobi SVD (Hestenes): A (n x n, row-major) = U diag(s) V^T with
 * s descending.  Column pairs (i, j) are rotated, in cyclic order, until
 * every pair is orthogonal to |a_i . a_j| <= 1e-15 |a_i| |a_j|; then s_j are
 * the column norms, U the normalised columns and V the accumulated
 * rotations.  Returns the number of sweeps, or -1 without convergence in 60. */
int ofmm_jacobi_svd(int n, const double* A, double* U, double* s, double* V) {
  double* W = (double*)malloc(sizeof(double) * n * n);  /* W[j] = column j */
  double* Z = (double*)malloc(sizeof(double) * n * n);  /* Z[j] = column j of V */
  double* nrm = (double*)malloc(sizeof(double) * n);
  int* ord = (int*)malloc(sizeof(int) * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      W[(size_t)j * n + i] = A[(size_t)i * n + j];
      Z[(size_t)j * n + i] = i == j ? 1.0 : 0.0;
    }
  int sweeps = -1;
  for (int sweep = 1; sweep <= 60; ++sweep) {
    int rotated = 0;
    for (int i = 0; i < n - 1; ++i)
      for (int j = i + 1; j < n; ++j) {
        double* wi = W + (size_t)i * n;
        double* wj = W + (size_t)j * n;
        double al = 0.0, be = 0.0, ga = 0.0;
        for (int k = 0; k < n; ++k) {
          al += wi[k] * wi[k];
          be += wj[k] * wj[k];
          ga += wi[k] * wj[k];
        }
        if (fabs(ga) <= 1e-15 * sqrt(al * be) || ga == 0.0) continue;
        rotated = 1;
        /* the rotation that zeroes a_i . a_j */
        double zeta = (be - al) / (2.0 * ga);
        double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        double* zi = Z + (size_t)i * n;
        double* zj = Z + (size_t)j * n;
        for (int k = 0; k < n; ++k) {
          double x = wi[k], y = wj[k];
          wi[k] = cs * x - sn * y;
          wj[k] = sn * x + cs * y;
          x = zi[k];
          y = zj[k];
          zi[k] = cs * x - sn * y;
          zj[k] = sn * x + cs * y;
        }
      }
    if (!rotated) {
      sweeps = sweep;
      break;
    }
  }
  for (int j = 0; j < n; ++j) {
    double q = 0.0;
    for (int k = 0; k < n; ++k) q += W[(size_t)j * n + k] * W[(size_t)j * n + k];
    nrm[j] = sqrt(q);
    ord[j] = j;
  }
  /* descending by norm, ties by index (insertion sort) */
  for (int i = 1; i < n; ++i) {
    int x = ord[i], k = i - 1;
    while (k >= 0 && nrm[ord[k]] < nrm[x]) {
      ord[k + 1] = ord[k];
      --k;
    }
    ord[k + 1] = x;
  }
  for (int c = 0; c < n; ++c) {
    int j = ord[c];
    s[c] = nrm[j];
    for (int k = 0; k < n; ++k) {
      U[(size_t)k * n + c] = nrm[j] > 0.0 ? W[(size_t)j * n + k] / nrm[j] : 0.0;
      V[(size_t)k * n + c] = Z[(size_t)j * n + k];
    }
  }
  free(W);
  free(Z);
  free(nrm);
  free(ord);
  return sweeps;
}

/* The kernel (|x - y|^2 + kc^2)^(-s/2): the operators are rebuilt with it
 * and a compressed set is dropped (compress again with ofmm_set_m2l_svd;
 * kc = 0 only).  -2 <= s <= 4, s != 0, kc >= 0. */
int ofmm_set_kernel(ofmm* c, double s, double kc) {
  if (!(s >= -2.0 && s <= 4.0 && s != 0.0) || !(kc >= 0.0 && isfinite(kc))) return -1;
  int had = c->K != NULL || c->Kl[c->leaf] != NULL;
  c->ks = s;
  c->kc = kc;
  free_operators(c);
  if (had) m2l_operators(c);
  c->svd_eps = 0.0;
  for (int k = 0; k < 16; ++k) {
    free(c->svd_US[k]);
    free(c->svd_V[k]);
    c->svd_US[k] = c->svd_V[k] = NULL;
    c->svd_rank[k] = 0;
  }
  return 0;
}

/* The 16 canonical operators K_that (unit half-width, the formula of
 * m2l_operators), each compressed by its own SVD to the rank
 * r = #{ i : s_i >= eps * s_0 } (Sec. 2.1.2 with (l, eps) = (Acc, 10^-Acc)). */
int ofmm_set_m2l_svd(ofmm* c, double eps) {
  int C = c->ncoef, bad = 0;
  if (c->leaf < 2 || eps <= 0.0 || c->kc != 0.0) return -1;
  c->svd_eps = eps;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : bad)
  for (int k = 0; k < 16; ++k) {
    int that[3], kk = 0;
    for (int a = 0; a <= 3; ++a)
      for (int b = a; b <= 3; ++b)
        for (int cc = b; cc <= 3; ++cc)
          if (cc >= 2) {
            if (kk == k) {
              that[0] = a;
              that[1] = b;
              that[2] = cc;
            }
            ++kk;
          }
    const double* K = c->K + (size_t)tslot(that[0], that[1], that[2]) * C * C;
    double* U = (double*)malloc(sizeof(double) * C * C);
    double* V = (double*)malloc(sizeof(double) * C * C);
    double* s = (double*)malloc(sizeof(double) * C);
    if (ofmm_jacobi_svd(C, K, U, s, V) < 0) bad += 1;
    int r = 0;
    while (r < C && s[r] >= eps * s[0]) ++r;
    free(c->svd_US[k]);
    free(c->svd_V[k]);
    c->svd_rank[k] = r;
    c->svd_US[k] = (double*)malloc(sizeof(double) * C * (r ? r : 1));
    c->svd_V[k] = (double*)malloc(sizeof(double) * C * (r ? r : 1));
    for (int m = 0; m < C; ++m)
      for (int i = 0; i < r; ++i) {
        c->svd_US[k][(size_t)m * r + i] = U[(size_t)m * C + i] * s[i];
        c->svd_V[k][(size_t)m * r + i] = V[(size_t)m * C + i];
      }
    free(U);
    free(V);
    free(s);
  }
  return bad ? -1 : 0;
}

/* Copies the compressed operators of `src` (same order) into `dst`, so that a
 * sequence of trees can share one set of SVDs, as the operators depend on
 * the order and eps only.  0 on success. */
int ofmm_copy_m2l_svd(ofmm* dst, const ofmm* src) {
  int C = dst->ncoef;
  if (src->svd_eps <= 0.0 || src->order != dst->order || dst->leaf < 2 || src->ks != dst->ks || dst->kc != 0.0)
    return -1;
  dst->svd_eps = src->svd_eps;
  for (int k = 0; k < 16; ++k) {
    int r = src->svd_rank[k];
    free(dst->svd_US[k]);
    free(dst->svd_V[k]);
    dst->svd_rank[k] = r;
    dst->svd_US[k] = (double*)malloc(sizeof(double) * C * (r ? r : 1));
    dst->svd_V[k] = (double*)malloc(sizeof(double) * C * (r ? r : 1));
    memcpy(dst->svd_US[k], src->svd_US[k], sizeof(double) * C * r);
    memcpy(dst->svd_V[k], src->svd_V[k], sizeof(double) * C * r);
  }
  return 0;
}

int ofmm_svd_rank(const ofmm* c, int k) { return (k >= 0 && k < 16 && c->svd_eps > 0.0) ? c->svd_rank[k] : -1; }

/* out += K_t M for transfer vector t at unit half-width, with the operator
 * the FMM applies: the full K_t, or, with the compression on,
 *     (K_t M)[sigma.m] = (U_k Sigma_k V_k^T Mt)[m],  Mt[n] = M[sigma.n],
 * where t = sigma(that) and k indexes that (K_t[sigma.m][sigma.n] = K_that[m][n]
 * because sigma is an isometry that maps the nodes onto the nodes). */
void ofmm_m2l_apply(const ofmm* c, const int* t, const double* M, double* out) {
  int C = c->ncoef;
  if (c->svd_eps <= 0.0 && !c->K) return; /* kc > 0: no unit-half-width set */
  if (c->svd_eps <= 0.0) {
    const double* K = c->K + (size_t)tslot(t[0], t[1], t[2]) * C * C;
    for (int m = 0; m < C; ++m) {
      double s = 0.0;
      for (int nn = 0; nn < C; ++nn) s += K[(size_t)m * C + nn] * M[nn];
      out[m] += s;
    }
    return;
  }
  int that[3], axis[3], sign[3];
  ofmm_transfer_symmetry(t, that, axis, sign);
  int k = ofmm_canonical_index(that), r = c->svd_rank[k];
  int32_t* sm = (int32_t*)malloc(sizeof(int32_t) * C);
  double* y = (double*)calloc(r ? r : 1, sizeof(double));
  ofmm_node_permutation(c->order, axis, sign, sm);
  for (int nn = 0; nn < C; ++nn)
    for (int i = 0; i < r; ++i) y[i] += c->svd_V[k][(size_t)nn * r + i] * M[sm[nn]];
  for (int m = 0; m < C; ++m) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s += c->svd_US[k][(size_t)m * r + i] * y[i];
    out[sm[m]] += s;
  }
  free(sm);
  free(y);
}

/* M2L at one cell with the compressed operators (same sum as m2l_cell). */
static void m2l_cell_svd(ofmm* c, int l, int64_t T, int64_t* src, int* tv, double* z) {
  int C = c->ncoef;
  double a = ldexp(c->width, -l - 1);
  double* LT = c->L[l] + (size_t)T * C;
  for (int m = 0; m < C; ++m) LT[m] = 0.0;
  int nf = far_list(c, l, T, src, tv);
  for (int k = 0; k < nf; ++k) {
    for (int m = 0; m < C; ++m) z[m] = 0.0;
    ofmm_m2l_apply(c, tv + 3 * k, c->M[l] + (size_t)src[k] * C, z);
    for (int m = 0; m < C; ++m) LT[m] += scale_a(z[m], a, c->ks);
  }
}

void ofmm_m2l(ofmm* c) {
  for (int l = 2; l <= c->leaf; ++l) {
#pragma omp parallel
    {
      int64_t src[216];
      int tv[3 * 216];
      double* z = (double*)malloc(sizeof(double) * c->ncoef);
#pragma omp for schedule(dynamic, 4)
      for (int64_t T = 0; T < c->ncell[l]; ++T) {
        if (c->svd_eps > 0.0) m2l_cell_svd(c, l, T, src, tv, z);
        else m2l_cell(c, l, T, src, tv);
      }
      free(z);
    }
  }
}

/* L2L: the child's local expansion adds the parent's evaluated at the
 * child's nodes: L_C[m'] += sum_m S_m(xi_P(child node m')) L_P[m]. */
static void l2l_cell(ofmm* c, int l, int64_t ch) {
  int p = c->order, C = c->ncoef;
  double cp[3], ap, cc[3], ac, A[3][MAXP][MAXP];
  int64_t P = c->parent[l + 1][ch];
  cell_geometry(c, l, P, cp, &ap);
  cell_geometry(c, l + 1, ch, cc, &ac);
  child_weights(c, cc, ac, cp, ap, A);
  const double* LP = c->L[l] + (size_t)P * C;
  double* LC = c->L[l + 1] + (size_t)ch * C;
  for (int mm = 0; mm < C; ++mm) {
    int ax = mm / (p * p), ay = (mm / p) % p, az = mm % p;
    double s = 0.0;
    for (int m = 0; m < C; ++m)
      s += A[0][m / (p * p)][ax] * A[1][(m / p) % p][ay] * A[2][m % p][az] * LP[m];
    LC[mm] += s;
  }
}

void ofmm_l2l(ofmm* c) {
  for (int l = 2; l <= c->leaf - 1; ++l) {
#pragma omp parallel for schedule(dynamic, 8)
    for (int64_t ch = 0; ch < c->ncell[l + 1]; ++ch) l2l_cell(c, l, ch);
  }
}

/* L2P for one particle of leaf `cell`: phi = sum_m S_m(xi) L_m and
 * F = -grad phi = -(1/a) sum_m grad_xi S_m(xi) L_m (eq. 3, gradient on S). */
static void l2p_particle(const ofmm* c, int64_t cell, int64_t r, double* phi, double* F) {
  int p = c->order, C = c->ncoef, Lf = c->leaf;
  double ctr[3], a, S[3][MAXP], dS[3][MAXP];
  cell_geometry(c, Lf, cell, ctr, &a);
  for (int d = 0; d < 3; ++d) {
    double xi = (c->x[3 * r + d] - ctr[d]) / a;
    for (int k = 0; k < p; ++k) {
      S[d][k] = ofmm_cheb_S(p, c->xbar[k], xi);
      dS[d][k] = ofmm_cheb_dS(p, c->xbar[k], xi);
    }
  }
  const double* L = c->L[Lf] + (size_t)cell * C;
  double f = 0.0, g[3] = {0.0, 0.0, 0.0};
  for (int m = 0; m < C; ++m) {
    int mx = m / (p * p), my = (m / p) % p, mz = m % p;
    f += L[m] * S[0][mx] * S[1][my] * S[2][mz];
    g[0] += L[m] * dS[0][mx] * S[1][my] * S[2][mz];
    g[1] += L[m] * S[0][mx] * dS[1][my] * S[2][mz];
    g[2] += L[m] * S[0][mx] * S[1][my] * dS[2][mz];
  }
  *phi = f;
  for (int d = 0; d < 3; ++d) F[d] = -g[d] / a;
}

void ofmm_l2p(const ofmm* c, double* phi, double* F) {
  int Lf = c->leaf;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t cell = 0; cell < c->ncell[Lf]; ++cell)
    for (int64_t r = c->first[Lf][cell]; r < c->first[Lf][cell] + c->count[Lf][cell]; ++r)
      l2p_particle(c, cell, r, &phi[r], &F[3 * r]);
}

/* P2P for one particle: eq. 1 with the kernels of eq. 2 over the particles of
 * the near-field leaves, skipping the particle itself and r = 0. */
static void p2p_particle(const ofmm* c, const int64_t* src, int ns, int64_t r, double* phi,
                         double* F) {
  int Lf = c->leaf;
  double f = 0.0, g[3] = {0.0, 0.0, 0.0};
  const double* xi = c->x + 3 * r;
  for (int k = 0; k < ns; ++k)
    for (int64_t j = c->first[Lf][src[k]]; j < c->first[Lf][src[k]] + c->count[Lf][src[k]]; ++j) {
      if (j == r) continue;
      double d[3] = {xi[0] - c->x[3 * j], xi[1] - c->x[3 * j + 1], xi[2] - c->x[3 * j + 2]};
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 == 0.0) continue;
      if (c->ks == 1.0 && c->kc == 0.0) {
        double rr = sqrt(r2);
        f += c->q[j] / rr;
        for (int e = 0; e < 3; ++e) g[e] += c->q[j] * d[e] / (rr * r2);
      } else { /* F = -grad phi = s q d (|d|^2 + kc^2)^-(s+2)/2 */
        double re = r2 + c->kc * c->kc;
        double pk = c->q[j] * pow(re, -0.5 * c->ks);
        f += pk;
        for (int e = 0; e < 3; ++e) g[e] += c->ks * pk * d[e] / re;
      }
    }
  *phi = f;
  for (int e = 0; e < 3; ++e) F[e] = g[e];
}

void ofmm_p2p(const ofmm* c, double* phi, double* F) {
  int Lf = c->leaf;
#pragma omp parallel
  {
    int64_t src[27];
#pragma omp for schedule(dynamic, 8)
    for (int64_t cell = 0; cell < c->ncell[Lf]; ++cell) {
      int ns = near_list(c, cell, src);
      for (int64_t r = c->first[Lf][cell]; r < c->first[Lf][cell] + c->count[Lf][cell]; ++r)
        p2p_particle(c, src, ns, r, &phi[r], &F[3 * r]);
    }
  }
}

void ofmm_evaluate(ofmm* c, double* phi, double* F) {
  int64_t n = c->n;
  double* pf = (double*)calloc(n ? n : 1, sizeof(double));
  double* Ff = (double*)calloc(3 * (n ? n : 1), sizeof(double));
  double* pn = (double*)calloc(n ? n : 1, sizeof(double));
  double* Fn = (double*)calloc(3 * (n ? n : 1), sizeof(double));
  if (c->leaf >= 2) {
    ofmm_p2m(c);
    ofmm_m2m(c);
    ofmm_m2l(c);
    ofmm_l2l(c);
    ofmm_l2p(c, pf, Ff);
  }
  ofmm_p2p(c, pn, Fn);
  for (int64_t r = 0; r < n; ++r) {
    int64_t i = c->perm[r];
    phi[i] = pf[r] + pn[r];
    for (int d = 0; d < 3; ++d) F[3 * i + d] = Ff[3 * r + d] + Fn[3 * r + d];
  }
  free(pf);
  free(Ff);
  free(pn);
  free(Fn);
}

/* Leaf cell holding Morton rank r (binary search over leaf first ranks). */
static int64_t leaf_of_rank(const ofmm* c, int64_t r) {
  int Lf = c->leaf;
  int64_t a = 0, b = c->ncell[Lf] - 1;
  while (a < b) {
    int64_t m = a + (b - a + 1) / 2;
    if (c->first[Lf][m] <= r) a = m;
    else b = m - 1;
  }
  return a;
}

void ofmm_evaluate_sampled(ofmm* c, int64_t ns, const int64_t* idx, double* phi, double* F) {
  int Lf = c->leaf;
  int64_t n = c->n;
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (n ? n : 1));
  for (int64_t r = 0; r < n; ++r) rank[c->perm[r]] = r;
  if (Lf >= 2) {
    ofmm_p2m(c);
    ofmm_m2m(c);
    /* mark the ancestors of every sampled particle's leaf */
    char* need[MAXH];
    for (int l = 0; l <= Lf; ++l) need[l] = (char*)calloc(c->ncell[l] ? c->ncell[l] : 1, 1);
    for (int64_t s = 0; s < ns; ++s) {
      int64_t cell = leaf_of_rank(c, rank[idx[s]]);
      for (int l = Lf; l >= 2; --l) {
        need[l][cell] = 1;
        cell = c->parent[l][cell];
      }
    }
    for (int l = 2; l <= Lf; ++l) {
#pragma omp parallel
      {
        int64_t src[216];
        int tv[3 * 216];
        double* z = (double*)malloc(sizeof(double) * c->ncoef);
#pragma omp for schedule(dynamic, 1)
        for (int64_t T = 0; T < c->ncell[l]; ++T) {
          if (!need[l][T]) continue;
          if (c->svd_eps > 0.0) m2l_cell_svd(c, l, T, src, tv, z);
          else m2l_cell(c, l, T, src, tv);
        }
        free(z);
      }
      if (l > 2) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t T = 0; T < c->ncell[l]; ++T)
          if (need[l][T]) l2l_cell(c, l - 1, T);
      }
    }
    for (int l = 0; l <= Lf; ++l) free(need[l]);
  }
#pragma omp parallel
  {
    int64_t src[27];
#pragma omp for schedule(dynamic, 1)
    for (int64_t s = 0; s < ns; ++s) {
      int64_t r = rank[idx[s]];
      int64_t cell = leaf_of_rank(c, r);
      double pf = 0.0, Ff[3] = {0.0, 0.0, 0.0}, pn, Fn[3];
      if (Lf >= 2) l2p_particle(c, cell, r, &pf, Ff);
      int nsrc = near_list(c, cell, src);
      p2p_particle(c, src, nsrc, r, &pn, Fn);
      phi[s] = pf + pn;
      for (int d = 0; d < 3; ++d) F[3 * s + d] = Ff[d] + Fn[d];
    }
  }
  free(rank);
}

int64_t ofmm_m2l_pair_count(const ofmm* c, int level) {
  int64_t total = 0;
  if (level < 2 || level > c->leaf) return 0;
#pragma omp parallel reduction(+ : total)
  {
    int64_t src[216];
    int tv[3 * 216];
#pragma omp for schedule(static)
    for (int64_t T = 0; T < c->ncell[level]; ++T) total += far_list(c, level, T, src, tv);
  }
  return total;
}

void ofmm_coverage(const ofmm* c, int32_t* counts) {
  int Lf = c->leaf;
  int64_t nl = c->ncell[Lf];
  memset(counts, 0, sizeof(int32_t) * nl * nl);
  int64_t* anc = (int64_t*)malloc(sizeof(int64_t) * (nl ? nl : 1) * (Lf + 1));
  for (int64_t i = 0; i < nl; ++i) {
    int64_t cell = i;
    for (int l = Lf; l >= 0; --l) {
      anc[i * (Lf + 1) + l] = cell;
      if (l > 0) cell = c->parent[l][cell];
    }
  }
  int64_t src[216];
  int tv[3 * 216];
  for (int64_t T = 0; T < nl; ++T) {
    int ns = near_list(c, T, src);
    for (int k = 0; k < ns; ++k) counts[T * nl + src[k]]++;
    for (int l = 2; l <= Lf; ++l) {
      int nf = far_list(c, l, anc[T * (Lf + 1) + l], src, tv);
      for (int k = 0; k < nf; ++k)
        for (int64_t S = 0; S < nl; ++S)
          if (anc[S * (Lf + 1) + l] == src[k]) counts[T * nl + S]++;
    }
  }
  free(anc);
}

/* ------------------------------------------------------------------------ */
/* Direct summation, eq. 1 with eq. 2                                        */
/* ------------------------------------------------------------------------ */

static void direct_one(int64_t n, const double* xyz, const double* q, double ks, double kc, int64_t i,
                       double* phi, double* F) {
  double f = 0.0, g[3] = {0.0, 0.0, 0.0};
  for (int64_t j = 0; j < n; ++j) {
    if (j == i) continue;
    double d[3] = {xyz[3 * i] - xyz[3 * j], xyz[3 * i + 1] - xyz[3 * j + 1],
                   xyz[3 * i + 2] - xyz[3 * j + 2]};
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (r2 == 0.0) continue;
    if (ks == 1.0 && kc == 0.0) {
      double r = sqrt(r2);
      f += q[j] / r;
      for (int e = 0; e < 3; ++e) g[e] += q[j] * d[e] / (r * r2);
    } else { /* P = (|d|^2 + kc^2)^(-s/2), F = -grad phi = s q d (|d|^2 + kc^2)^-(s+2)/2 */
      double re = r2 + kc * kc;
      double pk = q[j] * pow(re, -0.5 * ks);
      f += pk;
      for (int e = 0; e < 3; ++e) g[e] += ks * pk * d[e] / re;
    }
  }
  *phi = f;
  for (int e = 0; e < 3; ++e) F[e] = g[e];
}

void ofmm_direct_kernel(int64_t n, const double* xyz, const double* q, double ks, double kc, double* phi,
                        double* F) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) direct_one(n, xyz, q, ks, kc, i, &phi[i], &F[3 * i]);
}

void ofmm_direct_sampled_kernel(int64_t n, const double* xyz, const double* q, double ks, double kc, int64_t ns,
                                const int64_t* idx, double* phi, double* F) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t s = 0; s < ns; ++s) direct_one(n, xyz, q, ks, kc, idx[s], &phi[s], &F[3 * s]);
}

/* Stokeslet sums (the Stokes kernel of the black-box method, unit viscosity
 * factor): u_i = sum_{k != i, r > 0} [ f_k / r + d (d . f_k) / r^3 ],
 * d = x_i - x_k, r = |d|; xyz [n][3], f [n][3], u [n][3]. */
void ofmm_stokes_direct(int64_t n, const double* xyz, const double* f, double* u) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < n; ++i) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = 0; k < n; ++k) {
      if (k == i) continue;
      double d[3] = {xyz[3 * i] - xyz[3 * k], xyz[3 * i + 1] - xyz[3 * k + 1], xyz[3 * i + 2] - xyz[3 * k + 2]};
      double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
      if (r2 == 0.0) continue;
      double r = sqrt(r2);
      double df = d[0] * f[3 * k] + d[1] * f[3 * k + 1] + d[2] * f[3 * k + 2];
      for (int e = 0; e < 3; ++e) acc[e] += f[3 * k + e] / r + d[e] * df / (r * r2);
    }
    for (int e = 0; e < 3; ++e) u[3 * i + e] = acc[e];
  }
}

void ofmm_direct(int64_t n, const double* xyz, const double* q, double* phi, double* F) {
  ofmm_direct_kernel(n, xyz, q, 1.0, 0.0, phi, F);
}

void ofmm_direct_sampled(int64_t n, const double* xyz, const double* q, int64_t ns,
                         const int64_t* idx, double* phi, double* F) {
  ofmm_direct_sampled_kernel(n, xyz, q, 1.0, 0.0, ns, idx, phi, F);
}
