/*
 * oracle_fmm.c -- expansions, octree + lists, and the plain CPU FMM.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain FP64; every loop is the
 * textbook formula.  Must be compiled with -ffp-contract=off so that the
 * quantities that decide integers (Morton keys, cell centres, radii, the MAC)
 * are the rounded results of the stated operations in the stated order.
 *
 * Readings of the paper used here (the paper is silent on these points):
 *  - bounding cube (Sec. 3.1): lo = componentwise minimum of the nodes,
 *    side = (largest extent) * (1 + 2^-20), scale = 2^21 / side;
 *    quantised coordinate q = min(2^21-1, trunc((x - lo) * scale));
 *  - 63-bit Morton key, bit b of q_x -> bit 3b, q_y -> 3b+1, q_z -> 3b+2;
 *  - a tet belongs to the box of its centroid ((v0+v1)+(v2+v3))*0.25, a node
 *    to the box of its own position; sort by (key, original index);
 *  - a cell is split iff it holds more than leaf_size tets and its level is
 *    below 20; empty children (no tet and no node) are dropped; cells are
 *    numbered level by level, ascending key prefix within a level;
 *  - expansion centre = geometric box centre lo + (k + 0.5) side / 2^level;
 *  - source radius (Sec. 3.2) = max distance from the centre to any vertex of
 *    any tet of the cell; target radius = max distance to the cell's nodes;
 *  - MAC (Sec. 3.2): accept iff (r_T + r_S) < theta * |c_T - c_S|;
 *  - dual tree traversal (Sec. 3.3, Listings 1-2) with the MAC tested before
 *    the leaf-leaf test; the target is split iff it is the larger box (lower
 *    level) and not a leaf, else the source if it is not a leaf, else the
 *    target; pairs with no target node or no source tet are dropped;
 *  - lists are reported sorted by (target cell, source cell);
 *  - Taylor truncation |n| <= p (Sec. 2.2) and |n| + |m| <= p in M2L.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI (4.0 * 3.14159265358979323846)
#define MAX_LEVEL 20
#define KEY_BITS 21

/* ------------------------------------------------------------------------- */
/* multi-indices                                                              */
/* ------------------------------------------------------------------------- */
int oracle_ncoef(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

void oracle_multi_indices(int p, int32_t* nxyz) {
  int i = 0;
  for (int t = 0; t <= p; t++)
    for (int nx = t; nx >= 0; nx--)
      for (int ny = t - nx; ny >= 0; ny--) {
        nxyz[3 * i] = nx;
        nxyz[3 * i + 1] = ny;
        nxyz[3 * i + 2] = t - nx - ny;
        i++;
      }
}

typedef struct {
  int p, nc;
  int32_t* n;  /* nc x 3 */
  int* lut;    /* (p+1)^3, -1 if |n|>p */
} mi_table;

static void mi_init(mi_table* m, int p) {
  m->p = p;
  m->nc = oracle_ncoef(p);
  m->n = malloc(sizeof(int32_t) * 3 * m->nc);
  oracle_multi_indices(p, m->n);
  int P = p + 1;
  m->lut = malloc(sizeof(int) * P * P * P);
  for (int i = 0; i < P * P * P; i++) m->lut[i] = -1;
  for (int i = 0; i < m->nc; i++) m->lut[(m->n[3 * i] * P + m->n[3 * i + 1]) * P + m->n[3 * i + 2]] = i;
}
static void mi_free(mi_table* m) {
  free(m->n);
  free(m->lut);
}
static inline int mi_idx(const mi_table* m, int a, int b, int c) {
  if (a < 0 || b < 0 || c < 0 || a + b + c > m->p) return -1;
  int P = m->p + 1;
  return m->lut[(a * P + b) * P + c];
}

static double factorial(int n) {
  double f = 1;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}
static double binom(int n, int k) {
  if (k < 0 || k > n) return 0;
  double b = 1;
  for (int i = 1; i <= k; i++) b = b * (n - k + i) / i;
  return b;
}
static double ipow(double x, int e) {
  double r = 1;
  for (int i = 0; i < e; i++) r *= x;
  return r;
}

/* ------------------------------------------------------------------------- */
/* D_n(x) = d^n(1/|x|) (Sec. 2.2 expansion kernel).  Recurrence obtained by  */
/* applying d^m (m = n - e_i) to the identity |x|^2 d_i(1/|x|) + x_i/|x| = 0  */
/* with the Leibniz rule:                                                     */
/*  r^2 D_n = -2 sum_j m_j x_j D_{n-e_j} - sum_j m_j(m_j-1) D_{n-2e_j}        */
/*            - x_i D_{n-e_i} - m_i D_{n-2e_i}.                               */
/* ------------------------------------------------------------------------- */
static void laplace_derivs_tab(const mi_table* T, const double x[3], double* D) {
  double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  D[0] = 1.0 / sqrt(r2);
  for (int id = 1; id < T->nc; id++) {
    int n[3] = {T->n[3 * id], T->n[3 * id + 1], T->n[3 * id + 2]};
    int i = n[0] > 0 ? 0 : (n[1] > 0 ? 1 : 2);
    double s = 0;
    for (int j = 0; j < 3; j++) {
      int mj = n[j] - (j == i);
      int nm[3] = {n[0], n[1], n[2]};
      nm[j] -= 1;
      if (mj > 0) s += 2.0 * mj * x[j] * D[mi_idx(T, nm[0], nm[1], nm[2])];
      nm[j] -= 1;
      if (mj > 1) s += (double)mj * (mj - 1) * D[mi_idx(T, nm[0], nm[1], nm[2])];
    }
    int ni[3] = {n[0], n[1], n[2]};
    ni[i] -= 1;
    s += x[i] * D[mi_idx(T, ni[0], ni[1], ni[2])];
    int mi = n[i] - 1;
    ni[i] -= 1;
    if (mi > 0) s += mi * D[mi_idx(T, ni[0], ni[1], ni[2])];
    D[id] = -s / r2;
  }
}

void oracle_laplace_derivs(const double x[3], int p, double* D) {
  mi_table T;
  mi_init(&T, p);
  laplace_derivs_tab(&T, x, D);
  mi_free(&T);
}

/* ------------------------------------------------------------------------- */
/* Exact tet moments, Eq. (expCoeffs): Q_n = int_tet M . grad(y^n) dV with    */
/* y = r' - c.  The integrand is a polynomial of degree |n| <= p, integrated  */
/* exactly by the collapsed-cube Gauss-Legendre product rule with             */
/* q = ceil((p+3)/2) points per direction (the map adds degree 2 in u and 1   */
/* in v through the Jacobian (1-u)^2 (1-v)).                                  */
/* ------------------------------------------------------------------------- */
static void gl01(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; i++) {
    double z = cos(pi * (i + 0.75) / (n + 0.5)), pp = 1;
    for (int it = 0; it < 100; it++) {
      double p1 = 1, p2 = 0;
      for (int j = 1; j <= n; j++) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double dz = p1 / pp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * pp * pp);
  }
}

typedef struct {
  int q;
  double x[16], w[16];
} gl_rule;

static void tet_moments_tab(const mi_table* T, const gl_rule* G, const double v[12], const double M[12],
                            const double c[3], double* Q) {
  int p = T->p;
  double e1[3], e2[3], e3[3];
  for (int a = 0; a < 3; a++) {
    e1[a] = v[3 + a] - v[a];
    e2[a] = v[6 + a] - v[a];
    e3[a] = v[9 + a] - v[a];
  }
  double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
               e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
  for (int i = 0; i < T->nc; i++) Q[i] = 0;
  double pw[3][16];
  for (int i = 0; i < G->q; i++)
    for (int j = 0; j < G->q; j++)
      for (int k = 0; k < G->q; k++) {
        double u = G->x[i], s = G->x[j], t = G->x[k];
        /* barycentric coordinates of the point: lambda_1..3 = (x, y, z) */
        double l1 = u, l2 = s * (1 - u), l3 = t * (1 - u) * (1 - s), l0 = 1 - l1 - l2 - l3;
        double wt = G->w[i] * G->w[j] * G->w[k] * (1 - u) * (1 - u) * (1 - s) * fabs(det);
        double Mq[3], y[3];
        for (int a = 0; a < 3; a++) {
          Mq[a] = l0 * M[a] + l1 * M[3 + a] + l2 * M[6 + a] + l3 * M[9 + a];
          y[a] = v[a] + l1 * e1[a] + l2 * e2[a] + l3 * e3[a] - c[a];
          pw[a][0] = 1;
          for (int e = 1; e <= p; e++) pw[a][e] = pw[a][e - 1] * y[a];
        }
        for (int id = 1; id < T->nc; id++) {
          int nx = T->n[3 * id], ny = T->n[3 * id + 1], nz = T->n[3 * id + 2];
          double g = 0;
          if (nx) g += nx * Mq[0] * pw[0][nx - 1] * pw[1][ny] * pw[2][nz];
          if (ny) g += ny * Mq[1] * pw[0][nx] * pw[1][ny - 1] * pw[2][nz];
          if (nz) g += nz * Mq[2] * pw[0][nx] * pw[1][ny] * pw[2][nz - 1];
          Q[id] += wt * g;
        }
      }
}

static void gl_rule_for(int p, gl_rule* G) {
  G->q = (p + 4) / 2; /* ceil((p+3)/2) */
  gl01(G->q, G->x, G->w);
}

void oracle_tet_moments(const double v[12], const double M[12], const double c[3], int p, double* Q) {
  mi_table T;
  mi_init(&T, p);
  gl_rule G;
  gl_rule_for(p, &G);
  tet_moments_tab(&T, &G, v, M, c, Q);
  mi_free(&T);
}

/* int_tet lambda_0^a0 ... lambda_3^a3 dV = 6|tet| a0! a1! a2! a3! / (a0+a1+a2+a3+3)!
 * applied to the multinomial expansion of lambda_k y^m, y = sum_l lambda_l (v_l - c). */
double oracle_tet_lambda_monomial_exact(const double v[12], const double c[3], int k, int mx, int my, int mz) {
  int D = mx + my + mz + 1;
  int P = D + 1;
  size_t sz = (size_t)P * P * P * P;
  double* poly = calloc(sz, sizeof(double));
  double* tmp = calloc(sz, sizeof(double));
  poly[0] = 1.0; /* constant 1 */
  int ms[3] = {mx, my, mz};
  for (int a = 0; a < 3; a++)
    for (int rep = 0; rep < ms[a]; rep++) {
      memset(tmp, 0, sz * sizeof(double));
      for (int i0 = 0; i0 < P; i0++)
        for (int i1 = 0; i1 < P; i1++)
          for (int i2 = 0; i2 < P; i2++)
            for (int i3 = 0; i3 < P; i3++) {
              double cf = poly[((i0 * P + i1) * P + i2) * P + i3];
              if (cf == 0) continue;
              int ex[4] = {i0, i1, i2, i3};
              for (int l = 0; l < 4; l++) {
                int e2[4] = {ex[0], ex[1], ex[2], ex[3]};
                e2[l] += 1;
                if (e2[l] >= P) continue;
                tmp[((e2[0] * P + e2[1]) * P + e2[2]) * P + e2[3]] += cf * (v[3 * l + a] - c[a]);
              }
            }
      memcpy(poly, tmp, sz * sizeof(double));
    }
  double e1[3], e2v[3], e3[3];
  for (int a = 0; a < 3; a++) {
    e1[a] = v[3 + a] - v[a];
    e2v[a] = v[6 + a] - v[a];
    e3[a] = v[9 + a] - v[a];
  }
  double det = e1[0] * (e2v[1] * e3[2] - e2v[2] * e3[1]) - e1[1] * (e2v[0] * e3[2] - e2v[2] * e3[0]) +
               e1[2] * (e2v[0] * e3[1] - e2v[1] * e3[0]);
  double vol = fabs(det) / 6.0;
  double s = 0;
  for (int i0 = 0; i0 < P; i0++)
    for (int i1 = 0; i1 < P; i1++)
      for (int i2 = 0; i2 < P; i2++)
        for (int i3 = 0; i3 < P; i3++) {
          double cf = poly[((i0 * P + i1) * P + i2) * P + i3];
          if (cf == 0) continue;
          int ex[4] = {i0, i1, i2, i3};
          ex[k] += 1; /* times lambda_k */
          int tot = ex[0] + ex[1] + ex[2] + ex[3];
          s += cf * 6.0 * vol * factorial(ex[0]) * factorial(ex[1]) * factorial(ex[2]) * factorial(ex[3]) /
               factorial(tot + 3);
        }
  free(poly);
  free(tmp);
  return s;
}

/* ------------------------------------------------------------------------- */
/* translations                                                               */
/* ------------------------------------------------------------------------- */
static void m2m_tab(const mi_table* T, const double d[3], const double* Qc, double* Qp) {
  int p = T->p;
  double pw[3][32];
  for (int a = 0; a < 3; a++) {
    pw[a][0] = 1;
    for (int e = 1; e <= p; e++) pw[a][e] = pw[a][e - 1] * d[a];
  }
  for (int id = 0; id < T->nc; id++) {
    int n0 = T->n[3 * id], n1 = T->n[3 * id + 1], n2 = T->n[3 * id + 2];
    double s = 0;
    for (int k0 = 0; k0 <= n0; k0++)
      for (int k1 = 0; k1 <= n1; k1++)
        for (int k2 = 0; k2 <= n2; k2++) {
          double cf = binom(n0, k0) * binom(n1, k1) * binom(n2, k2) * pw[0][n0 - k0] * pw[1][n1 - k1] * pw[2][n2 - k2];
          s += cf * Qc[mi_idx(T, k0, k1, k2)];
        }
    Qp[id] += s;
  }
}

static void m2l_tab(const mi_table* T, const double R[3], const double* Q, double* L, double* Dbuf) {
  laplace_derivs_tab(T, R, Dbuf);
  int p = T->p;
  for (int im = 0; im < T->nc; im++) {
    int m0 = T->n[3 * im], m1 = T->n[3 * im + 1], m2 = T->n[3 * im + 2];
    int tm = m0 + m1 + m2;
    double s = 0;
    for (int in = 0; in < T->nc; in++) {
      int n0 = T->n[3 * in], n1 = T->n[3 * in + 1], n2 = T->n[3 * in + 2];
      int tn = n0 + n1 + n2;
      if (tn + tm > p) break; /* graded order: all later n have |n| >= tn */
      double sg = (tn & 1) ? -1.0 : 1.0;
      s += sg / (factorial(n0) * factorial(n1) * factorial(n2)) * Dbuf[mi_idx(T, n0 + m0, n1 + m1, n2 + m2)] * Q[in];
    }
    L[im] += s / FOUR_PI;
  }
}

static void l2l_tab(const mi_table* T, const double d[3], const double* Lp, double* Lc) {
  int p = T->p;
  double pw[3][32];
  for (int a = 0; a < 3; a++) {
    pw[a][0] = 1;
    for (int e = 1; e <= p; e++) pw[a][e] = pw[a][e - 1] * d[a];
  }
  for (int im = 0; im < T->nc; im++) {
    int m0 = T->n[3 * im], m1 = T->n[3 * im + 1], m2 = T->n[3 * im + 2];
    double s = 0;
    for (int ik = 0; ik < T->nc; ik++) {
      int k0 = T->n[3 * ik], k1 = T->n[3 * ik + 1], k2 = T->n[3 * ik + 2];
      if (k0 < m0 || k1 < m1 || k2 < m2) continue;
      s += Lp[ik] * pw[0][k0 - m0] * pw[1][k1 - m1] * pw[2][k2 - m2] /
           (factorial(k0 - m0) * factorial(k1 - m1) * factorial(k2 - m2));
    }
    Lc[im] += s;
  }
}

static double l2p_tab(const mi_table* T, const double z[3], const double* L) {
  double s = 0;
  for (int im = 0; im < T->nc; im++) {
    int m0 = T->n[3 * im], m1 = T->n[3 * im + 1], m2 = T->n[3 * im + 2];
    s += L[im] * ipow(z[0], m0) * ipow(z[1], m1) * ipow(z[2], m2) / (factorial(m0) * factorial(m1) * factorial(m2));
  }
  return s;
}

void oracle_m2m(int p, const double d[3], const double* Qc, double* Qp) {
  mi_table T;
  mi_init(&T, p);
  m2m_tab(&T, d, Qc, Qp);
  mi_free(&T);
}
void oracle_m2l(int p, const double R[3], const double* Q, double* L) {
  mi_table T;
  mi_init(&T, p);
  double* D = malloc(sizeof(double) * T.nc);
  m2l_tab(&T, R, Q, L, D);
  free(D);
  mi_free(&T);
}
void oracle_l2l(int p, const double d[3], const double* Lp, double* Lc) {
  mi_table T;
  mi_init(&T, p);
  l2l_tab(&T, d, Lp, Lc);
  mi_free(&T);
}
double oracle_l2p(int p, const double z[3], const double* L) {
  mi_table T;
  mi_init(&T, p);
  double s = l2p_tab(&T, z, L);
  mi_free(&T);
  return s;
}
double oracle_multipole_eval(int p, const double c[3], const double* Q, const double r[3]) {
  mi_table T;
  mi_init(&T, p);
  double* D = malloc(sizeof(double) * T.nc);
  double x[3] = {r[0] - c[0], r[1] - c[1], r[2] - c[2]};
  laplace_derivs_tab(&T, x, D);
  double s = 0;
  for (int id = 0; id < T.nc; id++) {
    int n0 = T.n[3 * id], n1 = T.n[3 * id + 1], n2 = T.n[3 * id + 2];
    double sg = ((n0 + n1 + n2) & 1) ? -1.0 : 1.0;
    s += sg / (factorial(n0) * factorial(n1) * factorial(n2)) * D[id] * Q[id];
  }
  free(D);
  mi_free(&T);
  return s / FOUR_PI;
}

/* ------------------------------------------------------------------------- */
/* octree (Sec. 3.1), radii and MAC (Sec. 3.2), traversal (Sec. 3.3)          */
/* ------------------------------------------------------------------------- */
struct oracle_tree {
  int64_t nn, nt;
  int leaf;
  double theta;
  double lo[3], side, scale;
  const double* nodes; /* caller's arrays are copied */
  double* nodes_c;
  int32_t* tets_c;
  uint64_t *node_key, *tet_key;
  int64_t *node_perm, *tet_perm;
  int64_t ncells, cap;
  int32_t* level;
  uint64_t* prefix;
  int64_t *tb, *te, *nb, *ne, *parent, *child0;
  int32_t* nchild;
  double *centre, *r_src, *r_tgt;
  int nlevels;
  int64_t n_m2l, n_p2p;
  int64_t *m2l_off, *m2l_src, *p2p_off, *p2p_src;
  int dipoles;      /* sources: point dipoles V_i M_i at the nodes */
  int patches;      /* sources: vertex patches lambda_i M_i over the tets around node i */
  double* node_vol; /* lumped nodal volumes (dipole sources) */
  int64_t *nt_off, *nt_tet; /* node -> incident tets (vertex patches) */
};

static uint64_t spread_bits(uint64_t q) {
  uint64_t k = 0;
  for (int b = 0; b < KEY_BITS; b++) k |= ((q >> b) & 1ull) << (3 * b);
  return k;
}
static uint64_t compact_bits(uint64_t k) {
  uint64_t q = 0;
  for (int b = 0; b < KEY_BITS; b++) q |= ((k >> (3 * b)) & 1ull) << b;
  return q;
}
static uint64_t quantise(double x, double lo, double scale) {
  double s = (x - lo) * scale;
  uint64_t q = (uint64_t)s;
  const uint64_t qmax = (1ull << KEY_BITS) - 1;
  return q > qmax ? qmax : q;
}
static uint64_t morton_key(const double x[3], const double lo[3], double scale) {
  return spread_bits(quantise(x[0], lo[0], scale)) | (spread_bits(quantise(x[1], lo[1], scale)) << 1) |
         (spread_bits(quantise(x[2], lo[2], scale)) << 2);
}

typedef struct {
  uint64_t key;
  int64_t idx;
} key_idx;
static int cmp_key_idx(const void* a, const void* b) {
  const key_idx *x = a, *y = b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static void tree_grow(oracle_tree* t) {
  if (t->ncells < t->cap) return;
  t->cap = t->cap ? 2 * t->cap : 1024;
  t->level = realloc(t->level, sizeof(int32_t) * t->cap);
  t->prefix = realloc(t->prefix, sizeof(uint64_t) * t->cap);
  t->tb = realloc(t->tb, sizeof(int64_t) * t->cap);
  t->te = realloc(t->te, sizeof(int64_t) * t->cap);
  t->nb = realloc(t->nb, sizeof(int64_t) * t->cap);
  t->ne = realloc(t->ne, sizeof(int64_t) * t->cap);
  t->parent = realloc(t->parent, sizeof(int64_t) * t->cap);
  t->child0 = realloc(t->child0, sizeof(int64_t) * t->cap);
  t->nchild = realloc(t->nchild, sizeof(int32_t) * t->cap);
}

static double dist3(const double* a, const double* b) {
  double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

typedef struct {
  int64_t *a;
  int64_t n, cap;
} pair_vec; /* pairs stored as 2 int64 */
static void pv_push(pair_vec* v, int64_t x, int64_t y) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 1024;
    v->a = realloc(v->a, sizeof(int64_t) * 2 * v->cap);
  }
  v->a[2 * v->n] = x;
  v->a[2 * v->n + 1] = y;
  v->n++;
}
static int cmp_pair(const void* a, const void* b) {
  const int64_t *x = a, *y = b;
  if (x[0] != y[0]) return x[0] < y[0] ? -1 : 1;
  return x[1] < y[1] ? -1 : (x[1] > y[1]);
}

static int is_leaf(const oracle_tree* t, int64_t c) { return t->nchild[c] == 0; }

static int mac_ok(const oracle_tree* t, int64_t T, int64_t S) {
  double d = dist3(t->centre + 3 * T, t->centre + 3 * S);
  return (t->r_tgt[T] + t->r_src[S]) < t->theta * d;
}

/* Listing 2 with the MAC tested first. */
static void interact(const oracle_tree* t, int64_t A, int64_t B, pair_vec* stack, pair_vec* m2l, pair_vec* p2p) {
  const int node_sources = t->dipoles || t->patches;
  if (t->ne[A] == t->nb[A] || (node_sources ? t->ne[B] == t->nb[B] : t->te[B] == t->tb[B])) return;
  if (mac_ok(t, A, B))
    pv_push(m2l, A, B);
  else if (is_leaf(t, A) && is_leaf(t, B))
    pv_push(p2p, A, B);
  else
    pv_push(stack, A, B);
}

static void build_csr(pair_vec* v, int64_t ncells, int64_t** off, int64_t** src) {
  qsort(v->a, v->n, 2 * sizeof(int64_t), cmp_pair);
  *off = calloc(ncells + 1, sizeof(int64_t));
  *src = malloc(sizeof(int64_t) * (v->n ? v->n : 1));
  for (int64_t i = 0; i < v->n; i++) {
    (*off)[v->a[2 * i] + 1]++;
    (*src)[i] = v->a[2 * i + 1];
  }
  for (int64_t c = 0; c < ncells; c++) (*off)[c + 1] += (*off)[c];
}

oracle_tree* oracle_tree_build(const double* nodes, int64_t nn, const int32_t* tets, int64_t nt, int leaf,
                               double theta, int* status) {
  return oracle_tree_build_sources(nodes, nn, tets, nt, leaf, theta, 0, status);
}

oracle_tree* oracle_tree_build_sources(const double* nodes, int64_t nn, const int32_t* tets, int64_t nt, int leaf,
                                       double theta, int sources, int* status) {
  *status = 1;
  if (!nodes || !tets || nn < 1 || nt < 1 || leaf < 1 || !(theta > 0)) return NULL;
  for (int64_t i = 0; i < 4 * nt; i++)
    if (tets[i] < 0 || tets[i] >= nn) return NULL;
  oracle_tree* t = calloc(1, sizeof(oracle_tree));
  t->nn = nn;
  t->nt = nt;
  t->leaf = leaf;
  t->theta = theta;
  t->dipoles = sources == 1;
  t->patches = sources == 2;
  if (t->patches) { /* node -> incident tets */
    t->nt_off = calloc(nn + 1, sizeof(int64_t));
    for (int64_t q = 0; q < 4 * nt; q++) t->nt_off[tets[q] + 1]++;
    for (int64_t i = 0; i < nn; i++) t->nt_off[i + 1] += t->nt_off[i];
    int64_t* fill = malloc(sizeof(int64_t) * (nn + 1));
    memcpy(fill, t->nt_off, sizeof(int64_t) * (nn + 1));
    t->nt_tet = malloc(sizeof(int64_t) * 4 * nt);
    for (int64_t q = 0; q < 4 * nt; q++) t->nt_tet[fill[tets[q]]++] = q / 4;
    free(fill);
  }
  if (t->dipoles) { /* lumped nodal volumes: a quarter of each incident tet */
    double* vol = malloc(sizeof(double) * nt);
    oracle_tet_volumes(nodes, tets, nt, vol);
    t->node_vol = calloc(nn, sizeof(double));
    for (int64_t j = 0; j < nt; j++)
      for (int k = 0; k < 4; k++) t->node_vol[tets[4 * j + k]] += 0.25 * fabs(vol[j]);
    free(vol);
  }
  t->nodes_c = malloc(sizeof(double) * 3 * nn);
  memcpy(t->nodes_c, nodes, sizeof(double) * 3 * nn);
  t->tets_c = malloc(sizeof(int32_t) * 4 * nt);
  memcpy(t->tets_c, tets, sizeof(int32_t) * 4 * nt);
  t->nodes = t->nodes_c;

  /* bounding cube */
  double hi[3];
  for (int a = 0; a < 3; a++) t->lo[a] = hi[a] = nodes[a];
  for (int64_t i = 1; i < nn; i++)
    for (int a = 0; a < 3; a++) {
      double x = nodes[3 * i + a];
      if (x < t->lo[a]) t->lo[a] = x;
      if (x > hi[a]) hi[a] = x;
    }
  double ext = 0;
  for (int a = 0; a < 3; a++) {
    double e = hi[a] - t->lo[a];
    if (e > ext) ext = e;
  }
  t->side = ext * (1.0 + 1.0 / 1048576.0);
  t->scale = 2097152.0 / t->side;

  /* keys and sort */
  t->node_key = malloc(sizeof(uint64_t) * nn);
  t->tet_key = malloc(sizeof(uint64_t) * nt);
  key_idx* ki = malloc(sizeof(key_idx) * (nn > nt ? nn : nt));
  for (int64_t i = 0; i < nn; i++) {
    t->node_key[i] = morton_key(nodes + 3 * i, t->lo, t->scale);
    ki[i].key = t->node_key[i];
    ki[i].idx = i;
  }
  qsort(ki, nn, sizeof(key_idx), cmp_key_idx);
  t->node_perm = malloc(sizeof(int64_t) * nn);
  for (int64_t i = 0; i < nn; i++) t->node_perm[i] = ki[i].idx;
  for (int64_t j = 0; j < nt; j++) {
    const double *v0 = nodes + 3 * (int64_t)tets[4 * j], *v1 = nodes + 3 * (int64_t)tets[4 * j + 1],
                 *v2 = nodes + 3 * (int64_t)tets[4 * j + 2], *v3 = nodes + 3 * (int64_t)tets[4 * j + 3];
    double cen[3];
    for (int a = 0; a < 3; a++) cen[a] = ((v0[a] + v1[a]) + (v2[a] + v3[a])) * 0.25;
    t->tet_key[j] = morton_key(cen, t->lo, t->scale);
    ki[j].key = t->tet_key[j];
    ki[j].idx = j;
  }
  qsort(ki, nt, sizeof(key_idx), cmp_key_idx);
  t->tet_perm = malloc(sizeof(int64_t) * nt);
  for (int64_t j = 0; j < nt; j++) t->tet_perm[j] = ki[j].idx;
  free(ki);

  /* octree, level by level */
  tree_grow(t);
  t->ncells = 1;
  t->level[0] = 0;
  t->prefix[0] = 0;
  t->tb[0] = 0; t->te[0] = nt; t->nb[0] = 0; t->ne[0] = nn;
  t->parent[0] = -1;
  int64_t lev_begin = 0, lev_end = 1;
  int level = 0;
  while (lev_begin < lev_end) {
    for (int64_t c = lev_begin; c < lev_end; c++) {
      t->child0[c] = -1;
      t->nchild[c] = 0;
      if (!(t->te[c] - t->tb[c] > leaf && level < MAX_LEVEL)) continue;
      int shift = 3 * (KEY_BITS - 1 - level);
      int64_t tpos = t->tb[c], npos = t->nb[c];
      for (int o = 0; o < 8; o++) {
        int64_t t0 = tpos, n0 = npos;
        while (tpos < t->te[c] && (int)((t->tet_key[t->tet_perm[tpos]] >> shift) & 7) == o) tpos++;
        while (npos < t->ne[c] && (int)((t->node_key[t->node_perm[npos]] >> shift) & 7) == o) npos++;
        if (tpos == t0 && npos == n0) continue;
        tree_grow(t);
        int64_t k = t->ncells++;
        t->level[k] = level + 1;
        t->prefix[k] = (t->prefix[c] << 3) | (uint64_t)o;
        t->tb[k] = t0; t->te[k] = tpos; t->nb[k] = n0; t->ne[k] = npos;
        t->parent[k] = c;
        if (t->child0[c] < 0) t->child0[c] = k;
        t->nchild[c]++;
      }
    }
    lev_begin = lev_end;
    lev_end = t->ncells;
    level++;
  }
  t->nlevels = level;

  /* centres and radii */
  t->centre = malloc(sizeof(double) * 3 * t->ncells);
  t->r_src = malloc(sizeof(double) * t->ncells);
  t->r_tgt = malloc(sizeof(double) * t->ncells);
  for (int64_t c = 0; c < t->ncells; c++) {
    double cs = ldexp(t->side, -t->level[c]);
    uint64_t pk = t->prefix[c];
    uint64_t kk[3] = {compact_bits(pk), compact_bits(pk >> 1), compact_bits(pk >> 2)};
    for (int a = 0; a < 3; a++) t->centre[3 * c + a] = t->lo[a] + ((double)kk[a] + 0.5) * cs;
    double rs = 0, rt = 0;
    for (int64_t j = t->tb[c]; j < t->te[c]; j++)
      for (int k = 0; k < 4; k++) {
        double d = dist3(nodes + 3 * (int64_t)tets[4 * t->tet_perm[j] + k], t->centre + 3 * c);
        if (d > rs) rs = d;
      }
    for (int64_t i = t->nb[c]; i < t->ne[c]; i++) {
      double d = dist3(nodes + 3 * t->node_perm[i], t->centre + 3 * c);
      if (d > rt) rt = d;
    }
    if (t->patches) { /* a vertex patch reaches every vertex of the tets around its node */
      rs = 0;
      for (int64_t i = t->nb[c]; i < t->ne[c]; i++) {
        const int64_t g = t->node_perm[i];
        for (int64_t e = t->nt_off[g]; e < t->nt_off[g + 1]; e++)
          for (int k = 0; k < 4; k++) {
            double d = dist3(nodes + 3 * (int64_t)tets[4 * t->nt_tet[e] + k], t->centre + 3 * c);
            if (d > rs) rs = d;
          }
      }
    }
    t->r_src[c] = t->dipoles ? rt : rs; /* dipoles sit at the cell's own nodes */
    t->r_tgt[c] = rt;
  }

  /* dual tree traversal (Listing 1), starting with Interact(root, root) */
  pair_vec stack = {0}, m2l = {0}, p2p = {0};
  interact(t, 0, 0, &stack, &m2l, &p2p);
  while (stack.n > 0) {
    stack.n--;
    int64_t A = stack.a[2 * stack.n], B = stack.a[2 * stack.n + 1];
    int split_target;
    if (t->level[A] < t->level[B] && !is_leaf(t, A))
      split_target = 1;
    else if (!is_leaf(t, B))
      split_target = 0;
    else
      split_target = 1;
    if (split_target) {
      for (int64_t a = t->child0[A]; a < t->child0[A] + t->nchild[A]; a++) interact(t, a, B, &stack, &m2l, &p2p);
    } else {
      for (int64_t b = t->child0[B]; b < t->child0[B] + t->nchild[B]; b++) interact(t, A, b, &stack, &m2l, &p2p);
    }
  }
  t->n_m2l = m2l.n;
  t->n_p2p = p2p.n;
  build_csr(&m2l, t->ncells, &t->m2l_off, &t->m2l_src);
  build_csr(&p2p, t->ncells, &t->p2p_off, &t->p2p_src);
  free(stack.a);
  free(m2l.a);
  free(p2p.a);
  *status = 0;
  return t;
}

void oracle_tree_free(oracle_tree* t) {
  if (!t) return;
  free(t->nodes_c); free(t->tets_c);
  free(t->node_key); free(t->tet_key); free(t->node_perm); free(t->tet_perm);
  free(t->level); free(t->prefix); free(t->tb); free(t->te); free(t->nb); free(t->ne);
  free(t->parent); free(t->child0); free(t->nchild);
  free(t->centre); free(t->r_src); free(t->r_tgt);
  free(t->m2l_off); free(t->m2l_src); free(t->p2p_off); free(t->p2p_src);
  free(t->node_vol);
  free(t->nt_off);
  free(t->nt_tet);
  free(t);
}

void oracle_tree_info(const oracle_tree* t, int64_t* info) {
  int64_t nleaves = 0;
  for (int64_t c = 0; c < t->ncells; c++) nleaves += t->nchild[c] == 0;
  info[0] = t->ncells;
  info[1] = t->n_m2l;
  info[2] = t->n_p2p;
  info[3] = t->nlevels;
  info[4] = nleaves;
}

void oracle_tree_box(const oracle_tree* t, double* o) {
  o[0] = t->lo[0]; o[1] = t->lo[1]; o[2] = t->lo[2];
  o[3] = t->side;
  o[4] = t->scale;
}

void oracle_tree_export(const oracle_tree* t, uint64_t* node_key, uint64_t* tet_key, int64_t* node_perm,
                        int64_t* tet_perm, int32_t* cell_level, uint64_t* cell_prefix, int64_t* cell_ranges,
                        int64_t* cell_parent, int64_t* cell_child, double* cell_centre, double* cell_radius,
                        int64_t* m2l_off, int64_t* m2l_src, int64_t* p2p_off, int64_t* p2p_src) {
  int64_t nc = t->ncells;
  if (node_key) memcpy(node_key, t->node_key, sizeof(uint64_t) * t->nn);
  if (tet_key) memcpy(tet_key, t->tet_key, sizeof(uint64_t) * t->nt);
  if (node_perm) memcpy(node_perm, t->node_perm, sizeof(int64_t) * t->nn);
  if (tet_perm) memcpy(tet_perm, t->tet_perm, sizeof(int64_t) * t->nt);
  if (cell_level) memcpy(cell_level, t->level, sizeof(int32_t) * nc);
  if (cell_prefix) memcpy(cell_prefix, t->prefix, sizeof(uint64_t) * nc);
  for (int64_t c = 0; c < nc; c++) {
    if (cell_ranges) {
      cell_ranges[4 * c] = t->tb[c];
      cell_ranges[4 * c + 1] = t->te[c];
      cell_ranges[4 * c + 2] = t->nb[c];
      cell_ranges[4 * c + 3] = t->ne[c];
    }
    if (cell_parent) cell_parent[c] = t->parent[c];
    if (cell_child) {
      cell_child[2 * c] = t->child0[c];
      cell_child[2 * c + 1] = t->nchild[c];
    }
    if (cell_radius) {
      cell_radius[2 * c] = t->r_src[c];
      cell_radius[2 * c + 1] = t->r_tgt[c];
    }
  }
  if (cell_centre) memcpy(cell_centre, t->centre, sizeof(double) * 3 * nc);
  if (m2l_off) memcpy(m2l_off, t->m2l_off, sizeof(int64_t) * (nc + 1));
  if (m2l_src) memcpy(m2l_src, t->m2l_src, sizeof(int64_t) * t->n_m2l);
  if (p2p_off) memcpy(p2p_off, t->p2p_off, sizeof(int64_t) * (nc + 1));
  if (p2p_src) memcpy(p2p_src, t->p2p_src, sizeof(int64_t) * t->n_p2p);
}

/* ------------------------------------------------------------------------- */
/* FMM evaluation: P2M, M2M, M2L, L2L, L2P (Sec. 2 steps 1-5) + P2P (Sec 2.1) */
/* ------------------------------------------------------------------------- */
static void gather_tet(const oracle_tree* t, int64_t tet, const double* M, int b, double v[12], double Mt[12]) {
  for (int k = 0; k < 4; k++) {
    int64_t g = t->tets_c[4 * tet + k];
    for (int a = 0; a < 3; a++) {
      v[3 * k + a] = t->nodes_c[3 * g + a];
      Mt[3 * k + a] = M[((int64_t)b * t->nn + g) * 3 + a];
    }
  }
}

int oracle_fmm_eval(const oracle_tree* t, int p, const double* M, int B, double* u, const int64_t* target_leaves,
                    int64_t n_target_leaves, int nthreads) {
  if (!t || !M || !u || B < 1 || p < 1 || p > 14) return 1;
#ifdef _OPENMP
  /* thread count of this call only (a num_threads clause, not a global setting) */
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
  mi_table T;
  mi_init(&T, p);
  gl_rule G;
  gl_rule_for(p, &G);
  int nc = T.nc;
  int64_t ncell = t->ncells;
  double* Q = calloc((size_t)B * ncell * nc, sizeof(double));
  double* L = calloc((size_t)B * ncell * nc, sizeof(double));
  char* mark = calloc(ncell, 1);
  int64_t* leaves = NULL;
  int64_t nleaves = 0;
  if (target_leaves) {
    leaves = malloc(sizeof(int64_t) * (n_target_leaves ? n_target_leaves : 1));
    for (int64_t i = 0; i < n_target_leaves; i++) {
      int64_t c = target_leaves[i];
      if (c < 0 || c >= ncell || !is_leaf(t, c)) continue;
      leaves[nleaves++] = c;
      for (int64_t a = c; a >= 0 && !mark[a]; a = t->parent[a]) mark[a] = 1;
    }
  } else {
    leaves = malloc(sizeof(int64_t) * ncell);
    for (int64_t c = 0; c < ncell; c++) {
      mark[c] = 1;
      if (is_leaf(t, c)) leaves[nleaves++] = c;
    }
  }

  /* P2M of point dipoles: Q_n = sum_i V_i M_i . grad(y^n) at y_i = r_i - c, leaves holding nodes */
  if (t->dipoles) {
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t c = 0; c < ncell; c++) {
      if (!is_leaf(t, c) || t->ne[c] == t->nb[c]) continue;
      for (int b = 0; b < B; b++) {
        double* Qc = Q + ((size_t)b * ncell + c) * nc;
        for (int64_t i = t->nb[c]; i < t->ne[c]; i++) {
          const int64_t g = t->node_perm[i];
          const double* m = M + ((int64_t)b * t->nn + g) * 3;
          double pw[3][32];
          for (int a = 0; a < 3; a++) {
            const double y = t->nodes_c[3 * g + a] - t->centre[3 * c + a];
            pw[a][0] = 1;
            for (int e = 1; e <= p; e++) pw[a][e] = pw[a][e - 1] * y;
          }
          for (int id = 1; id < nc; id++) {
            const int nx = T.n[3 * id], ny = T.n[3 * id + 1], nz = T.n[3 * id + 2];
            double gsum = 0;
            if (nx) gsum += nx * m[0] * pw[0][nx - 1] * pw[1][ny] * pw[2][nz];
            if (ny) gsum += ny * m[1] * pw[0][nx] * pw[1][ny - 1] * pw[2][nz];
            if (nz) gsum += nz * m[2] * pw[0][nx] * pw[1][ny] * pw[2][nz - 1];
            Qc[id] += t->node_vol[g] * gsum;
          }
        }
      }
    }
  }
  /* P2M of vertex patches: the exact moments of lambda_j M_j over every tet around node j */
  if (t->patches) {
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
    for (int64_t c = 0; c < ncell; c++) {
      if (!is_leaf(t, c) || t->ne[c] == t->nb[c]) continue;
      double* q = malloc(sizeof(double) * nc);
      for (int b = 0; b < B; b++) {
        double* Qc = Q + ((size_t)b * ncell + c) * nc;
        for (int64_t i = t->nb[c]; i < t->ne[c]; i++) {
          const int64_t g = t->node_perm[i];
          for (int64_t e = t->nt_off[g]; e < t->nt_off[g + 1]; e++) {
            double v[12], Mt[12];
            gather_tet(t, t->nt_tet[e], M, b, v, Mt);
            for (int k = 0; k < 4; k++)
              if (t->tets_c[4 * t->nt_tet[e] + k] != g) Mt[3 * k] = Mt[3 * k + 1] = Mt[3 * k + 2] = 0;
            tet_moments_tab(&T, &G, v, Mt, t->centre + 3 * c, q);
            for (int m = 0; m < nc; m++) Qc[m] += q[m];
          }
        }
      }
      free(q);
    }
  }
  /* P2M: leaves holding tets */
#pragma omp parallel for schedule(dynamic, 8) num_threads(nt)
  for (int64_t c = 0; c < ncell; c++) {
    if (t->dipoles || t->patches || !is_leaf(t, c) || t->te[c] == t->tb[c]) continue;
    double* q = malloc(sizeof(double) * nc);
    for (int b = 0; b < B; b++) {
      double* Qc = Q + ((size_t)b * ncell + c) * nc;
      for (int64_t j = t->tb[c]; j < t->te[c]; j++) {
        double v[12], Mt[12];
        gather_tet(t, t->tet_perm[j], M, b, v, Mt);
        tet_moments_tab(&T, &G, v, Mt, t->centre + 3 * c, q);
        for (int i = 0; i < nc; i++) Qc[i] += q[i];
      }
    }
    free(q);
  }
  /* M2M: children have larger indices than their parent */
  for (int64_t c = ncell - 1; c >= 0; c--) {
    if (is_leaf(t, c)) continue;
    for (int b = 0; b < B; b++)
      for (int64_t k = t->child0[c]; k < t->child0[c] + t->nchild[c]; k++) {
        double d[3] = {t->centre[3 * k] - t->centre[3 * c], t->centre[3 * k + 1] - t->centre[3 * c + 1],
                       t->centre[3 * k + 2] - t->centre[3 * c + 2]};
        m2m_tab(&T, d, Q + ((size_t)b * ncell + k) * nc, Q + ((size_t)b * ncell + c) * nc);
      }
  }
  /* M2L */
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t c = 0; c < ncell; c++) {
    if (!mark[c]) continue;
    double* D = malloc(sizeof(double) * nc);
    for (int64_t e = t->m2l_off[c]; e < t->m2l_off[c + 1]; e++) {
      int64_t s = t->m2l_src[e];
      double R[3] = {t->centre[3 * c] - t->centre[3 * s], t->centre[3 * c + 1] - t->centre[3 * s + 1],
                     t->centre[3 * c + 2] - t->centre[3 * s + 2]};
      for (int b = 0; b < B; b++)
        m2l_tab(&T, R, Q + ((size_t)b * ncell + s) * nc, L + ((size_t)b * ncell + c) * nc, D);
    }
    free(D);
  }
  /* L2L: parents before children */
  for (int64_t c = 0; c < ncell; c++) {
    if (is_leaf(t, c) || !mark[c]) continue;
    for (int64_t k = t->child0[c]; k < t->child0[c] + t->nchild[c]; k++) {
      if (!mark[k]) continue;
      double d[3] = {t->centre[3 * k] - t->centre[3 * c], t->centre[3 * k + 1] - t->centre[3 * c + 1],
                     t->centre[3 * k + 2] - t->centre[3 * c + 2]};
      for (int b = 0; b < B; b++)
        l2l_tab(&T, d, L + ((size_t)b * ncell + c) * nc, L + ((size_t)b * ncell + k) * nc);
    }
  }
  /* L2P + P2P per target leaf */
#pragma omp parallel for schedule(dynamic, 2) num_threads(nt)
  for (int64_t li = 0; li < nleaves; li++) {
    int64_t c = leaves[li];
    for (int64_t i = t->nb[c]; i < t->ne[c]; i++) {
      int64_t node = t->node_perm[i];
      const double* r = t->nodes_c + 3 * node;
      double z[3] = {r[0] - t->centre[3 * c], r[1] - t->centre[3 * c + 1], r[2] - t->centre[3 * c + 2]};
      for (int b = 0; b < B; b++) {
        double uf = l2p_tab(&T, z, L + ((size_t)b * ncell + c) * nc);
        double un = 0;
        for (int64_t e = t->p2p_off[c]; e < t->p2p_off[c + 1]; e++) {
          int64_t s = t->p2p_src[e];
          if (t->dipoles) { /* V_j M_j . (r - r_j) / |r - r_j|^3, no self term */
            for (int64_t jj = t->nb[s]; jj < t->ne[s]; jj++) {
              const int64_t j = t->node_perm[jj];
              if (j == node) continue;
              const double* rj = t->nodes_c + 3 * j;
              const double* mj = M + ((int64_t)b * t->nn + j) * 3;
              const double d0 = r[0] - rj[0], d1 = r[1] - rj[1], d2 = r[2] - rj[2];
              const double R2 = d0 * d0 + d1 * d1 + d2 * d2;
              un += t->node_vol[j] * (mj[0] * d0 + mj[1] * d1 + mj[2] * d2) / (R2 * sqrt(R2));
            }
            continue;
          }
          if (t->patches) { /* lambda_j M_j over the tets around each source node j */
            for (int64_t jj = t->nb[s]; jj < t->ne[s]; jj++) {
              const int64_t j = t->node_perm[jj];
              for (int64_t e = t->nt_off[j]; e < t->nt_off[j + 1]; e++) {
                double v[12], Mt[12];
                gather_tet(t, t->nt_tet[e], M, b, v, Mt);
                for (int k = 0; k < 4; k++)
                  if (t->tets_c[4 * t->nt_tet[e] + k] != j) Mt[3 * k] = Mt[3 * k + 1] = Mt[3 * k + 2] = 0;
                un += oracle_tet_potential(r, v, Mt);
              }
            }
            continue;
          }
          for (int64_t j = t->tb[s]; j < t->te[s]; j++) {
            double v[12], Mt[12];
            gather_tet(t, t->tet_perm[j], M, b, v, Mt);
            un += oracle_tet_potential(r, v, Mt);
          }
        }
        u[(int64_t)b * t->nn + node] = uf + un / FOUR_PI;
      }
    }
  }
  free(Q);
  free(L);
  free(mark);
  free(leaves);
  mi_free(&T);
  return 0;
}
