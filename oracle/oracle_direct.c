/*
 * oracle_direct.c -- single-tet integrals, the direct sum and mass-lumped H.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain FP64, written for a reader
 * checking it against the paper, not for speed.
 *
 * Closed form used here (deliberately NOT the paper's target-apex
 * decomposition of Sec. 2.1, so that the CUDA path, which follows Sec. 2.1,
 * is checked against an independent derivation).  Integration by parts of the
 * integrand of Eq. (2) over one tet Omega with affine M:
 *     int_Omega M.grad'(1/R) dV' = sum_F int_F sigma_F / R dA' + rho int_Omega 1/R dV',
 * with sigma_F = M.n_F (n_F the outward unit normal, affine on F),
 * rho = -div M (constant) and R = |r - r'|.  The volume term is reduced to
 * faces with div'((r'-r)/R) = 2/R:
 *     int_Omega 1/R dV' = 1/2 sum_F d_F int_F 1/R dA',  d_F = (r'-r).n_F on F.
 * The face integrals of a constant and of an affine density over a flat
 * triangle are the classical closed forms (Wilton et al., IEEE TAP 32, 1984):
 *     int_F 1/R dA     = sum_e P0_e ln((R+_e + l+_e)/(R-_e + l-_e)) - |h| sum_e beta_e
 *     int_F (q-rho0)/R dA = 1/2 sum_e m_e [ l+ R+ - l- R- + R0_e^2 ln(...) ]
 * with rho0 the projection of r on the plane, h the height of r above it,
 * m_e the outward in-plane edge normal, P0_e the signed distance of rho0 to
 * the edge line, l+-_e the edge-end coordinates along the edge, R+-_e the
 * distances of r to the edge ends, R0_e^2 = P0_e^2 + h^2 and
 * beta_e = atan(P0 l+/(R0^2+|h|R+)) - atan(P0 l-/(R0^2+|h|R-)).
 * Degenerate targets (on an edge line, in a face plane, at a vertex) take the
 * limits of these expressions: terms multiplied by a vanishing P0, R0^2 or |h|
 * are dropped, with "vanishing" meaning <= 1e-14 x the tet diameter.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FOUR_PI (4.0 * 3.14159265358979323846)

static inline void sub3(const double* a, const double* b, double* c) {
  c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}
static inline double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static inline void cross3(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double norm3(const double* a) { return sqrt(dot3(a, a)); }

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Affine (P1) magnetisation on a tet: M(r) = sum_k M_k lambda_k(r).
 * grad lambda_1 = (e2 x e3)/det, grad lambda_2 = (e3 x e1)/det,
 * grad lambda_3 = (e1 x e2)/det, grad lambda_0 = -(sum), e_i = v_i - v_0,
 * det = e1.(e2 x e3) = 6 x signed volume.
 * ------------------------------------------------------------------------- */
typedef struct {
  double g[4][3];  /* grad lambda_k */
  double det;      /* 6 x signed volume */
  double diam;     /* longest edge */
} tet_affine;

static void tet_affine_init(const double v[12], tet_affine* T) {
  double e1[3], e2[3], e3[3], c[3];
  sub3(v + 3, v, e1); sub3(v + 6, v, e2); sub3(v + 9, v, e3);
  cross3(e2, e3, c);
  T->det = dot3(e1, c);
  double inv = 1.0 / T->det;
  for (int i = 0; i < 3; i++) T->g[1][i] = c[i] * inv;
  cross3(e3, e1, c);
  for (int i = 0; i < 3; i++) T->g[2][i] = c[i] * inv;
  cross3(e1, e2, c);
  for (int i = 0; i < 3; i++) T->g[3][i] = c[i] * inv;
  for (int i = 0; i < 3; i++) T->g[0][i] = -(T->g[1][i] + T->g[2][i] + T->g[3][i]);
  double d = 0;
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      double e[3];
      sub3(v + 3 * b, v + 3 * a, e);
      double l = norm3(e);
      if (l > d) d = l;
    }
  T->diam = d;
}

/* lambda_k(r) for all k (extended affinely outside the tet). */
static void tet_lambda(const double v[12], const tet_affine* T, const double r[3], double lam[4]) {
  double d[3];
  sub3(r, v, d);
  lam[1] = dot3(T->g[1], d);
  lam[2] = dot3(T->g[2], d);
  lam[3] = dot3(T->g[3], d);
  lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

/* M(r) and J_ab = dM_a/dx_b of the affine field with nodal values M[4][3]. */
static void tet_field(const double v[12], const tet_affine* T, const double M[12], const double r[3],
                      double Mr[3], double J[9]) {
  double lam[4];
  tet_lambda(v, T, r, lam);
  for (int a = 0; a < 3; a++) {
    Mr[a] = 0;
    for (int k = 0; k < 4; k++) Mr[a] += lam[k] * M[3 * k + a];
    for (int b = 0; b < 3; b++) {
      double s = 0;
      for (int k = 0; k < 4; k++) s += M[3 * k + a] * T->g[k][b];
      J[3 * a + b] = s;
    }
  }
}

/* Face f of the tet is the face opposite vertex f; fills its three vertex
 * indices ordered counter-clockwise about the outward normal, and the unit
 * outward normal. */
static void tet_face(const double v[12], int f, int idx[3], double n[3]) {
  int j = 0;
  for (int k = 0; k < 4; k++)
    if (k != f) idx[j++] = k;
  double e1[3], e2[3], w[3];
  sub3(v + 3 * idx[1], v + 3 * idx[0], e1);
  sub3(v + 3 * idx[2], v + 3 * idx[0], e2);
  cross3(e1, e2, n);
  sub3(v + 3 * f, v + 3 * idx[0], w);
  if (dot3(n, w) > 0) { /* points towards the opposite vertex: flip */
    int t = idx[1]; idx[1] = idx[2]; idx[2] = t;
    n[0] = -n[0]; n[1] = -n[1]; n[2] = -n[2];
  }
  double l = norm3(n);
  n[0] /= l; n[1] /= l; n[2] /= l;
}

/* Closed-form face integrals of a constant and an affine density (Wilton
 * et al. 1984), for target r and triangle (a,b,c) CCW about unit normal n:
 *   *I = int_F 1/R dA,  K = int_F (q - rho0)/R dA,  *h = n.(r - a). */
static void face_charge_integrals(const double r[3], const double* const V[3], const double n[3],
                                  double tol, double* I, double K[3], double* h_out) {
  double ra[3];
  sub3(r, V[0], ra);
  double h = dot3(n, ra);
  double rho0[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
  double ah = fabs(h);
  double sum_log = 0, sum_beta = 0;
  K[0] = K[1] = K[2] = 0;
  for (int e = 0; e < 3; e++) {
    const double* s = V[e];
    const double* f = V[(e + 1) % 3];
    double tv[3], t[3], m[3], ds[3], df[3], rs[3], rf[3];
    sub3(f, s, tv);
    double L = norm3(tv);
    t[0] = tv[0] / L; t[1] = tv[1] / L; t[2] = tv[2] / L;
    cross3(t, n, m); /* outward in-plane normal of the edge */
    sub3(s, rho0, ds);
    sub3(f, rho0, df);
    double lm = dot3(ds, t), lp = dot3(df, t);
    double P0 = dot3(ds, m);
    sub3(s, r, rs);
    sub3(f, r, rf);
    double Rm = norm3(rs), Rp = norm3(rf);
    double R02 = P0 * P0 + h * h;
    double R0 = sqrt(R02);
    double Lam = 0;
    if (R0 > tol) Lam = asinh(lp / R0) - asinh(lm / R0); /* = ln((R+ + l+)/(R- + l-)) */
    sum_log += P0 * Lam;
    if (ah > tol && fabs(P0) > tol)
      sum_beta += atan(P0 * lp / (R02 + ah * Rp)) - atan(P0 * lm / (R02 + ah * Rm));
    double w = 0.5 * (lp * Rp - lm * Rm + R02 * Lam);
    K[0] += w * m[0]; K[1] += w * m[1]; K[2] += w * m[2];
  }
  *I = sum_log - ah * sum_beta;
  *h_out = h;
}

double oracle_tet_potential(const double r[3], const double v[12], const double M[12]) {
  tet_affine T;
  tet_affine_init(v, &T);
  double tol = 1e-14 * T.diam;
  double Mr[3], J[9];
  tet_field(v, &T, M, r, Mr, J);
  double rho = -(J[0] + J[4] + J[8]); /* -div M */
  double surf = 0, vol_int = 0;
  for (int f = 0; f < 4; f++) {
    int idx[3];
    double n[3];
    tet_face(v, f, idx, n);
    const double* V[3] = {v + 3 * idx[0], v + 3 * idx[1], v + 3 * idx[2]};
    double I, K[3], h;
    face_charge_integrals(r, V, n, tol, &I, K, &h);
    /* sigma = n.M is affine on the face: sigma(q) = sigma(rho0) + grad_s sigma.(q - rho0) */
    double Jn[3] = {J[0] * n[0] + J[1] * n[1] + J[2] * n[2], J[3] * n[0] + J[4] * n[1] + J[5] * n[2],
                    J[6] * n[0] + J[7] * n[1] + J[8] * n[2]};
    double sigma0 = dot3(n, Mr) - h * dot3(n, Jn); /* n.M(rho0), M(rho0) = M(r) - h J n */
    double JTn[3] = {J[0] * n[0] + J[3] * n[1] + J[6] * n[2], J[1] * n[0] + J[4] * n[1] + J[7] * n[2],
                     J[2] * n[0] + J[5] * n[1] + J[8] * n[2]};
    double nn = dot3(JTn, n);
    double gs[3] = {JTn[0] - nn * n[0], JTn[1] - nn * n[1], JTn[2] - nn * n[2]};
    surf += sigma0 * I + dot3(gs, K);
    vol_int += -0.5 * h * I; /* d_F = (r' - r).n = -h */
  }
  return surf + rho * vol_int;
}

/* ---------------------------------------------------------------------------
 * Gauss-Legendre nodes on [0,1] by Newton iteration on P_n (three-term
 * recurrence), weights 1/((1-z^2) P_n'(z)^2) after mapping from [-1,1].
 * ------------------------------------------------------------------------- */
static void gauss_legendre01(int n, double* x, double* w) {
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

/* ---------------------------------------------------------------------------
 * Cone route (Sec. 2.1, Fig. 2): the tet is the signed union of the four
 * cones joining r to its faces, the sign of face F being -sign(h_F) with
 * h_F = n_F.(r - a_F).  On the cone r' = r + t (q - r), q in F, t in [0,1],
 * dV = t^2 |h_F| dt dA_q and (r - r')/|r - r'|^3 = -(q - r)/(t^2 |q - r|^3):
 * the t^2 cancels (the regularising transform of Sec. 2.1) and, M being
 * affine, int_0^1 M(r + t(q-r)) dt = (M(r) + M(q))/2.  Hence
 *   int_tet M.(r-r')/R^3 dV = sum_F (h_F/2) int_F (M(r)+M(q)).(q-r)/|q-r|^3 dA_q,
 * and the face integrals are done numerically (adaptive collapsed Gauss).
 * ------------------------------------------------------------------------- */
typedef struct {
  double r[3], Mr2[3], J[9];
  double x[8], w[8];
  int n;
} cone_ctx;

static void cone_integrand(const cone_ctx* c, const double q[3], double* f, double* af) {
  double d[3];
  sub3(q, c->r, d);
  double R2 = dot3(d, d);
  double R = sqrt(R2);
  double Mq[3]; /* M(r) + M(q) = 2 M(r) + J (q - r) */
  for (int a = 0; a < 3; a++) Mq[a] = c->Mr2[a] + c->J[3 * a] * d[0] + c->J[3 * a + 1] * d[1] + c->J[3 * a + 2] * d[2];
  double v = dot3(Mq, d) / (R2 * R);
  *f = v;
  *af = fabs(v);
}

static void cone_tri_rule(const cone_ctx* c, const double* A, const double* B, const double* C, double* I,
                          double* aI) {
  double e1[3], e2[3], cr[3];
  sub3(B, A, e1);
  sub3(C, A, e2);
  cross3(e1, e2, cr);
  double jac = norm3(cr); /* 2 x area */
  double s = 0, as = 0;
  for (int i = 0; i < c->n; i++)
    for (int j = 0; j < c->n; j++) {
      double u = c->x[i], vv = c->x[j] * (1.0 - u);
      double q[3] = {A[0] + u * e1[0] + vv * e2[0], A[1] + u * e1[1] + vv * e2[1], A[2] + u * e1[2] + vv * e2[2]};
      double f, af;
      cone_integrand(c, q, &f, &af);
      double wt = c->w[i] * c->w[j] * (1.0 - u);
      s += wt * f;
      as += wt * af;
    }
  *I = s * jac;
  *aI = as * jac;
}

/* Global adaptive refinement: keep a max-heap of triangles keyed by the
 * estimated error |sum(children) - own rule|, split the worst one until the
 * summed estimate is below tol or a fixed budget of triangles is spent. */
typedef struct {
  double v[9];
  double Ic[4], err;
} cone_tri;

static void cone_tri_make(const cone_ctx* c, const double* A, const double* B, const double* C, double I, cone_tri* t) {
  for (int i = 0; i < 3; i++) {
    t->v[i] = A[i];
    t->v[3 + i] = B[i];
    t->v[6 + i] = C[i];
  }
  double ab[3], bc[3], ca[3];
  for (int i = 0; i < 3; i++) {
    ab[i] = 0.5 * (A[i] + B[i]);
    bc[i] = 0.5 * (B[i] + C[i]);
    ca[i] = 0.5 * (C[i] + A[i]);
  }
  const double* tris[4][3] = {{A, ab, ca}, {ab, B, bc}, {ca, bc, C}, {ab, bc, ca}};
  double s = 0, a;
  for (int k = 0; k < 4; k++) {
    cone_tri_rule(c, tris[k][0], tris[k][1], tris[k][2], &t->Ic[k], &a);
    s += t->Ic[k];
  }
  t->err = fabs(s - I);
}

static void heap_up(cone_tri* h, int i) {
  while (i > 0) {
    int p = (i - 1) / 2;
    if (h[p].err >= h[i].err) break;
    cone_tri tmp = h[p]; h[p] = h[i]; h[i] = tmp;
    i = p;
  }
}
static void heap_down(cone_tri* h, int n, int i) {
  for (;;) {
    int l = 2 * i + 1, r = l + 1, m = i;
    if (l < n && h[l].err > h[m].err) m = l;
    if (r < n && h[r].err > h[m].err) m = r;
    if (m == i) break;
    cone_tri tmp = h[m]; h[m] = h[i]; h[i] = tmp;
    i = m;
  }
}

static double cone_face_integral(const cone_ctx* c, const double* A, const double* B, const double* C, double rel_tol) {
  const int cap = 20000;
  cone_tri* h = malloc(sizeof(cone_tri) * cap);
  double I0, aI0;
  cone_tri_rule(c, A, B, C, &I0, &aI0);
  int n = 0;
  cone_tri_make(c, A, B, C, I0, &h[n++]);
  double tol = rel_tol * aI0;
  for (;;) {
    double err = 0;
    for (int i = 0; i < n; i++) err += h[i].err;
    if (err <= tol || n + 3 > cap) break;
    cone_tri w = h[0];
    h[0] = h[--n];
    heap_down(h, n, 0);
    double *A1 = w.v, *B1 = w.v + 3, *C1 = w.v + 6, ab[3], bc[3], ca[3];
    for (int i = 0; i < 3; i++) {
      ab[i] = 0.5 * (A1[i] + B1[i]);
      bc[i] = 0.5 * (B1[i] + C1[i]);
      ca[i] = 0.5 * (C1[i] + A1[i]);
    }
    const double* tris[4][3] = {{A1, ab, ca}, {ab, B1, bc}, {ca, bc, C1}, {ab, bc, ca}};
    for (int k = 0; k < 4; k++) {
      cone_tri_make(c, tris[k][0], tris[k][1], tris[k][2], w.Ic[k], &h[n]);
      heap_up(h, n);
      n++;
    }
  }
  double s = 0;
  for (int i = 0; i < n; i++) s += h[i].Ic[0] + h[i].Ic[1] + h[i].Ic[2] + h[i].Ic[3];
  free(h);
  return s;
}

double oracle_tet_potential_cone_quad(const double r[3], const double v[12], const double M[12], double rel_tol) {
  tet_affine T;
  tet_affine_init(v, &T);
  cone_ctx c;
  c.n = 8;
  gauss_legendre01(c.n, c.x, c.w);
  double Mr[3];
  tet_field(v, &T, M, r, Mr, c.J);
  for (int a = 0; a < 3; a++) {
    c.r[a] = r[a];
    c.Mr2[a] = 2.0 * Mr[a];
  }
  double tol_h = 1e-14 * T.diam;
  double total = 0;
  for (int f = 0; f < 4; f++) {
    int idx[3];
    double n[3], ra[3];
    tet_face(v, f, idx, n);
    sub3(r, v + 3 * idx[0], ra);
    double h = dot3(n, ra);
    if (fabs(h) <= tol_h) continue; /* the factor h_F vanishes */
    const double *A = v + 3 * idx[0], *B = v + 3 * idx[1], *C = v + 3 * idx[2];
    total += 0.5 * h * cone_face_integral(&c, A, B, C, rel_tol);
  }
  return total;
}

/* Collapsed-cube product rule on the tet: r' = v0 + x e1 + y e2 + z e3 with
 * (x,y,z) = (u, v(1-u), w(1-u)(1-v)), dV = |det| (1-u)^2 (1-v) du dv dw. */
double oracle_tet_potential_gauss3d(const double r[3], const double v[12], const double M[12], int q) {
  tet_affine T;
  tet_affine_init(v, &T);
  double *x = malloc(sizeof(double) * q), *w = malloc(sizeof(double) * q);
  gauss_legendre01(q, x, w);
  double e1[3], e2[3], e3[3];
  sub3(v + 3, v, e1); sub3(v + 6, v, e2); sub3(v + 9, v, e3);
  double s = 0;
  for (int i = 0; i < q; i++)
    for (int j = 0; j < q; j++)
      for (int k = 0; k < q; k++) {
        double u = x[i], vv = x[j] * (1 - u), ww = x[k] * (1 - u) * (1 - x[j]);
        double rp[3], Mr[3], J[9], d[3];
        for (int a = 0; a < 3; a++) rp[a] = v[a] + u * e1[a] + vv * e2[a] + ww * e3[a];
        tet_field(v, &T, M, rp, Mr, J);
        sub3(r, rp, d);
        double R = norm3(d);
        double wt = w[i] * w[j] * w[k] * (1 - u) * (1 - u) * (1 - x[j]);
        s += wt * dot3(Mr, d) / (R * R * R);
      }
  free(x);
  free(w);
  return s * fabs(T.det);
}

/* ---------------------------------------------------------------------------
 * Direct sum, Eq. (2): u_i = 1/(4pi) sum_t int_t M.grad'(1/R).
 * ------------------------------------------------------------------------- */
int oracle_direct(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, const double* M,
                  int B, const int64_t* targets, int64_t n_targets, double* u, int nthreads) {
  if (!nodes || !tets || !M || !u || B < 1) return 1;
  if (!targets && n_targets != n_nodes) return 1;
#ifdef _OPENMP
  /* thread count of this call only (a num_threads clause, not a global setting) */
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t i = 0; i < n_targets; i++) {
    int64_t node = targets ? targets[i] : i;
    const double* r = nodes + 3 * node;
    for (int b = 0; b < B; b++) {
      double s = 0;
      for (int64_t t = 0; t < n_tets; t++) {
        double v[12], Mt[12];
        for (int k = 0; k < 4; k++) {
          int32_t g = tets[4 * t + k];
          for (int a = 0; a < 3; a++) {
            v[3 * k + a] = nodes[3 * (int64_t)g + a];
            Mt[3 * k + a] = M[((int64_t)b * n_nodes + g) * 3 + a];
          }
        }
        s += oracle_tet_potential(r, v, Mt);
      }
      u[(int64_t)b * n_targets + i] = s / FOUR_PI;
    }
  }
  return 0;
}

/* Whole-mesh charge route: for a continuous P1 magnetisation the surface
 * charges n.M of an interior face cancel between its two tets (opposite
 * normals, same M), so the potential is that of the boundary faces' affine
 * surface charges plus every tet's constant volume charge -div M:
 *   4 pi u(r) = sum_{boundary (t, f)} int_f n_f.M / R dA + sum_t rho_t int_t 1/R dV.
 * A route to the same number that never forms an interior face charge.  The
 * boundary faces are given as (tet, local face) pairs (face f opposite vertex f). */
int oracle_direct_charges(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                          const int32_t* bfaces, int64_t n_bfaces, const double* M, int B,
                          const int64_t* targets, int64_t n_targets, double* u, int nthreads) {
  if (!nodes || !tets || !M || !u || B < 1 || (n_bfaces && !bfaces)) return 1;
  if (!targets && n_targets != n_nodes) return 1;
#ifdef _OPENMP
  /* thread count of this call only (a num_threads clause, not a global setting) */
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t i = 0; i < n_targets; i++) {
    const int64_t node = targets ? targets[i] : i;
    const double* r = nodes + 3 * node;
    for (int b = 0; b < B; b++) {
      double s = 0;
      for (int64_t t = 0; t < n_tets; t++) {  /* volume charges */
        double v[12], Mt[12], Mr[3], J[9];
        for (int k = 0; k < 4; k++) {
          const int32_t g = tets[4 * t + k];
          for (int a = 0; a < 3; a++) {
            v[3 * k + a] = nodes[3 * (int64_t)g + a];
            Mt[3 * k + a] = M[((int64_t)b * n_nodes + g) * 3 + a];
          }
        }
        tet_affine T;
        tet_affine_init(v, &T);
        tet_field(v, &T, Mt, r, Mr, J);
        const double rho = -(J[0] + J[4] + J[8]);
        double vol_int = 0;
        for (int f = 0; f < 4; f++) {
          int idx[3];
          double n[3], I, K[3], h;
          tet_face(v, f, idx, n);
          const double* V[3] = {v + 3 * idx[0], v + 3 * idx[1], v + 3 * idx[2]};
          face_charge_integrals(r, V, n, 1e-14 * T.diam, &I, K, &h);
          vol_int += -0.5 * h * I;
        }
        s += rho * vol_int;
      }
      for (int64_t q = 0; q < n_bfaces; q++) {  /* boundary surface charges */
        const int64_t t = bfaces[2 * q];
        const int f = bfaces[2 * q + 1];
        double v[12], Mt[12], Mr[3], J[9];
        for (int k = 0; k < 4; k++) {
          const int32_t g = tets[4 * t + k];
          for (int a = 0; a < 3; a++) {
            v[3 * k + a] = nodes[3 * (int64_t)g + a];
            Mt[3 * k + a] = M[((int64_t)b * n_nodes + g) * 3 + a];
          }
        }
        tet_affine T;
        tet_affine_init(v, &T);
        tet_field(v, &T, Mt, r, Mr, J);
        int idx[3];
        double n[3], I, K[3], h;
        tet_face(v, f, idx, n);
        const double* V[3] = {v + 3 * idx[0], v + 3 * idx[1], v + 3 * idx[2]};
        face_charge_integrals(r, V, n, 1e-14 * T.diam, &I, K, &h);
        const double Jn[3] = {J[0] * n[0] + J[1] * n[1] + J[2] * n[2], J[3] * n[0] + J[4] * n[1] + J[5] * n[2],
                              J[6] * n[0] + J[7] * n[1] + J[8] * n[2]};
        const double sigma0 = dot3(n, Mr) - h * dot3(n, Jn);
        const double JTn[3] = {J[0] * n[0] + J[3] * n[1] + J[6] * n[2], J[1] * n[0] + J[4] * n[1] + J[7] * n[2],
                               J[2] * n[0] + J[5] * n[1] + J[8] * n[2]};
        const double nn = dot3(JTn, n);
        const double gs[3] = {JTn[0] - nn * n[0], JTn[1] - nn * n[1], JTn[2] - nn * n[2]};
        s += sigma0 * I + dot3(gs, K);
      }
      u[(int64_t)b * n_targets + i] = s / FOUR_PI;
    }
  }
  return 0;
}

/* ---------------------------------------------------------------------------
 * Pointwise field H = -grad u (the remark of Sec. 4.1-4.2 that computing H
 * directly gives lower errors), from the whole-mesh charge route above:
 *   4 pi H(r) = sum_{boundary faces F} int_F sigma(r') (r - r')/R^3 dA
 *             + sum_t rho_t int_t (r - r')/R^3 dV.
 * Volume term (divergence theorem, grad'(1/R) = (r - r')/R^3):
 *   int_t (r - r')/R^3 dV = sum_{F of t} n_F int_F 1/R dA.
 * Face term for an affine sigma(r') = sigma0 + g.(r' - rho0) on a plane
 * triangle F (rho0 the projection of r, h = n.(r - rho0), Omega = int_F h/R^3
 * the signed solid angle, and per edge e: outward in-plane normal m_e, unit
 * tangent t_e, signed distance P0_e of rho0 to its line, Lambda_e =
 * int_e 1/R dl, dR_e = R+ - R- the difference of the end distances):
 * with r - r' = h n - (r' - rho0), the in-plane Gauss theorem
 * int_F grad_s f dA = sum_e m_e int_e f dl applied to f = 1/R and to
 * (r' - rho0)_a / R gives
 *   int_F (r' - rho0)/R^3 dA = -sum_e m_e Lambda_e,
 *   int_F (r' - rho0)(r' - rho0)^T/R^3 dA . g = Phi g - sum_e (m_e.g)(P0_e Lambda_e m_e + dR_e t_e),
 * hence
 *   int_F sigma (r - r')/R^3 dA = sigma0 Omega n - h (sum_e (g.m_e) Lambda_e) n + sigma0 sum_e Lambda_e m_e
 *                                 - Phi g + sum_e (m_e.g)(P0_e Lambda_e m_e + dR_e t_e),
 * Phi = int_F 1/R dA.  The point must not lie on a boundary face (the face
 * term diverges there); on the line of an edge outside the edge Lambda_e is
 * the finite log of the end distances.
 * ------------------------------------------------------------------------- */
static double edge_log(double lm, double lp, double R0, double Rm, double Rp, double tol) {
  if (R0 > tol) return asinh(lp / R0) - asinh(lm / R0);
  if (lm > tol) return log(lp / lm);     /* the point on the edge's line, before it */
  if (lp < -tol) return log(lm / lp);    /* ... behind it */
  (void)Rm; (void)Rp;
  return NAN;                            /* on the edge itself */
}

static void face_field(const double r[3], const double* const V[3], const double n[3], double tol, double sigma0,
                       const double g[3], double E[3], double* Phi_out) {
  double ra[3];
  sub3(r, V[0], ra);
  const double h = dot3(n, ra), ah = fabs(h);
  const double rho0[3] = {r[0] - h * n[0], r[1] - h * n[1], r[2] - h * n[2]};
  double sum_log = 0, sum_beta = 0, gl = 0, A[3] = {0, 0, 0}, C[3] = {0, 0, 0};
  for (int e = 0; e < 3; e++) {
    const double* s = V[e];
    const double* f = V[(e + 1) % 3];
    double tv[3], t[3], m[3], ds[3], df[3], rs[3], rf[3];
    sub3(f, s, tv);
    const double L = norm3(tv);
    t[0] = tv[0] / L; t[1] = tv[1] / L; t[2] = tv[2] / L;
    cross3(t, n, m);
    sub3(s, rho0, ds);
    sub3(f, rho0, df);
    const double lm = dot3(ds, t), lp = dot3(df, t);
    const double P0 = dot3(ds, m);
    sub3(s, r, rs);
    sub3(f, r, rf);
    const double Rm = norm3(rs), Rp = norm3(rf);
    const double R02 = P0 * P0 + h * h, R0 = sqrt(R02);
    const double Lam = edge_log(lm, lp, R0, Rm, Rp, tol);
    if (fabs(P0) > tol) sum_log += P0 * Lam;
    if (ah > tol && fabs(P0) > tol)
      sum_beta += atan(P0 * lp / (R02 + ah * Rp)) - atan(P0 * lm / (R02 + ah * Rm));
    const double gm = dot3(g, m);
    gl += gm * Lam;
    for (int a = 0; a < 3; a++) {
      A[a] += Lam * m[a];
      C[a] += gm * ((fabs(P0) > tol ? P0 * Lam : 0.0) * m[a] + (Rp - Rm) * t[a]);
    }
  }
  const double Phi = sum_log - ah * sum_beta;
  const double Omega = h > 0 ? sum_beta : (h < 0 ? -sum_beta : 0.0);
  for (int a = 0; a < 3; a++) E[a] = sigma0 * Omega * n[a] - h * gl * n[a] + sigma0 * A[a] - Phi * g[a] + C[a];
  if (Phi_out) *Phi_out = Phi;
}

/* H (B x n_pts x 3) at the points pts (n_pts x 3), none of them on a boundary
 * face; boundary faces as (tet, local face) pairs. */
int oracle_field_charges(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                         const int32_t* bfaces, int64_t n_bfaces, const double* M, int B, const double* pts,
                         int64_t n_pts, double* H, int nthreads) {
  if (!nodes || !tets || !M || !H || !pts || B < 1 || (n_bfaces && !bfaces)) return 1;
#ifdef _OPENMP
  /* thread count of this call only (a num_threads clause, not a global setting) */
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
  (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 4) num_threads(nt)
  for (int64_t i = 0; i < n_pts; i++) {
    const double* r = pts + 3 * i;
    for (int b = 0; b < B; b++) {
      double Hs[3] = {0, 0, 0};
      for (int64_t t = 0; t < n_tets; t++) { /* volume charges: rho_t sum_F n_F Phi_F */
        double v[12], Mt[12], Mr[3], J[9];
        for (int k = 0; k < 4; k++) {
          const int32_t gi = tets[4 * t + k];
          for (int a = 0; a < 3; a++) {
            v[3 * k + a] = nodes[3 * (int64_t)gi + a];
            Mt[3 * k + a] = M[((int64_t)b * n_nodes + gi) * 3 + a];
          }
        }
        tet_affine T;
        tet_affine_init(v, &T);
        tet_field(v, &T, Mt, r, Mr, J);
        const double rho = -(J[0] + J[4] + J[8]);
        if (rho == 0.0) continue;
        for (int f = 0; f < 4; f++) {
          int idx[3];
          double n[3], I, K[3], h;
          tet_face(v, f, idx, n);
          const double* V[3] = {v + 3 * idx[0], v + 3 * idx[1], v + 3 * idx[2]};
          face_charge_integrals(r, V, n, 1e-14 * T.diam, &I, K, &h);
          for (int a = 0; a < 3; a++) Hs[a] += rho * n[a] * I;
        }
      }
      for (int64_t q = 0; q < n_bfaces; q++) { /* boundary surface charges */
        const int64_t t = bfaces[2 * q];
        const int f = bfaces[2 * q + 1];
        double v[12], Mt[12], Mr[3], J[9];
        for (int k = 0; k < 4; k++) {
          const int32_t gi = tets[4 * t + k];
          for (int a = 0; a < 3; a++) {
            v[3 * k + a] = nodes[3 * (int64_t)gi + a];
            Mt[3 * k + a] = M[((int64_t)b * n_nodes + gi) * 3 + a];
          }
        }
        tet_affine T;
        tet_affine_init(v, &T);
        tet_field(v, &T, Mt, r, Mr, J);
        int idx[3];
        double n[3], E[3];
        tet_face(v, f, idx, n);
        const double* V[3] = {v + 3 * idx[0], v + 3 * idx[1], v + 3 * idx[2]};
        double ra[3];
        sub3(r, V[0], ra);
        const double h = dot3(n, ra);
        const double Jn[3] = {J[0] * n[0] + J[1] * n[1] + J[2] * n[2], J[3] * n[0] + J[4] * n[1] + J[5] * n[2],
                              J[6] * n[0] + J[7] * n[1] + J[8] * n[2]};
        const double sigma0 = dot3(n, Mr) - h * dot3(n, Jn); /* n.M(rho0) */
        const double JTn[3] = {J[0] * n[0] + J[3] * n[1] + J[6] * n[2], J[1] * n[0] + J[4] * n[1] + J[7] * n[2],
                               J[2] * n[0] + J[5] * n[1] + J[8] * n[2]};
        const double nn = dot3(JTn, n);
        const double gs[3] = {JTn[0] - nn * n[0], JTn[1] - nn * n[1], JTn[2] - nn * n[2]};
        face_field(r, V, n, 1e-14 * T.diam, sigma0, gs, E, NULL);
        for (int a = 0; a < 3; a++) Hs[a] += E[a];
      }
      for (int a = 0; a < 3; a++) H[((int64_t)b * n_pts + i) * 3 + a] = Hs[a] / FOUR_PI;
    }
  }
  return 0;
}

void oracle_tet_volumes(const double* nodes, const int32_t* tets, int64_t n_tets, double* vol) {
  for (int64_t t = 0; t < n_tets; t++) {
    double v[12];
    for (int k = 0; k < 4; k++)
      for (int a = 0; a < 3; a++) v[3 * k + a] = nodes[3 * (int64_t)tets[4 * t + k] + a];
    tet_affine T;
    tet_affine_init(v, &T);
    vol[t] = T.det / 6.0;
  }
}

/* Mass lumping (Sec. 4.1): the lumped mass of node i is sum_{t ni i} |t|/4 and
 * the lumped gradient is the volume-weighted mean of the constant P1 gradients
 * of the tets around i; H = -(that).  Nodes in no tet get H = 0. */
int oracle_lumped_H(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, const double* u,
                    int B, double* H) {
  double* num = calloc((size_t)n_nodes * 3 * B, sizeof(double));
  double* den = calloc((size_t)n_nodes, sizeof(double));
  if (!num || !den) {
    free(num);
    free(den);
    return 2;
  }
  for (int64_t t = 0; t < n_tets; t++) {
    double v[12];
    int32_t g[4];
    for (int k = 0; k < 4; k++) {
      g[k] = tets[4 * t + k];
      for (int a = 0; a < 3; a++) v[3 * k + a] = nodes[3 * (int64_t)g[k] + a];
    }
    tet_affine T;
    tet_affine_init(v, &T);
    double vol = fabs(T.det) / 6.0;
    for (int k = 0; k < 4; k++) den[g[k]] += vol;
    for (int b = 0; b < B; b++) {
      double gu[3] = {0, 0, 0};
      for (int k = 0; k < 4; k++) {
        double uk = u[(int64_t)b * n_nodes + g[k]];
        for (int a = 0; a < 3; a++) gu[a] += uk * T.g[k][a];
      }
      for (int k = 0; k < 4; k++)
        for (int a = 0; a < 3; a++) num[((int64_t)b * n_nodes + g[k]) * 3 + a] += vol * gu[a];
    }
  }
  for (int b = 0; b < B; b++)
    for (int64_t i = 0; i < n_nodes; i++)
      for (int a = 0; a < 3; a++) {
        int64_t o = ((int64_t)b * n_nodes + i) * 3 + a;
        H[o] = den[i] > 0 ? -num[o] / den[i] : 0.0;
      }
  free(num);
  free(den);
  return 0;
}
