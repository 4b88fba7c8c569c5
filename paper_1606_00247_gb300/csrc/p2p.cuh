// p2p.cuh -- analytic near-field integral of one P1-magnetised tet at one
// target point (Palmesi et al., Sec. 2.1 and Appendix A), device code.
//
// Derivation followed here (the paper's target-apex route, re-derived because
// its printed coefficients are garbled):
//  * Sec. 2.1, Fig. 2: the tet is the signed union of the four cones joining
//    the target r to its faces F; the cone of F enters with sign -sign(h_F),
//    h_F = n_F.(r - a_F) the height of r above the plane of F (outward n_F).
//  * On the cone r' = r + t(q - r), q in F, dV = t^2 |h_F| dt dA_q and the
//    kernel (r - r')/|r - r'|^3 = -(q - r)/(t^2 |q - r|^3): the singular t^2
//    cancels (the regularising transform of Sec. 2.1) and, M being affine,
//    the t-integral of M is (M(r) + M(q))/2.  Hence, with lambda_k the
//    barycentric coordinates and g_k = grad lambda_k,
//        W_k = int_tet lambda_k (r - r')/|r - r'|^3 dV
//            = sum_F (h_F/2) [ 2 lambda_k(r) A_F + T_F g_k ],
//        A_F = int_F (q - r)/|q - r|^3 dA,  T_F = int_F (q-r)(q-r)^T/|q-r|^3 dA.
//  * Triangle integrals (the tri_potential integrals of Sec. 2.1 / App. A),
//    reduced to the edges by the divergence theorem in the plane
//    (p = q - rho0 the in-plane offset from the foot rho0 of r):
//        A_F = -sum_e m_e Lam_e + n_F Omega_F
//        T_F = -sum_e [P0_e Lam_e m_e m_e^T + (R_end - R_start) t_e m_e^T]
//              + (I - n n^T) I_F - h_F (P_F n^T + n P_F^T) - h_F Omega_F n n^T
//        I_F = int_F dA/|q - r| = sum_e P0_e Lam_e + h_F Omega_F,  P_F = -sum_e m_e Lam_e
//    with m_e / t_e the outward normal / tangent of edge e in the plane,
//    P0_e = m_e.(start_e - r), Lam_e = int_e dl/|q - r|
//          = ln((R_a + R_b + L_e)/(R_a + R_b - L_e)),
//    and Omega_F the signed solid angle of F seen from r (Van Oosterom and
//    Strackee, IEEE TBME 30, 1983).
//  * Contracted with the nodal M:  sum_k M_k . W_k = M(r).a + (1/2) T : J,
//    a = sum_F h_F A_F, T = sum_F h_F T_F, J = dM/dx.  The J-contractions that
//    do not depend on r are precomputed per tet and state (alpha, beta, mu,
//    gamma, eps below).
// Faces whose plane contains r (|h_F| <= 1e-13 x longest edge) contribute
// exactly 0 (factor h_F), which also covers targets at vertices and on edges.
#pragma once
#include "common.cuh"

namespace demag {

// face F is opposite vertex F; vertex order counter-clockwise about the
// outward normal of a positively oriented tet
__host__ __device__ constexpr int face_vertex(int F, int i) {
  return F == 0 ? (i == 0 ? 1 : i == 1 ? 2 : 3)
       : F == 1 ? (i == 0 ? 0 : i == 1 ? 3 : 2)
       : F == 2 ? (i == 0 ? 0 : i == 1 ? 1 : 3)
                : (i == 0 ? 0 : i == 1 ? 2 : 1);
}
// edge id of the vertex pair {a,b}: (0,1)0 (0,2)1 (0,3)2 (1,2)3 (1,3)4 (2,3)5
__host__ __device__ constexpr int edge_id(int a, int b) {
  return (a > b) ? edge_id(b, a) : (a == 0 ? b - 1 : (a == 1 ? b + 1 : 5));
}
__host__ __device__ constexpr int edge_v0(int e) { return e < 3 ? 0 : (e < 5 ? 1 : 2); }
__host__ __device__ constexpr int edge_v1(int e) { return e < 3 ? e + 1 : (e < 5 ? e - 1 : 3); }

// W-form outputs of one (target, tet) pair: a (3) and the symmetric T (6:
// xx, yy, zz, xy, xz, yz), so that W_k = lambda_k(r) a + T g_k / 2.
struct PairAT {
  double a[3];
  double T[6];
};

// Contracted form: returns sum_k M_k . W_k for the state record `st`.
__device__ __forceinline__ double pair_contract(const double* __restrict__ geo, const double* __restrict__ st,
                                                double rx, double ry, double rz) {
  double a[4][3], R[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    a[k][0] = geo[3 * k] - rx;
    a[k][1] = geo[3 * k + 1] - ry;
    a[k][2] = geo[3 * k + 2] - rz;
    R[k] = sqrt(a[k][0] * a[k][0] + a[k][1] * a[k][1] + a[k][2] * a[k][2]);
  }
  double Lam[6], Lmax = 0;
#pragma unroll
  for (int e = 0; e < 6; e++) {
    double L = geo[60 + e];
    Lmax = fmax(Lmax, L);
    double S = R[edge_v0(e)] + R[edge_v1(e)];
    double D = S - L;
    Lam[e] = D > 0 ? log1p(2.0 * L / D) : 0.0;
  }
  const double tol = 1e-13 * Lmax;
  // M(r) = M(v0) + J (r - v0) = M(v0) - J a_0
  double Mr[3];
#pragma unroll
  for (int c = 0; c < 3; c++)
    Mr[c] = st[c] - (st[3 + 3 * c] * a[0][0] + st[4 + 3 * c] * a[0][1] + st[5 + 3 * c] * a[0][2]);
  double aM = 0, TJ = 0;
#pragma unroll
  for (int F = 0; F < 4; F++) {
    const int p = face_vertex(F, 0), q = face_vertex(F, 1), s = face_vertex(F, 2);
    const double* n = geo + 12 + 3 * F;
    double h = -(n[0] * a[p][0] + n[1] * a[p][1] + n[2] * a[p][2]);
    if (fabs(h) <= tol) continue;
    double cx = a[q][1] * a[s][2] - a[q][2] * a[s][1];
    double cy = a[q][2] * a[s][0] - a[q][0] * a[s][2];
    double cz = a[q][0] * a[s][1] - a[q][1] * a[s][0];
    double trip = a[p][0] * cx + a[p][1] * cy + a[p][2] * cz;
    double dpq = a[p][0] * a[q][0] + a[p][1] * a[q][1] + a[p][2] * a[q][2];
    double dps = a[p][0] * a[s][0] + a[p][1] * a[s][1] + a[p][2] * a[s][2];
    double dqs = a[q][0] * a[s][0] + a[q][1] * a[s][1] + a[q][2] * a[s][2];
    double den = R[p] * R[q] * R[s] + dpq * R[s] + dps * R[q] + dqs * R[p];
    double Om = 2.0 * atan2(trip, den);
    double I = h * Om, sLm = 0, Jp = 0, sLmu = 0;
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int v0 = face_vertex(F, e), v1 = face_vertex(F, (e + 1) % 3);
      const double* m = geo + 24 + 9 * F + 3 * e;
      double P0 = m[0] * a[v0][0] + m[1] * a[v0][1] + m[2] * a[v0][2];
      double lam = Lam[edge_id(v0, v1)];
      double dR = R[v1] - R[v0];
      I += P0 * lam;
      sLm += lam * (m[0] * Mr[0] + m[1] * Mr[1] + m[2] * Mr[2]);
      Jp += P0 * lam * st[12 + 3 * F + e] + dR * st[24 + 3 * F + e];
      sLmu += lam * st[36 + 3 * F + e];
    }
    double nM = n[0] * Mr[0] + n[1] * Mr[1] + n[2] * Mr[2];
    aM += h * (Om * nM - sLm);
    TJ += h * (I * st[48 + F] - Jp + 2.0 * h * sLmu - h * Om * st[52 + F]);
  }
  return aM + 0.5 * TJ;
}

// W-form: a and T of the pair (for the precomputed near-field coefficients).
__device__ __forceinline__ void pair_at(const double* __restrict__ geo, double rx, double ry, double rz, PairAT& o) {
  double a[4][3], R[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    a[k][0] = geo[3 * k] - rx;
    a[k][1] = geo[3 * k + 1] - ry;
    a[k][2] = geo[3 * k + 2] - rz;
    R[k] = sqrt(a[k][0] * a[k][0] + a[k][1] * a[k][1] + a[k][2] * a[k][2]);
  }
  double Lam[6], Lmax = 0;
#pragma unroll
  for (int e = 0; e < 6; e++) {
    double L = geo[60 + e];
    Lmax = fmax(Lmax, L);
    double S = R[edge_v0(e)] + R[edge_v1(e)];
    double D = S - L;
    Lam[e] = D > 0 ? log1p(2.0 * L / D) : 0.0;
  }
  const double tol = 1e-13 * Lmax;
  for (int i = 0; i < 3; i++) o.a[i] = 0;
  for (int i = 0; i < 6; i++) o.T[i] = 0;
#pragma unroll
  for (int F = 0; F < 4; F++) {
    const int p = face_vertex(F, 0), q = face_vertex(F, 1), s = face_vertex(F, 2);
    const double* n = geo + 12 + 3 * F;
    double h = -(n[0] * a[p][0] + n[1] * a[p][1] + n[2] * a[p][2]);
    if (fabs(h) <= tol) continue;
    double cx = a[q][1] * a[s][2] - a[q][2] * a[s][1];
    double cy = a[q][2] * a[s][0] - a[q][0] * a[s][2];
    double cz = a[q][0] * a[s][1] - a[q][1] * a[s][0];
    double trip = a[p][0] * cx + a[p][1] * cy + a[p][2] * cz;
    double dpq = a[p][0] * a[q][0] + a[p][1] * a[q][1] + a[p][2] * a[q][2];
    double dps = a[p][0] * a[s][0] + a[p][1] * a[s][1] + a[p][2] * a[s][2];
    double dqs = a[q][0] * a[s][0] + a[q][1] * a[s][1] + a[q][2] * a[s][2];
    double den = R[p] * R[q] * R[s] + dpq * R[s] + dps * R[q] + dqs * R[p];
    double Om = 2.0 * atan2(trip, den);
    double I = h * Om;
    double PF[3] = {0, 0, 0};
    double Te[6] = {0, 0, 0, 0, 0, 0};  // -sum_e [P0 Lam m m^T + dR sym(t m^T)]
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int v0 = face_vertex(F, e), v1 = face_vertex(F, (e + 1) % 3);
      const double* m = geo + 24 + 9 * F + 3 * e;
      double P0 = m[0] * a[v0][0] + m[1] * a[v0][1] + m[2] * a[v0][2];
      double lam = Lam[edge_id(v0, v1)];
      double dR = R[v1] - R[v0];
      // unit tangent t = n x m  (m = t x n, both unit and orthogonal)
      double t[3] = {n[1] * m[2] - n[2] * m[1], n[2] * m[0] - n[0] * m[2], n[0] * m[1] - n[1] * m[0]};
      I += P0 * lam;
      for (int c = 0; c < 3; c++) PF[c] -= m[c] * lam;
      double w = P0 * lam;
      Te[0] -= w * m[0] * m[0] + dR * t[0] * m[0];
      Te[1] -= w * m[1] * m[1] + dR * t[1] * m[1];
      Te[2] -= w * m[2] * m[2] + dR * t[2] * m[2];
      Te[3] -= w * m[0] * m[1] + 0.5 * dR * (t[0] * m[1] + t[1] * m[0]);
      Te[4] -= w * m[0] * m[2] + 0.5 * dR * (t[0] * m[2] + t[2] * m[0]);
      Te[5] -= w * m[1] * m[2] + 0.5 * dR * (t[1] * m[2] + t[2] * m[1]);
    }
    for (int c = 0; c < 3; c++) o.a[c] += h * (PF[c] + n[c] * Om);
    // (I - n n^T) I_F - h (P n^T + n P^T) - h Om n n^T
    const int ia[6] = {0, 1, 2, 0, 0, 1}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int k = 0; k < 6; k++) {
      int x = ia[k], y = ib[k];
      double v = Te[k] + ((x == y) ? I : 0.0) - n[x] * n[y] * I - h * (PF[x] * n[y] + n[x] * PF[y]) -
                 h * Om * n[x] * n[y];
      o.T[k] += h * v;
    }
  }
}

}  // namespace demag
