// field.cu -- pointwise field H = -grad u at the interior nodes (the remark of
// Sec. 4.1-4.2 that computing H directly, instead of from the potential by mass
// lumping, gives lower errors).
//
//   far field:  -grad u_far(r) = -sum_{|m| <= p-1} L_{m+e_a} z^m / m!   (L2P of the gradient)
//   near field: the field of the charges of every near tet t, in closed form,
//     4 pi H_t(r) = sum_{faces F of t} int_F sigma (r - r')/R^3 dA + rho_t sum_F n_F Phi_F(r),
//     sigma = n_F . M affine on F, rho_t = -div M, Phi_F = int_F dA / R;
//     the face term, with sigma(r') = sigma0 + g.(r' - rho0) (rho0 the foot of
//     r on the plane, h = n.(r - rho0), Omega = int_F h/R^3 dA), reduces by the
//     divergence theorem in the plane to
//       sigma0 Omega n - h (sum_e (g.m_e) Lam_e) n + sigma0 sum_e Lam_e m_e - Phi g
//       + sum_e (m_e.g)(P0_e Lam_e m_e + dR_e t_e)
//     (edge normals m_e, tangents t_e, P0_e the signed distance of rho0 to the
//     edge line, Lam_e = int_e dl/R, dR_e = R_end - R_start).
// At an interior node every face that contains the node is shared by two tets
// whose charges n.M cancel (M continuous, normals opposite), and both tets are
// in the node's near field (a tet touching the node cannot pass the MAC), so
// those face terms are left out on both sides -- each is log-singular at the
// node, their sum is zero.  At boundary nodes the pointwise field has these
// singularities; they keep the mass-lumped H.
#include <algorithm>
#include <array>
#include <vector>

#include "common.cuh"
#include "p2p.cuh"

namespace demag {

namespace {

inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// -grad u_far at every interior node, sorted layout Hs[node][3][B]
__global__ void k_l2p_grad(int64_t nn, const int32_t* __restrict__ node_leaf, const double* __restrict__ nodes_s,
                           const double* __restrict__ centre, const uint8_t* __restrict__ boundary, int p, int nc, int B,
                           const double* __restrict__ L, double* Hs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn || boundary[i]) return;
  const int32_t c = node_leaf[i];
  double px[MAX_P + 1], py[MAX_P + 1], pz[MAX_P + 1];
  const double zx = nodes_s[3 * i] - centre[3 * c], zy = nodes_s[3 * i + 1] - centre[3 * c + 1],
               zz = nodes_s[3 * i + 2] - centre[3 * c + 2];
  px[0] = py[0] = pz[0] = 1.0;
  for (int e = 1; e <= p; e++) {
    px[e] = px[e - 1] * zx / e;
    py[e] = py[e - 1] * zy / e;
    pz[e] = pz[e - 1] * zz / e;
  }
  const double* Lc = L + (int64_t)c * nc * B;
  for (int b = 0; b < B; b++) {
    double g[3] = {0, 0, 0};
    for (int t = 0; t < p; t++)  // |m| <= p - 1
      for (int j = 0; j <= t; j++)
        for (int mz = 0; mz <= j; mz++) {
          const int mx = t - j, my = j - mz;
          const double mono = px[mx] * py[my] * pz[mz];
          g[0] += Lc[(int64_t)mi_index(mx + 1, my, mz) * B + b] * mono;
          g[1] += Lc[(int64_t)mi_index(mx, my + 1, mz) * B + b] * mono;
          g[2] += Lc[(int64_t)mi_index(mx, my, mz + 1) * B + b] * mono;
        }
    for (int a = 0; a < 3; a++) Hs[(i * 3 + a) * B + b] = -g[a];
  }
}

// field of one tet's charges at r for FS states (nodal M of the 4 vertices in
// Mk[s][k][3]), the faces that contain r (vertex kv of the tet) left out of
// the surface term; adds 4 pi H_t into acc
template <int FS>
__device__ __forceinline__ void tet_field(const double* __restrict__ geo, const double* __restrict__ grad,
                                         double rx, double ry, double rz, int kv, const double (&Mk)[FS][4][3],
                                         double (&acc)[FS][3]) {
  double a[4][3], R[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    a[k][0] = geo[3 * k] - rx;
    a[k][1] = geo[3 * k + 1] - ry;
    a[k][2] = geo[3 * k + 2] - rz;
    R[k] = sqrt(a[k][0] * a[k][0] + a[k][1] * a[k][1] + a[k][2] * a[k][2]);
  }
  double Lam[6];
#pragma unroll
  for (int e = 0; e < 6; e++) {
    const double L = geo[60 + e], D = R[edge_v0(e)] + R[edge_v1(e)] - L;
    Lam[e] = D > 0 ? log1p(2.0 * L / D) : 0.0;
  }
  // per state: J = sum_k M_k (x) g_k, M(r), rho
  double J[FS][9], Mr[FS][3], rho[FS];
  double lam[4];
  {
    const double* g = grad;
    // lambda_k(r) = lambda_k(v0) + g_k.(r - v0), a[0] = v0 - r
    lam[1] = -(g[3] * a[0][0] + g[4] * a[0][1] + g[5] * a[0][2]);
    lam[2] = -(g[6] * a[0][0] + g[7] * a[0][1] + g[8] * a[0][2]);
    lam[3] = -(g[9] * a[0][0] + g[10] * a[0][1] + g[11] * a[0][2]);
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
  }
#pragma unroll
  for (int s = 0; s < FS; s++) {
#pragma unroll
    for (int x = 0; x < 3; x++) {
      Mr[s][x] = 0;
      for (int y = 0; y < 3; y++) J[s][3 * x + y] = 0;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        Mr[s][x] += lam[k] * Mk[s][k][x];
#pragma unroll
        for (int y = 0; y < 3; y++) J[s][3 * x + y] += Mk[s][k][x] * grad[3 * k + y];
      }
    }
    rho[s] = -(J[s][0] + J[s][4] + J[s][8]);
  }
#pragma unroll
  for (int F = 0; F < 4; F++) {
    const int p = face_vertex(F, 0), q = face_vertex(F, 1), sv = face_vertex(F, 2);
    const double* n = geo + 12 + 3 * F;
    const double h = -(n[0] * a[p][0] + n[1] * a[p][1] + n[2] * a[p][2]);
    const double cx = a[q][1] * a[sv][2] - a[q][2] * a[sv][1];
    const double cy = a[q][2] * a[sv][0] - a[q][0] * a[sv][2];
    const double cz = a[q][0] * a[sv][1] - a[q][1] * a[sv][0];
    const double trip = a[p][0] * cx + a[p][1] * cy + a[p][2] * cz;
    const double dpq = a[p][0] * a[q][0] + a[p][1] * a[q][1] + a[p][2] * a[q][2];
    const double dps = a[p][0] * a[sv][0] + a[p][1] * a[sv][1] + a[p][2] * a[sv][2];
    const double dqs = a[q][0] * a[sv][0] + a[q][1] * a[sv][1] + a[q][2] * a[sv][2];
    const double den = R[p] * R[q] * R[sv] + dpq * R[sv] + dps * R[q] + dqs * R[p];
    const double Om = -2.0 * atan2(trip, den);  // int_F h / R^3 dA (the opposite sign of p2p.cuh's Omega)
    double Phi = -h * Om;                       // int_F dA/R = sum_e P0_e Lam_e + h Omega_p2p
    double P0[3], L3[3], dR[3], m[3][3], t[3][3];
#pragma unroll
    for (int e = 0; e < 3; e++) {
      const int v0 = face_vertex(F, e), v1 = face_vertex(F, (e + 1) % 3);
      const double* me = geo + 24 + 9 * F + 3 * e;
      for (int x = 0; x < 3; x++) m[e][x] = me[x];
      t[e][0] = n[1] * me[2] - n[2] * me[1];
      t[e][1] = n[2] * me[0] - n[0] * me[2];
      t[e][2] = n[0] * me[1] - n[1] * me[0];
      P0[e] = me[0] * a[v0][0] + me[1] * a[v0][1] + me[2] * a[v0][2];
      L3[e] = Lam[edge_id(v0, v1)];
      dR[e] = R[v1] - R[v0];
      Phi += P0[e] * L3[e];
    }
    const bool surf = kv < 0 || kv == F;  // the faces through the target (kv != F) cancel with their neighbours
#pragma unroll
    for (int s = 0; s < FS; s++) {
      for (int x = 0; x < 3; x++) acc[s][x] += rho[s] * n[x] * Phi;  // volume charge
      if (!surf) continue;
      // sigma0 = n.M(rho0), M(rho0) = M(r) - h J n; g = (J^T n) projected on the plane
      const double* Js = J[s];
      const double Jn[3] = {Js[0] * n[0] + Js[1] * n[1] + Js[2] * n[2], Js[3] * n[0] + Js[4] * n[1] + Js[5] * n[2],
                            Js[6] * n[0] + Js[7] * n[1] + Js[8] * n[2]};
      const double sigma0 = n[0] * Mr[s][0] + n[1] * Mr[s][1] + n[2] * Mr[s][2] -
                            h * (n[0] * Jn[0] + n[1] * Jn[1] + n[2] * Jn[2]);
      double gv[3] = {Js[0] * n[0] + Js[3] * n[1] + Js[6] * n[2], Js[1] * n[0] + Js[4] * n[1] + Js[7] * n[2],
                      Js[2] * n[0] + Js[5] * n[1] + Js[8] * n[2]};
      const double gn = gv[0] * n[0] + gv[1] * n[1] + gv[2] * n[2];
      for (int x = 0; x < 3; x++) gv[x] -= gn * n[x];
      double gl = 0, E[3];
      for (int x = 0; x < 3; x++) E[x] = sigma0 * Om * n[x] - Phi * gv[x];
#pragma unroll
      for (int e = 0; e < 3; e++) {
        const double gm = gv[0] * m[e][0] + gv[1] * m[e][1] + gv[2] * m[e][2];
        gl += gm * L3[e];
        for (int x = 0; x < 3; x++) E[x] += sigma0 * L3[e] * m[e][x] + gm * (P0[e] * L3[e] * m[e][x] + dR[e] * t[e][x]);
      }
      for (int x = 0; x < 3; x++) acc[s][x] += E[x] - h * gl * n[x];
    }
  }
}

// near field of every interior node: one block per node, its leaf's P2P source
// tets over the threads, FS states per block (grid.y), fixed-order reduction
constexpr int FN_THREADS = 128, FN_FS = 2;
__global__ void __launch_bounds__(FN_THREADS) k_field_near(
    const int32_t* __restrict__ node_leaf, const int64_t* __restrict__ p2p_off, const int32_t* __restrict__ p2p_src,
    const int4* __restrict__ range, const double* __restrict__ nodes_s, const int32_t* __restrict__ tets_s,
    const double* __restrict__ geo, const double* __restrict__ grad, const uint8_t* __restrict__ boundary,
    const double* __restrict__ Ms, int B, double* Hs) {
  __shared__ double red[FN_THREADS][FN_FS][3];
  const int64_t i = blockIdx.x;
  if (boundary[i]) return;  // uniform over the block
  const int b0 = blockIdx.y * FN_FS;
  const int32_t T = node_leaf[i];
  const double rx = nodes_s[3 * i], ry = nodes_s[3 * i + 1], rz = nodes_s[3 * i + 2];
  double acc[FN_FS][3] = {};
  for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
    const int4 rS = range[p2p_src[e]];
    for (int32_t t = rS.x + threadIdx.x; t < rS.y; t += FN_THREADS) {
      double Mk[FN_FS][4][3];
      int kv = -1;
#pragma unroll
      for (int k = 0; k < 4; k++) {
        const int32_t node = tets_s[4ll * t + k];
        if (node == i) kv = k;
#pragma unroll
        for (int s = 0; s < FN_FS; s++)
#pragma unroll
          for (int c = 0; c < 3; c++) Mk[s][k][c] = b0 + s < B ? Ms[((int64_t)node * 3 + c) * B + b0 + s] : 0.0;
      }
      tet_field<FN_FS>(geo + (int64_t)t * TET_GEO, grad + 12ll * t, rx, ry, rz, kv, Mk, acc);
    }
  }
#pragma unroll
  for (int s = 0; s < FN_FS; s++)
    for (int c = 0; c < 3; c++) red[threadIdx.x][s][c] = acc[s][c];
  __syncthreads();
  if (threadIdx.x < FN_FS * 3) {
    const int s = threadIdx.x / 3, c = threadIdx.x % 3;
    double v = 0;
    for (int k = 0; k < FN_THREADS; k++) v += red[k][s][c];
    if (b0 + s < B) Hs[(i * 3 + c) * B + b0 + s] += v / (4.0 * M_PI);
  }
}

// interior nodes: the user layout H[b][node][c] from the sorted field
__global__ void k_field_out(int64_t nn, int B, const int32_t* __restrict__ perm, const uint8_t* __restrict__ boundary,
                            const double* __restrict__ Hs, double* H) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn || boundary[i]) return;
  const int64_t g = perm[i];
  for (int b = 0; b < B; b++)
    for (int c = 0; c < 3; c++) H[((int64_t)b * nn + g) * 3 + c] = Hs[(i * 3 + c) * B + b];
}

// sorted nodes on a boundary face (a face of exactly one tet), from the host copy of the sorted tets
std::vector<uint8_t> boundary_flags(int64_t nn, const std::vector<int32_t>& tets) {
  const int64_t nt = (int64_t)tets.size() / 4;
  std::vector<std::array<int32_t, 3>> faces;
  faces.reserve(4 * nt);
  for (int64_t t = 0; t < nt; t++)
    for (int f = 0; f < 4; f++) {
      std::array<int32_t, 3> v;
      int j = 0;
      for (int k = 0; k < 4; k++)
        if (k != f) v[j++] = tets[4 * t + k];
      std::sort(v.begin(), v.end());
      faces.push_back(v);
    }
  std::sort(faces.begin(), faces.end());
  std::vector<uint8_t> flag(nn, 0);
  for (size_t q = 0; q < faces.size();) {
    size_t r = q + 1;
    while (r < faces.size() && faces[r] == faces[q]) r++;
    if (r - q == 1)
      for (int32_t v : faces[q]) flag[v] = 1;
    q = r;
  }
  return flag;
}

}  // namespace

void eval_field(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s) {
  if (P.opt.precision != DEMAG_FP64 || P.opt.sources != DEMAG_SOURCES_TETS)
    fail(DEMAG_ERR_UNSUPPORTED, "the pointwise field is built for FP64 plans with tet sources");
  if (!is_device_ptr(M) || !is_device_ptr(u) || !is_device_ptr(H))
    fail(DEMAG_ERR_INVALID_ARG, "demag_eval_field takes device pointers");
  if (!P.tet_geo || !P.tet_grad) fail(DEMAG_ERR_UNSUPPORTED, "the plan holds no per-tet geometry");
  if (!P.bnd_flag) {  // first call: nodes on boundary faces
    std::vector<int32_t> ht(4 * P.nt);
    DM_CUDA(cudaMemcpy(ht.data(), P.tets_s, ht.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    const std::vector<uint8_t> f = boundary_flags(P.nn, ht);
    P.bnd_flag = dalloc<uint8_t>(P, P.nn);
    DM_CUDA(cudaMemcpy(P.bnd_flag, f.data(), P.nn, cudaMemcpyHostToDevice));
  }
  if (P.field_states < B) {
    if (P.field_buf) dfree(P, P.field_buf);
    P.field_buf = dalloc<double>(P, (size_t)P.nn * 3 * B);
    P.field_states = B;
  }
  Workspace& W = workspace(P, B);
  eval_fp64_ws(P, W, M, B, u, H, s, false);  // u, the mass-lumped H, and the local expansions in W.L
  k_l2p_grad<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, P.node_leaf, P.nodes_s, P.cell_centre, P.bnd_flag, P.p, P.nc, B,
                                             W.L, P.field_buf);
  DM_LAUNCH("k_l2p_grad");
  k_field_near<<<dim3((unsigned)P.nn, (unsigned)((B + FN_FS - 1) / FN_FS)), FN_THREADS, 0, s>>>(
      P.node_leaf, P.p2p_off, P.p2p_src, P.cell_range, P.nodes_s, P.tets_s, P.tet_geo, P.tet_grad, P.bnd_flag, W.Ms, B,
      P.field_buf);
  DM_LAUNCH("k_field_near");
  k_field_out<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, B, P.node_perm, P.bnd_flag, P.field_buf, H);
  DM_LAUNCH("k_field_out");
}

}  // namespace demag
