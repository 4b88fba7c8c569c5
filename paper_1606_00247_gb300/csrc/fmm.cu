// fmm.cu -- far field (Sec. 2 steps 1-5, Sec. 2.2-2.3), lumped H (Sec. 4.1)
// and the FP64 evaluation driver.
//
// Normalisation used on the device (equivalent to the paper's, cheaper):
//   Qhat_n = Q_n / n!              multipole moments, Q_n of Eq. (expCoeffs)
//   L_m    = d^m u (c_T)           local coefficients, Sec. 2.3
//   s_j(d) = d^j / j!              scaled monomials
//   b_k(x) = (-1)^|k| d^k (1/|x|)  (so that 1/|x - y| = sum_k b_k(x) y^k / k!)
// with which
//   P2M:  Qhat_n = sum_j sum_c Ghat_j[n - e_c] M_c(j)
//   M2M:  Qhat^P_n = sum_{k<=n} s_{n-k}(c_C - c_P) Qhat^C_k
//   M2L:  L_m = (-1)^|m| / (4 pi) sum_{|n|<=p-|m|} b_{n+m}(c_T - c_S) Qhat_n
//   L2L:  L^C_m = sum_{k>=m} s_{k-m}(c_C - c_P) L^P_k
//   L2P:  u(c + z) = sum_m s_m(z) L_m
// and b_k follows from the Taylor-coefficient recurrence of 1/|x|:
//   |k| r^2 b_k = (2|k|-1) sum_i k_i x_i b_{k-e_i} - (|k|-1) sum_i k_i (k_i-1) b_{k-2e_i}.
// All arrays keep the state index innermost: X[item][coef][state].
#include "common.cuh"

namespace demag {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

// multi-index table in shared memory
__device__ __forceinline__ void load_mi(int nc, unsigned char (*mi)[3]) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    int a, b, c;
    mi_decode(i, a, b, c);
    mi[i][0] = (unsigned char)a;
    mi[i][1] = (unsigned char)b;
    mi[i][2] = (unsigned char)c;
  }
}

// scaled monomials s_j(d) = d^j/j! for all |j| <= p into s[]
__device__ __forceinline__ void scaled_monomials(int p, int nc, const unsigned char (*mi)[3], double dx, double dy,
                                                 double dz, double* px, double* s) {
  // px: 3 x (p+1) scratch
  if (threadIdx.x == 0) {
    px[0] = px[p + 1] = px[2 * (p + 1)] = 1.0;
    for (int e = 1; e <= p; e++) {
      px[e] = px[e - 1] * dx / e;
      px[p + 1 + e] = px[p + e] * dy / e;
      px[2 * (p + 1) + e] = px[2 * (p + 1) + e - 1] * dz / e;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nc; j += blockDim.x) s[j] = px[mi[j][0]] * px[p + 1 + mi[j][1]] * px[2 * (p + 1) + mi[j][2]];
}

// ---------------------------------------------------------------------------
// input / output layout
// ---------------------------------------------------------------------------
// Ms[(i*3+c)*B + b] = M[(b*nn + perm[i])*3 + c]
// block per (sorted node, 128 states), thread = state: stores coalesce over states
__global__ void __launch_bounds__(128) k_gather_M(int64_t nn, int B, const int32_t* __restrict__ perm,
                                                  const double* __restrict__ M, double* Ms) {
  const int64_t i = blockIdx.x;
  const int b = blockIdx.y * 128 + threadIdx.x;
  if (b >= B) return;
  const int64_t g = perm[i];
#pragma unroll
  for (int c = 0; c < 3; c++) Ms[(i * 3 + c) * B + b] = M[((int64_t)b * nn + g) * 3 + c];
}

// ---------------------------------------------------------------------------
// P2M: one block per source leaf
// ---------------------------------------------------------------------------
__global__ void k_p2m(const int32_t* __restrict__ leaves, const int64_t* __restrict__ sup_off,
                      const int32_t* __restrict__ sup_node, const double* __restrict__ Ghat, const double* __restrict__ Ms,
                      int p, int nc, int nc1, int B, double* Q) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  load_mi(nc, mi);
  __syncthreads();
  const int32_t c = leaves[blockIdx.x];
  const int64_t so = sup_off[c], eo = sup_off[c + 1];
  for (int idx = threadIdx.x; idx < nc * B; idx += blockDim.x) {
    const int n = idx / B, b = idx - n * B;
    const int na = mi[n][0], nb = mi[n][1], nz = mi[n][2];
    const int ix = na ? mi_index(na - 1, nb, nz) : -1;
    const int iy = nb ? mi_index(na, nb - 1, nz) : -1;
    const int iz = nz ? mi_index(na, nb, nz - 1) : -1;
    double acc = 0;
    for (int64_t e = so; e < eo; e++) {
      const double* G = Ghat + e * nc1;
      const double* m = Ms + (int64_t)sup_node[e] * 3 * B + b;
      if (ix >= 0) acc += G[ix] * m[0];
      if (iy >= 0) acc += G[iy] * m[B];
      if (iz >= 0) acc += G[iz] * m[2 * B];
    }
    Q[((int64_t)c * nc + n) * B + b] = acc;
  }
}

// ---------------------------------------------------------------------------
// M2M: one block per parent cell of one level
// ---------------------------------------------------------------------------
__global__ void k_m2m(int64_t lb, const int32_t* __restrict__ child0, const int32_t* __restrict__ nchild,
                      const double* __restrict__ centre, int p, int nc, int B, double* Q) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ double s[8][MAX_NCOEF];
  __shared__ double px[3 * (MAX_P + 1)];
  const int64_t P = lb + blockIdx.x;
  const int n_ch = nchild[P];
  if (n_ch == 0) return;
  load_mi(nc, mi);
  __syncthreads();
  const int32_t c0 = child0[P];
  for (int k = 0; k < n_ch; k++) {
    const int32_t C = c0 + k;
    scaled_monomials(p, nc, mi, centre[3 * C] - centre[3 * P], centre[3 * C + 1] - centre[3 * P + 1],
                     centre[3 * C + 2] - centre[3 * P + 2], px, s[k]);
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nc * B; idx += blockDim.x) {
    const int n = idx / B, b = idx - n * B;
    const int na = mi[n][0], nb = mi[n][1], nz = mi[n][2];
    double acc = 0;
    for (int k = 0; k < n_ch; k++) {
      const double* Qc = Q + (int64_t)(c0 + k) * nc * B + b;
      for (int ka = 0; ka <= na; ka++)
        for (int kb = 0; kb <= nb; kb++)
          for (int kz = 0; kz <= nz; kz++)
            acc += s[k][mi_index(na - ka, nb - kb, nz - kz)] * Qc[(int64_t)mi_index(ka, kb, kz) * B];
    }
    Q[(P * nc + n) * B + b] = acc;
  }
}

// ---------------------------------------------------------------------------
// M2L: one block per target cell with a non-empty list
// ---------------------------------------------------------------------------
__global__ void k_m2l_fp64(const int32_t* __restrict__ targets, const int64_t* __restrict__ m2l_off,
                           const int32_t* __restrict__ m2l_src, const double* __restrict__ centre, int p, int nc, int B,
                           const double* __restrict__ Q, double* L) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ double bk[MAX_NCOEF];
  load_mi(nc, mi);
  const int32_t T = targets[blockIdx.x];
  const double cx = centre[3 * T], cy = centre[3 * T + 1], cz = centre[3 * T + 2];
  // this block handles the (m, state) items [i0, i1): at most PER per thread
  constexpr int PER = 4;
  const int i0 = blockIdx.y * blockDim.x * PER, i1 = min(nc * B, i0 + (int)blockDim.x * PER);
  double acc[PER];
  for (int r = 0; r < PER; r++) acc[r] = 0;
  for (int64_t e = m2l_off[T]; e < m2l_off[T + 1]; e++) {
    const int32_t S = m2l_src[e];
    const double x = cx - centre[3 * S], y = cy - centre[3 * S + 1], z = cz - centre[3 * S + 2];
    const double r2 = x * x + y * y + z * z;
    __syncthreads();
    if (threadIdx.x == 0) bk[0] = 1.0 / sqrt(r2);
    __syncthreads();
    for (int t = 1; t <= p; t++) {
      const int o = t * (t + 1) * (t + 2) / 6, cnt = (t + 1) * (t + 2) / 2;
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int k = o + q;
        const int ka = mi[k][0], kb = mi[k][1], kz = mi[k][2];
        double s1 = 0, s2 = 0;
        if (ka) s1 += ka * x * bk[mi_index(ka - 1, kb, kz)];
        if (kb) s1 += kb * y * bk[mi_index(ka, kb - 1, kz)];
        if (kz) s1 += kz * z * bk[mi_index(ka, kb, kz - 1)];
        if (ka > 1) s2 += ka * (ka - 1) * bk[mi_index(ka - 2, kb, kz)];
        if (kb > 1) s2 += kb * (kb - 1) * bk[mi_index(ka, kb - 2, kz)];
        if (kz > 1) s2 += kz * (kz - 1) * bk[mi_index(ka, kb, kz - 2)];
        bk[k] = ((2 * t - 1) * s1 - (t - 1) * s2) / (t * r2);
      }
      __syncthreads();
    }
    const double* Qs = Q + (int64_t)S * nc * B;
    int r = 0;
    for (int idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x, r++) {
      const int m = idx / B, b = idx - m * B;
      const int ma = mi[m][0], mb = mi[m][1], mz = mi[m][2];
      const int tm = ma + mb + mz;
      double a = 0;
      // n over |n| <= p - |m| in graded order
      int n = 0;
      for (int t = 0; t <= p - tm; t++)
        for (int j = 0; j <= t; j++)
          for (int cz2 = 0; cz2 <= j; cz2++, n++) {
            const int na = t - j, nz = cz2, nb = j - cz2;
            a += bk[mi_index(na + ma, nb + mb, nz + mz)] * Qs[(int64_t)n * B + b];
          }
      acc[r] += a;
    }
  }
  int r = 0;
  const double inv4pi = 1.0 / (4.0 * M_PI);
  for (int idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x, r++) {
    const int m = idx / B, b = idx - m * B;
    const int tm = mi[m][0] + mi[m][1] + mi[m][2];
    const double sg = (tm & 1) ? -inv4pi : inv4pi;
    L[((int64_t)T * nc + m) * B + b] = sg * acc[r];
  }
}

// ---------------------------------------------------------------------------
// L2L: one block per cell of one level (cells holding target nodes)
// ---------------------------------------------------------------------------
__global__ void k_l2l(int64_t lb, const int32_t* __restrict__ parent, const int4* __restrict__ range,
                      const double* __restrict__ centre, int p, int nc, int B, double* L) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ double s[MAX_NCOEF];
  __shared__ double px[3 * (MAX_P + 1)];
  const int64_t C = lb + blockIdx.x;
  const int4 r = range[C];
  if (r.w == r.z) return;
  const int32_t P = parent[C];
  load_mi(nc, mi);
  __syncthreads();
  scaled_monomials(p, nc, mi, centre[3 * C] - centre[3 * P], centre[3 * C + 1] - centre[3 * P + 1],
                   centre[3 * C + 2] - centre[3 * P + 2], px, s);
  __syncthreads();
  const double* Lp = L + (int64_t)P * nc * B;
  for (int idx = threadIdx.x; idx < nc * B; idx += blockDim.x) {
    const int m = idx / B, b = idx - m * B;
    const int ma = mi[m][0], mb = mi[m][1], mz = mi[m][2];
    const int tm = ma + mb + mz;
    double acc = 0;
    int j = 0;
    for (int t = 0; t <= p - tm; t++)
      for (int jj = 0; jj <= t; jj++)
        for (int jz = 0; jz <= jj; jz++, j++) {
          const int ja = t - jj, jb = jj - jz;
          acc += s[j] * Lp[(int64_t)mi_index(ma + ja, mb + jb, mz + jz) * B + b];
        }
    L[((int64_t)C * nc + m) * B + b] += acc;
  }
}

// ---------------------------------------------------------------------------
// L2P: one thread per target node
// ---------------------------------------------------------------------------
__global__ void k_l2p(int64_t nn, const int32_t* __restrict__ node_leaf, const double* __restrict__ nodes_s,
                      const double* __restrict__ centre, int p, int nc, int B, const double* __restrict__ L, double* u_s) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
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
    double u = 0;
    int m = 0;
    for (int t = 0; t <= p; t++)
      for (int j = 0; j <= t; j++)
        for (int mz = 0; mz <= j; mz++, m++) u += Lc[(int64_t)m * B + b] * px[t - j] * py[j - mz] * pz[mz];
    u_s[i * B + b] = u;
  }
}

// ---------------------------------------------------------------------------
// mass-lumped H (Sec. 4.1) and the output layout
//   H_i = -sum_{t ni i} |t| grad u_h|_t / sum_{t ni i} |t|
// ---------------------------------------------------------------------------
__global__ void k_lumped_H_out(int64_t nn, int B, const int32_t* __restrict__ perm, const int64_t* __restrict__ nt_off,
                               const int32_t* __restrict__ nt_tet, const int32_t* __restrict__ tets_s,
                               const double* __restrict__ grad, const double* __restrict__ vol,
                               const double* __restrict__ u_s, double* u_out, double* H_out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int64_t g = perm[i];
  for (int b = 0; b < B; b++) u_out[(int64_t)b * nn + g] = u_s[i * B + b];
  if (!H_out) return;
  double V = 0;
  for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) V += vol[nt_tet[e]];
  for (int b = 0; b < B; b++) {
    double h[3] = {0, 0, 0};
    for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) {
      const int64_t t = nt_tet[e];
      const double* gr = grad + 12 * t;
      double gu[3] = {0, 0, 0};
      for (int k = 0; k < 4; k++) {
        const double uk = u_s[(int64_t)tets_s[4 * t + k] * B + b];
        gu[0] += uk * gr[3 * k];
        gu[1] += uk * gr[3 * k + 1];
        gu[2] += uk * gr[3 * k + 2];
      }
      for (int c = 0; c < 3; c++) h[c] += vol[t] * gu[c];
    }
    for (int c = 0; c < 3; c++) H_out[((int64_t)b * nn + g) * 3 + c] = V > 0 ? -h[c] / V : 0.0;
  }
}

// ---------------------------------------------------------------------------
// workspace and the FP64 driver
// ---------------------------------------------------------------------------
static void* ws_alloc(Workspace& W, size_t bytes) {
  void* p = nullptr;
  if (cudaMalloc(&p, bytes ? bytes : 16) != cudaSuccess) {
    cudaGetLastError();
    fail(DEMAG_ERR_OUT_OF_MEMORY, "workspace allocation failed");
  }
  W.ptrs.push_back(p);
  return p;
}

void destroy_workspace(Plan& P) {
  if (!P.ws) return;
  multi_forget_plan(&P);  // graphs recorded with this workspace
  for (void* p : P.ws->ptrs) cudaFree(p);
  delete P.ws;
  P.ws = nullptr;
}

// sized for the largest batch evaluated so far (grown, never shrunk), so a plan
// built for max_batch states holds only what its evaluations use
Workspace& workspace(Plan& P, int B) {
  const int need = B;
  if (P.ws && P.ws->B >= need) return *P.ws;
  destroy_workspace(P);
  Workspace* W = new Workspace();
  W->B = need;
  const size_t nn = P.nn, nt = P.nt, nc = P.nc, ncell = P.ncells;
  const bool mixed = P.opt.precision != DEMAG_FP64, otf = P.opt.near_mode == 0;
  if (!mixed || otf) W->Ms = (double*)ws_alloc(*W, sizeof(double) * nn * 3 * need);  // FP64 sorted M
  if (!mixed) {
    W->Q = (double*)ws_alloc(*W, sizeof(double) * ncell * nc * need);
    W->L = (double*)ws_alloc(*W, sizeof(double) * ncell * nc * need);
  } else {
    W->Ms32 = (float*)ws_alloc(*W, sizeof(float) * nn * 3 * need);
    W->Q32 = (float*)ws_alloc(*W, sizeof(float) * (ncell * nc * need + 16));  // tail pad for 16-byte bulk copies
    W->L32 = (float*)ws_alloc(*W, sizeof(float) * ncell * nc * need);
    W->u32 = (float*)ws_alloc(*W, sizeof(float) * nn * need);
    const size_t qp = m2l_tc_pack_bytes(P, need);
    if (qp) W->QP = (unsigned char*)ws_alloc(*W, qp);
    const size_t mp = nf_mp_floats(P, need);
    if (mp) W->MP = (float*)ws_alloc(*W, sizeof(float) * mp);
  }
  if (!mixed || otf) W->u_s = (double*)ws_alloc(*W, sizeof(double) * nn * need);  // FP64 sorted u
  if (otf) W->state = (double*)ws_alloc(*W, sizeof(double) * nt * TET_STATE * std::min(need, P2P_AT_MIN_B - 1));
  W->err = (int*)ws_alloc(*W, sizeof(int));  // staging for host M, u, H: at the first host-pointer call
  P.ws = W;
  return *W;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void eval_fp64(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s) {
  eval_fp64_ws(P, workspace(P, B), M, B, u, H, s, true);
}

void eval_fp64_ws(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, cudaStream_t s,
                  bool profile_ok) {
  const double* Md;
  double *ud, *Hd;
  const bool dev = eval_io_begin(P, W, M, B, u, H, &Md, &ud, &Hd, s);
  const int p = P.p, nc = P.nc;
  StageClock clk(P, s, profile_ok);
  clk.begin(DEMAG_STAGE_GATHER);
  k_gather_M<<<dim3((unsigned)P.nn, (unsigned)((B + 127) / 128)), 128, 0, s>>>(P.nn, B, P.node_perm, Md, W.Ms);
  DM_LAUNCH("k_gather_M");
  clk.launched();
  clk.end();
  // upward pass
  clk.begin(DEMAG_STAGE_P2M);
  DM_CUDA(cudaMemsetAsync(W.Q, 0, sizeof(double) * P.ncells * nc * B, s));
  if (!P.h_src_leaves.empty()) {
    k_p2m<<<(unsigned)P.h_src_leaves.size(), 128, 0, s>>>(P.src_leaves, P.sup_off, P.sup_node, P.Ghat, W.Ms, p, nc,
                                                          P.nc1, B, W.Q);
    DM_LAUNCH("k_p2m");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_M2M);
  for (int l = P.nlevels - 2; l >= 0; l--) {
    int64_t lb = P.level_start[l], le = P.level_start[l + 1];
    k_m2m<<<(unsigned)(le - lb), 128, 0, s>>>(lb, P.cell_child0, P.cell_nchild, P.cell_centre, p, nc, B, W.Q);
    DM_LAUNCH("k_m2m");
    clk.launched();
  }
  clk.end();
  // M2L
  clk.begin(DEMAG_STAGE_M2L);
  DM_CUDA(cudaMemsetAsync(W.L, 0, sizeof(double) * P.ncells * nc * B, s));
  if (!P.h_m2l_targets.empty()) {
    dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((nc * B + 128 * 4 - 1) / (128 * 4)));
    k_m2l_fp64<<<grid, 128, 0, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, p, nc, B, W.Q, W.L);
    DM_LAUNCH("k_m2l_fp64");
    clk.launched();
  }
  clk.end();
  // downward pass
  clk.begin(DEMAG_STAGE_L2L);
  for (int l = 1; l < P.nlevels; l++) {
    int64_t lb = P.level_start[l], le = P.level_start[l + 1];
    k_l2l<<<(unsigned)(le - lb), 128, 0, s>>>(lb, P.cell_parent, P.cell_range, P.cell_centre, p, nc, B, W.L);
    DM_LAUNCH("k_l2l");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_L2P);
  k_l2p<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, P.node_leaf, P.nodes_s, P.cell_centre, p, nc, B, W.L, W.u_s);
  DM_LAUNCH("k_l2p");
  clk.launched();
  clk.end();
  // near field
  near_field_fp64(P, W, B, clk, s);
  // lumped H and output layout
  clk.begin(DEMAG_STAGE_H);
  launch_lumped_H_out(P, B, W.u_s, ud, Hd, s);
  clk.launched();
  clk.end();
  clk.finish();
  eval_io_end(P, W, dev, B, u, H, s);
}

void near_field_fp64(Plan& P, Workspace& W, int B, StageClock& clk, cudaStream_t s) {
  if (P.opt.near_mode == 1) {
    clk.begin(DEMAG_STAGE_P2P);
    if (!P.h_p2p_targets.empty()) {
      launch_near_apply64(P, W.Ms, B, W.u_s, s);
      clk.launched();
    }
    clk.end();
    return;
  }
  if (B < P2P_AT_MIN_B) {
    clk.begin(DEMAG_STAGE_NEAR_PREP);
    launch_tet_state(P, W.Ms, B, W.state, s);
    clk.launched();
    clk.end();
  }
  clk.begin(DEMAG_STAGE_P2P);
  if (!P.h_p2p_targets.empty()) {
    launch_p2p_fp64(P, W.Ms, W.state, B, W.u_s, W.err, s);
    clk.launched();
  }
  clk.end();
}

void launch_gather_M(Plan& P, const double* M, int B, double* Ms, cudaStream_t s) {
  k_gather_M<<<dim3((unsigned)P.nn, (unsigned)((B + 127) / 128)), 128, 0, s>>>(P.nn, B, P.node_perm, M, Ms);
  DM_LAUNCH("k_gather_M");
}

void launch_lumped_H_out(Plan& P, int B, const double* u_s, double* u, double* H, cudaStream_t s) {
  k_lumped_H_out<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, B, P.node_perm, P.nt_off, P.nt_tet, P.tets_s, P.tet_grad,
                                                 P.tet_vol, u_s, u, H);
  DM_LAUNCH("k_lumped_H_out");
}

// host/device pointer handling shared by the evaluation paths
bool eval_io_begin(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, const double** Md, double** ud,
                   double** Hd, cudaStream_t s) {
  const bool dev = is_device_ptr(M);
  if (dev != is_device_ptr(u) || (H && dev != is_device_ptr(H)))
    fail(DEMAG_ERR_INVALID_ARG, "M, u and H must be all device or all host pointers");
  *Md = M;
  *ud = u;
  *Hd = H;
  if (!dev) {
    if (!W.M_dev) {
      const size_t nn = P.nn, need = W.B;
      W.M_dev = (double*)ws_alloc(W, sizeof(double) * nn * 3 * need);
      W.u_dev = (double*)ws_alloc(W, sizeof(double) * nn * need);
      W.H_dev = (double*)ws_alloc(W, sizeof(double) * nn * 3 * need);
    }
    DM_CUDA(cudaMemcpyAsync(W.M_dev, M, sizeof(double) * P.nn * 3 * B, cudaMemcpyHostToDevice, s));
    *Md = W.M_dev;
    *ud = W.u_dev;
    *Hd = H ? W.H_dev : nullptr;
  }
  DM_CUDA(cudaMemsetAsync(W.err, 0, sizeof(int), s));
  P.last_err = W.err;
  return dev;
}

void eval_io_end(Plan& P, Workspace& W, bool dev, int B, double* u, double* H, cudaStream_t s) {
  if (dev) return;
  DM_CUDA(cudaMemcpyAsync(u, W.u_dev, sizeof(double) * P.nn * B, cudaMemcpyDeviceToHost, s));
  if (H) DM_CUDA(cudaMemcpyAsync(H, W.H_dev, sizeof(double) * P.nn * 3 * B, cudaMemcpyDeviceToHost, s));
  int herr = 0;
  DM_CUDA(cudaMemcpyAsync(&herr, W.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  if (herr) fail((demag_status)herr, "a bounded device wait expired in the near-field kernel");
}

}  // namespace demag
