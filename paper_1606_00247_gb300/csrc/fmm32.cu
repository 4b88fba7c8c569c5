// fmm32.cu -- mixed-precision far field (FP32, per-level scaled expansions)
// and the mixed evaluation driver.
//
// With s the side of a cell, the stored coefficients are
//   Qt_n = Qhat_n / s^|n|      Lt_m = L_m s^|m|
// (Qhat_n = Q_n/n!, L_m = d^m u, see fmm.cu).  All of them are O(1) whatever
// the mesh scale, so FP32 neither overflows nor underflows, and the octree
// translations become level independent:
//   M2M: Qt^P_n = sum_{k<=n} s_{n-k}(+-1/4) 2^-|k| Qt^C_k          (child centre - parent centre = +-s_P/4)
//   L2L: Lt^C_m = sum_{k>=m} s_{k-m}(+-1/2) 2^-|k| Lt^P_k          (= +-s_C/2)
//   M2L: Lt^T_m = (-1)^|m| / (4 pi s_T) sum_n b_{n+m}(v) (s_S/s_T)^|n| Qt^S_n,  v = (c_T - c_S)/s_T
//   L2P: u(c + z) = sum_m s_m(z/s) Lt_m
//   P2M: Qt_n = sum_j sum_c Gt_j[n - e_c] M_c(j),  Gt_j[m] = Ghat_j[m] / s^(|m|+1)
// (s_j(d) = d^j/j!, b_k as in fmm.cu).  The near field is the precomputed
// FP64 coefficient set W rounded to FP32 (near.cu), or the FP64 on-the-fly
// P2P when near_mode = 0.  u is accumulated in FP32 and the mass-lumped H is
// formed in FP64 from it.
#include "common.cuh"

namespace demag {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

namespace {

__device__ __forceinline__ void load_mi(int nc, unsigned char (*mi)[3]) {
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    int a, b, c;
    mi_decode(i, a, b, c);
    mi[i][0] = (unsigned char)a;
    mi[i][1] = (unsigned char)b;
    mi[i][2] = (unsigned char)c;
  }
}

// s_j(d) for |j| <= p; d is one of (+-h, +-h, +-h) given by the octant bits
__device__ __forceinline__ void octant_monomials(int p, int nc, const unsigned char (*mi)[3], int octant, float h,
                                                 float* s) {
  const float dx = (octant & 1) ? h : -h, dy = (octant & 2) ? h : -h, dz = (octant & 4) ? h : -h;
  for (int j = threadIdx.x; j < nc; j += blockDim.x) {
    float v = 1.f;
    for (int e = 1; e <= mi[j][0]; e++) v = v * dx / e;
    for (int e = 1; e <= mi[j][1]; e++) v = v * dy / e;
    for (int e = 1; e <= mi[j][2]; e++) v = v * dz / e;
    s[j] = v;
  }
}

__global__ void k_gather_M32(int64_t nn, int B, const int32_t* __restrict__ perm, const double* __restrict__ M,
                             float* Ms, double* Ms64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int64_t g = perm[i];
  for (int b = 0; b < B; b++)
    for (int c = 0; c < 3; c++) {
      double v = M[((int64_t)b * nn + g) * 3 + c];
      Ms[(i * 3 + c) * B + b] = (float)v;
      if (Ms64) Ms64[(i * 3 + c) * B + b] = v;
    }
}

__global__ void k_ghat32(const int32_t* __restrict__ leaves, const int32_t* __restrict__ level,
                         const int64_t* __restrict__ sup_off, const double* __restrict__ Ghat, double side, int nc1,
                         float* G32) {
  const int32_t c = leaves[blockIdx.x];
  const double s = ldexp(side, -level[c]);
  for (int64_t e = sup_off[c]; e < sup_off[c + 1]; e++)
    for (int m = threadIdx.x; m < nc1; m += blockDim.x) {
      int a, b, z;
      mi_decode(m, a, b, z);
      G32[e * nc1 + m] = (float)(Ghat[e * nc1 + m] / pow(s, a + b + z + 1));
    }
}

__global__ void k_p2m32(const int32_t* __restrict__ leaves, const int64_t* __restrict__ sup_off,
                        const int32_t* __restrict__ sup_node, const float* __restrict__ G, const float* __restrict__ Ms,
                        int nc, int nc1, int B, float* Q) {
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
    float acc = 0;
    for (int64_t e = so; e < eo; e++) {
      const float* g = G + e * nc1;
      const float* m = Ms + (int64_t)sup_node[e] * 3 * B + b;
      if (ix >= 0) acc += g[ix] * m[0];
      if (iy >= 0) acc += g[iy] * m[B];
      if (iz >= 0) acc += g[iz] * m[2 * B];
    }
    Q[((int64_t)c * nc + n) * B + b] = acc;
  }
}

__global__ void k_m2m32(int64_t lb, const int32_t* __restrict__ child0, const int32_t* __restrict__ nchild,
                        const uint64_t* __restrict__ prefix, int p, int nc, int B, float* Q) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ float s[8][MAX_NCOEF];
  const int64_t P = lb + blockIdx.x;
  const int n_ch = nchild[P];
  if (n_ch == 0) return;
  load_mi(nc, mi);
  __syncthreads();
  const int32_t c0 = child0[P];
  for (int k = 0; k < n_ch; k++) octant_monomials(p, nc, mi, (int)(prefix[c0 + k] & 7ull), 0.25f, s[k]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < nc * B; idx += blockDim.x) {
    const int n = idx / B, b = idx - n * B;
    const int na = mi[n][0], nb = mi[n][1], nz = mi[n][2];
    float acc = 0;
    for (int k = 0; k < n_ch; k++) {
      const float* Qc = Q + (int64_t)(c0 + k) * nc * B + b;
      for (int ka = 0; ka <= na; ka++)
        for (int kb = 0; kb <= nb; kb++)
          for (int kz = 0; kz <= nz; kz++)
            acc += s[k][mi_index(na - ka, nb - kb, nz - kz)] * ldexpf(Qc[(int64_t)mi_index(ka, kb, kz) * B],
                                                                    -(ka + kb + kz));
    }
    Q[(P * nc + n) * B + b] = acc;
  }
}

// CUDA-core M2L: one block per target cell, threads over (m, state)
__global__ void k_m2l32(const int32_t* __restrict__ targets, const int64_t* __restrict__ m2l_off,
                        const int32_t* __restrict__ m2l_src, const double* __restrict__ centre,
                        const int32_t* __restrict__ level, double side, int p, int nc, int B,
                        const float* __restrict__ Q, float* L) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ float bk[MAX_NCOEF];
  __shared__ float fp[MAX_P + 1];
  load_mi(nc, mi);
  const int32_t T = targets[blockIdx.x];
  const double sT = ldexp(side, -level[T]);
  const double cx = centre[3 * T], cy = centre[3 * T + 1], cz = centre[3 * T + 2];
  // this block handles the (m, state) items [i0, i1): at most PER per thread
  constexpr int PER = 8;
  const int i0 = blockIdx.y * blockDim.x * PER, i1 = min(nc * B, i0 + (int)blockDim.x * PER);
  float acc[PER];
  for (int r = 0; r < PER; r++) acc[r] = 0;
  for (int64_t e = m2l_off[T]; e < m2l_off[T + 1]; e++) {
    const int32_t S = m2l_src[e];
    const float x = (float)((cx - centre[3 * S]) / sT), y = (float)((cy - centre[3 * S + 1]) / sT),
                z = (float)((cz - centre[3 * S + 2]) / sT);
    const float r2 = x * x + y * y + z * z;
    const int dl = level[T] - level[S];  // s_S / s_T = 2^dl
    __syncthreads();
    if (threadIdx.x == 0) bk[0] = rsqrtf(r2);
    if (threadIdx.x <= p) fp[threadIdx.x] = ldexpf(1.f, dl * (int)threadIdx.x);
    __syncthreads();
    for (int t = 1; t <= p; t++) {
      const int o = t * (t + 1) * (t + 2) / 6, cnt = (t + 1) * (t + 2) / 2;
      for (int q = threadIdx.x; q < cnt; q += blockDim.x) {
        const int k = o + q;
        const int ka = mi[k][0], kb = mi[k][1], kz = mi[k][2];
        float s1 = 0, s2 = 0;
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
    const float* Qs = Q + (int64_t)S * nc * B;
    int r = 0;
    for (int idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x, r++) {
      const int m = idx / B, b = idx - m * B;
      const int ma = mi[m][0], mb = mi[m][1], mz = mi[m][2];
      const int tm = ma + mb + mz;
      float a = 0;
      int n = 0;
      for (int t = 0; t <= p - tm; t++) {
        float at = 0;
        for (int j = 0; j <= t; j++)
          for (int cz2 = 0; cz2 <= j; cz2++, n++)
            at += bk[mi_index(t - j + ma, j - cz2 + mb, cz2 + mz)] * Qs[(int64_t)n * B + b];
        a += fp[t] * at;
      }
      acc[r] += a;
    }
  }
  int r = 0;
  const float inv = (float)(1.0 / (4.0 * M_PI * sT));
  for (int idx = i0 + threadIdx.x; idx < i1; idx += blockDim.x, r++) {
    const int m = idx / B, b = idx - m * B;
    const int tm = mi[m][0] + mi[m][1] + mi[m][2];
    const float sg = (tm & 1) ? -inv : inv;
    L[((int64_t)T * nc + m) * B + b] = sg * acc[r];
  }
}

__global__ void k_l2l32(int64_t lb, const int32_t* __restrict__ parent, const int4* __restrict__ range,
                        const uint64_t* __restrict__ prefix, int p, int nc, int B, float* L) {
  __shared__ unsigned char mi[MAX_NCOEF][3];
  __shared__ float s[MAX_NCOEF];
  const int64_t C = lb + blockIdx.x;
  const int4 r = range[C];
  if (r.w == r.z) return;
  const int32_t P = parent[C];
  load_mi(nc, mi);
  __syncthreads();
  octant_monomials(p, nc, mi, (int)(prefix[C] & 7ull), 0.5f, s);
  __syncthreads();
  const float* Lp = L + (int64_t)P * nc * B;
  for (int idx = threadIdx.x; idx < nc * B; idx += blockDim.x) {
    const int m = idx / B, b = idx - m * B;
    const int ma = mi[m][0], mb = mi[m][1], mz = mi[m][2];
    const int tm = ma + mb + mz;
    float acc = 0;
    int j = 0;
    for (int t = 0; t <= p - tm; t++)
      for (int jj = 0; jj <= t; jj++)
        for (int jz = 0; jz <= jj; jz++, j++) {
          const int ja = t - jj, jb = jj - jz;
          acc += s[j] * ldexpf(Lp[(int64_t)mi_index(ma + ja, mb + jb, mz + jz) * B + b], -(tm + t));
        }
    L[((int64_t)C * nc + m) * B + b] += acc;
  }
}

__global__ void k_l2p32(int64_t nn, const int32_t* __restrict__ node_leaf, const int32_t* __restrict__ level,
                        const double* __restrict__ nodes_s, const double* __restrict__ centre, double side, int p,
                        int nc, int B, const float* __restrict__ L, float* u) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  const int32_t c = node_leaf[i];
  const double inv_s = 1.0 / ldexp(side, -level[c]);
  float px[MAX_P + 1], py[MAX_P + 1], pz[MAX_P + 1];
  const float zx = (float)((nodes_s[3 * i] - centre[3 * c]) * inv_s),
              zy = (float)((nodes_s[3 * i + 1] - centre[3 * c + 1]) * inv_s),
              zz = (float)((nodes_s[3 * i + 2] - centre[3 * c + 2]) * inv_s);
  px[0] = py[0] = pz[0] = 1.f;
  for (int e = 1; e <= p; e++) {
    px[e] = px[e - 1] * zx / e;
    py[e] = py[e - 1] * zy / e;
    pz[e] = pz[e - 1] * zz / e;
  }
  const float* Lc = L + (int64_t)c * nc * B;
  for (int b = 0; b < B; b++) {
    float v = 0;
    int m = 0;
    for (int t = 0; t <= p; t++)
      for (int j = 0; j <= t; j++)
        for (int mz = 0; mz <= j; mz++, m++) v += Lc[(int64_t)m * B + b] * px[t - j] * py[j - mz] * pz[mz];
    u[i * B + b] = v;
  }
}

__global__ void k_u32_to_64(int64_t n, const float* __restrict__ a, double* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

void build_mixed_operators(Plan& P) {
  cudaStream_t s = P.stream;
  P.Ghat32 = dalloc<float>(P, std::max<int64_t>(P.n_sup, 1) * P.nc1);
  if (!P.h_src_leaves.empty()) {
    k_ghat32<<<(unsigned)P.h_src_leaves.size(), 128, 0, s>>>(P.src_leaves, P.cell_level, P.sup_off, P.Ghat, P.side,
                                                             P.nc1, P.Ghat32);
    DM_LAUNCH("k_ghat32");
  }
  build_m2l_tc(P);
}

void eval_mixed(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s) {
  eval_mixed_ws(P, workspace(P, B), M, B, u, H, s, true);
}

void eval_mixed_ws(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, cudaStream_t s,
                   bool profile_ok) {
  const double* Md;
  double *ud, *Hd;
  const bool dev = eval_io_begin(P, W, M, B, u, H, &Md, &ud, &Hd, s);
  const bool otf = P.opt.near_mode == 0;
  const int p = P.p, nc = P.nc;
  StageClock clk(P, s, profile_ok);
  clk.begin(DEMAG_STAGE_GATHER);
  k_gather_M32<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, B, P.node_perm, Md, W.Ms32, otf ? W.Ms : nullptr);
  DM_LAUNCH("k_gather_M32");
  clk.launched();
  clk.end();
  clk.begin(DEMAG_STAGE_P2M);
  DM_CUDA(cudaMemsetAsync(W.Q32, 0, sizeof(float) * P.ncells * nc * B, s));
  if (!P.h_src_leaves.empty()) {
    k_p2m32<<<(unsigned)P.h_src_leaves.size(), 128, 0, s>>>(P.src_leaves, P.sup_off, P.sup_node, P.Ghat32, W.Ms32,
                                                            nc, P.nc1, B, W.Q32);
    DM_LAUNCH("k_p2m32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_M2M);
  for (int l = P.nlevels - 2; l >= 0; l--) {
    int64_t lb = P.level_start[l], le = P.level_start[l + 1];
    k_m2m32<<<(unsigned)(le - lb), 128, 0, s>>>(lb, P.cell_child0, P.cell_nchild, P.cell_prefix, p, nc, B, W.Q32);
    DM_LAUNCH("k_m2m32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_M2L);
  DM_CUDA(cudaMemsetAsync(W.L32, 0, sizeof(float) * P.ncells * nc * B, s));
  if (P.h_m2l_targets.empty()) {
  } else if ((P.opt.precision == DEMAG_MIXED_TF32 || P.opt.precision == DEMAG_MIXED_BF16X3) &&
             launch_m2l_tc(P, B, W.Q32, W.QP, W.L32, W.err, s)) {
    clk.launched(2);
  } else if (launch_m2l32_fast(P, B, W.Q32, W.L32, W.err, s)) {
    clk.launched();
  } else {
    dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((nc * B + 128 * 8 - 1) / (128 * 8)));
    k_m2l32<<<grid, 128, 0, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, P.cell_level, P.side, p, nc, B,
                                 W.Q32, W.L32);
    DM_LAUNCH("k_m2l32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_L2L);
  for (int l = 1; l < P.nlevels; l++) {
    int64_t lb = P.level_start[l], le = P.level_start[l + 1];
    k_l2l32<<<(unsigned)(le - lb), 128, 0, s>>>(lb, P.cell_parent, P.cell_range, P.cell_prefix, p, nc, B, W.L32);
    DM_LAUNCH("k_l2l32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_L2P);
  k_l2p32<<<nblk(P.nn, 128), 128, 0, s>>>(P.nn, P.node_leaf, P.cell_level, P.nodes_s, P.cell_centre, P.side, p, nc, B,
                                          W.L32, W.u32);
  DM_LAUNCH("k_l2p32");
  clk.launched();
  clk.end();
  if (otf) {
    k_u32_to_64<<<nblk(P.nn * B, 256), 256, 0, s>>>(P.nn * B, W.u32, W.u_s);
    DM_LAUNCH("k_u32_to_64");
    near_field_fp64(P, W, B, clk, s);
  } else {
    clk.begin(DEMAG_STAGE_P2P);
    if (!P.h_p2p_targets.empty()) {
      launch_near_apply32(P, W.Ms32, B, W.u32, W.err, s);
      clk.launched();
    }
    clk.end();
  }
  clk.begin(DEMAG_STAGE_H);
  if (!otf) {
    k_u32_to_64<<<nblk(P.nn * B, 256), 256, 0, s>>>(P.nn * B, W.u32, W.u_s);
    DM_LAUNCH("k_u32_to_64");
    clk.launched();
  }
  launch_lumped_H_out(P, B, W.u_s, ud, Hd, s);
  clk.launched();
  clk.end();
  clk.finish();
  eval_io_end(P, W, dev, B, u, H, s);
}

}  // namespace demag
