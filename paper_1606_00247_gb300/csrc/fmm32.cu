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
#include <algorithm>
#include <array>
#include <cmath>

#include "common.cuh"

namespace demag {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

namespace {

// M (state, original node, component) -> Ms (sorted node, component, state):
// block per (sorted node, 128 states), thread = state, so the stores coalesce
// over the states; each thread reads the 24 contiguous bytes of its state's
// (node, x y z) row
__global__ void __launch_bounds__(128) k_gather_M32(int64_t nn, int B, const int32_t* __restrict__ perm,
                                                    const double* __restrict__ M, float* Ms, double* Ms64) {
  const int64_t i = blockIdx.x;
  const int b = blockIdx.y * 128 + threadIdx.x;
  if (b >= B) return;
  const int64_t g = perm[i];
  const double* src = M + ((int64_t)b * nn + g) * 3;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const double v = src[c];
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

// P2M: one block per (source leaf, 56 coefficients n, 128 SPT states), 128
// threads, thread = SPT states (bl, bl + 128; three blocks per leaf at
// p = 8).  Support nodes come in chunks of P2M_NE, double-buffered in shared
// memory by asynchronous copies (cp.async), the next chunk in flight while the
// current one is applied: per node the 168 values Gt[n - e_c] the block's 56
// coefficients need (0 where n_c = 0), in the order of use, and M of the
// states.  One node costs 42 broadcast 16-byte reads of Gt for 168 SPT FMAs
// (two states per thread halve the shared-memory reads per FMA).
constexpr int P2M_NN = 56, P2M_NE = 8, P2M_B = 128;
template <int SPT>
constexpr size_t p2m_smem() {  // two chunk buffers
  return sizeof(float) * 2 * P2M_NE * (P2M_NN * 3 + 3 * SPT * P2M_B);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

template <int SPT>
__global__ void __launch_bounds__(P2M_B) k_p2m32(const int32_t* __restrict__ leaves,
                                                 const int64_t* __restrict__ sup_off,
                                                 const int32_t* __restrict__ sup_node, const float* __restrict__ G,
                                                 const float* __restrict__ Ms, int nc, int nc1, int B, float* Q) {
  constexpr int NS = SPT * P2M_B;  // states per block
  extern __shared__ __align__(16) float p2m_smem_[];
  float(*sG)[P2M_NE][P2M_NN * 3] = (float(*)[P2M_NE][P2M_NN * 3])p2m_smem_;        // [2][node][(j, c)]
  float(*sM)[P2M_NE][3][NS] = (float(*)[P2M_NE][3][NS])(p2m_smem_ + 2 * P2M_NE * P2M_NN * 3);  // [2][node][c][state]
  __shared__ int six[P2M_NN * 3];
  const int32_t c = leaves[blockIdx.x];
  const int n0 = blockIdx.y * P2M_NN;
  const int tid = threadIdx.x, bb = blockIdx.z * NS;
  for (int t = tid; t < P2M_NN * 3; t += blockDim.x) {
    const int j = t / 3, comp = t - 3 * j;
    int na = 0, nb = 0, nz = 0, ix = -1;
    if (n0 + j < nc) {
      mi_decode(n0 + j, na, nb, nz);
      if (comp == 0 && na) ix = mi_index(na - 1, nb, nz);
      if (comp == 1 && nb) ix = mi_index(na, nb - 1, nz);
      if (comp == 2 && nz) ix = mi_index(na, nb, nz - 1);
    }
    six[t] = ix;
  }
  __syncthreads();
  const int64_t so = sup_off[c], eo = sup_off[c + 1];
  auto stage = [&](int64_t e0, int buf) {  // one chunk of support nodes into buffer buf
    const int ne = (int)min((int64_t)P2M_NE, eo - e0);
    for (int q = tid; q < P2M_NE * P2M_NN * 3; q += blockDim.x) {
      const int r = q / (P2M_NN * 3), jc = q - r * (P2M_NN * 3);
      const int ix = six[jc];
      const bool ok = r < ne && ix >= 0;
      cp_async4(&sG[buf][r][jc], ok ? G + (e0 + r) * nc1 + ix : G, ok);
    }
    for (int r = 0; r < P2M_NE; r++) {
      const int64_t node = r < ne ? sup_node[e0 + r] : 0;
#pragma unroll
      for (int s2 = 0; s2 < SPT; s2++) {
        const int b = bb + s2 * P2M_B + tid;
        const bool ok = r < ne && b < B;
        const float* mp = Ms + (ok ? node * 3 * B + b : 0);
#pragma unroll
        for (int cc = 0; cc < 3; cc++) cp_async4(&sM[buf][r][cc][s2 * P2M_B + tid], ok ? mp + (int64_t)cc * B : Ms, ok);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[SPT][P2M_NN];
#pragma unroll
  for (int s2 = 0; s2 < SPT; s2++)
#pragma unroll
    for (int j = 0; j < P2M_NN; j++) acc[s2][j] = 0.f;
  if (so < eo) stage(so, 0);
  int buf = 0;
  for (int64_t e0 = so; e0 < eo; e0 += P2M_NE, buf ^= 1) {
    const int ne = (int)min((int64_t)P2M_NE, eo - e0);
    if (e0 + P2M_NE < eo) {
      stage(e0 + P2M_NE, buf ^ 1);  // the other buffer was released by the barrier that ended the last chunk
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();  // this chunk complete in shared memory for every thread
    for (int r = 0; r < ne; r++) {
      float m[SPT][3];
#pragma unroll
      for (int s2 = 0; s2 < SPT; s2++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) m[s2][cc] = sM[buf][r][cc][s2 * P2M_B + tid];
      const float4* g4 = (const float4*)sG[buf][r];
#pragma unroll
      for (int q = 0; q < P2M_NN * 3 / 4; q++) {
        const float4 g = g4[q];  // values 4q .. 4q+3 = (j, comp) pairs in order
        const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int jc = 4 * q + u, j = jc / 3, comp = jc % 3;
#pragma unroll
          for (int s2 = 0; s2 < SPT; s2++) acc[s2][j] = fmaf(gv[u], m[s2][comp], acc[s2][j]);
        }
      }
    }
    __syncthreads();  // the buffer may be refilled
  }
#pragma unroll
  for (int s2 = 0; s2 < SPT; s2++) {
    const int b = bb + s2 * P2M_B + tid;
    if (b < B)
#pragma unroll
      for (int j = 0; j < P2M_NN; j++)
        if (n0 + j < nc) Q[((int64_t)c * nc + n0 + j) * B + b] = acc[s2][j];
  }
}

// M2M of one level: thread per (cell, n, state); the warp shares (cell, n), so
// the coefficient list is read as a broadcast and the child moments coalesce
__global__ void k_m2m32(const int32_t* __restrict__ parents, int64_t npar, const int32_t* __restrict__ child0,
                        const int32_t* __restrict__ nchild, const uint64_t* __restrict__ prefix,
                        const int32_t* __restrict__ eoff, const TEnt* __restrict__ ent, int nc, int B, float* Q) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nc * B;
  if (idx >= npar * per) return;
  const int64_t P = parents[idx / per];
  const int rem = (int)(idx % per), n = rem / B, b = rem - n * B;
  const int nch = nchild[P];
  const int32_t c0 = child0[P];
  const int e0 = eoff[n], e1 = eoff[n + 1];
  float acc = 0.f;
  for (int k = 0; k < nch; k++) {
    const int oct = (int)(prefix[c0 + k] & 7ull);
    const float* Qc = Q + (int64_t)(c0 + k) * per + b;
    for (int e = e0; e < e1; e++) {
      const TEnt E = ent[e];
      const float v = Qc[(int64_t)E.k * B];
      acc = fmaf(((E.neg >> oct) & 1) ? -E.c : E.c, v, acc);
    }
  }
  Q[P * per + (int64_t)n * B + b] = acc;
}

// L2L from the parents of one level: thread per (parent, m, state) feeding all
// children at once (each parent coefficient is loaded once; the octant only
// flips signs); added to the children's own M2L results
__global__ void k_l2l32(const int32_t* __restrict__ parents, int64_t npar, const int32_t* __restrict__ child0,
                        const int32_t* __restrict__ nchild, const int4* __restrict__ range,
                        const uint64_t* __restrict__ prefix, const int32_t* __restrict__ eoff,
                        const TEnt* __restrict__ ent, int nc, int B, float* L) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)nc * B;
  if (idx >= npar * per) return;
  const int64_t P = parents[idx / per];
  const int nch = nchild[P];
  if (range[P].w == range[P].z) return;  // no target node below this cell
  const int rem = (int)(idx % per), m = rem / B, b = rem - m * B;
  const int32_t c0 = child0[P];
  int oct[8];
  float acc[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    oct[k] = k < nch ? (int)(prefix[c0 + k] & 7ull) : 0;
    acc[k] = 0.f;
  }
  const float* Lp = L + P * per + b;
  for (int e = eoff[m], e1 = eoff[m + 1]; e < e1; e++) {
    const TEnt E = ent[e];
    const float v = E.c * Lp[(int64_t)E.k * B];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] += ((E.neg >> oct[k]) & 1) ? -v : v;
  }
#pragma unroll
  for (int k = 0; k < 8; k++)
    if (k < nch) {
      const int4 r = range[c0 + k];
      if (r.w > r.z) L[(int64_t)(c0 + k) * per + (int64_t)m * B + b] += acc[k];  // only cells with target nodes
    }
}

// L2P, node-wise (orders whose leaf-wise tile exceeds shared memory): block
// per (node, 128 states); the node's monomials s_m(z/s) are formed once in
// shared memory, then thread = state: u = sum_m Lt_m s_m (coalesced L)
__global__ void __launch_bounds__(128) k_l2p32(const int32_t* __restrict__ node_leaf, const int32_t* __restrict__ level,
                                               const double* __restrict__ nodes_s, const double* __restrict__ centre,
                                               double side, int nc, int B, const float* __restrict__ L, float* u) {
  __shared__ float sm_[MAX_NCOEF];
  const int64_t i = blockIdx.x;
  const int32_t c = node_leaf[i];
  const double inv_s = 1.0 / ldexp(side, -level[c]);
  const float z[3] = {(float)((nodes_s[3 * i] - centre[3 * c]) * inv_s),
                      (float)((nodes_s[3 * i + 1] - centre[3 * c + 1]) * inv_s),
                      (float)((nodes_s[3 * i + 2] - centre[3 * c + 2]) * inv_s)};
  for (int m = threadIdx.x; m < nc; m += blockDim.x) {
    int e[3];
    mi_decode(m, e[0], e[1], e[2]);
    float v = 1.f;
    for (int a = 0; a < 3; a++)
      for (int k = 1; k <= e[a]; k++) v = v * z[a] / k;
    sm_[m] = v;
  }
  __syncthreads();
  const int b = blockIdx.y * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float* Lc = L + (int64_t)c * nc * B + b;
  float v0 = 0.f, v1 = 0.f;
  int m = 0;
  for (; m + 1 < nc; m += 2) {
    v0 = fmaf(Lc[(int64_t)m * B], sm_[m], v0);
    v1 = fmaf(Lc[(int64_t)(m + 1) * B], sm_[m + 1], v1);
  }
  if (m < nc) v0 = fmaf(Lc[(int64_t)m * B], sm_[m], v0);
  u[i * B + b] = v0 + v1;
}

// L2P, leaf-wise: block per (leaf holding nodes, 128 states), 512 threads.
// The leaf's local expansion (nc coefficients x 128 states, 84 KB at p = 8)
// is staged once in shared memory by asynchronous copies (coalesced over
// states); the nodes follow in chunks of 16: their monomials s_m(z/s) are
// formed in shared memory ([m][16 nodes]), and thread (group g, state b)
// accumulates the potentials of nodes 4g .. 4g + 3 of the chunk, per m one
// read of its coefficient and one broadcast float4 of monomials.
constexpr int L2P_NCH = 16, L2P_THREADS = 512;

__global__ void __launch_bounds__(L2P_THREADS) k_l2p32_leaf(const int32_t* __restrict__ leaves,
                                                            const int4* __restrict__ range,
                                                            const int32_t* __restrict__ level,
                                                            const double* __restrict__ nodes_s,
                                                            const double* __restrict__ centre, double side, int nc,
                                                            int B, const float* __restrict__ L, float* u) {
  extern __shared__ __align__(16) float l2p_smem[];
  float* sL = l2p_smem;                                // [m][128 states]
  float4* smono = (float4*)(l2p_smem + nc * 128);      // [m][16 nodes] as 4 float4
  const int32_t c = leaves[blockIdx.x];
  const int4 r = range[c];
  const int tid = threadIdx.x, bl = tid & 127, grp = tid >> 7, b = blockIdx.y * 128 + bl;
  const bool live = b < B;
  if (grp == 0) {  // the tile by asynchronous 4-byte copies, all in flight (zero fill beyond B)
    const float* Lc = L + (int64_t)c * nc * B + (live ? b : 0);
    for (int m = 0; m < nc; m++)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(
                       sL + m * 128 + bl)),
                   "l"(Lc + (int64_t)m * B), "r"(live ? 4 : 0)
                   : "memory");
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  const double inv_s = 1.0 / ldexp(side, -level[c]);
  float* sm = (float*)smono;
  for (int32_t i0 = r.z; i0 < r.w; i0 += L2P_NCH) {
    const int nk = min(L2P_NCH, r.w - i0);
    __syncthreads();  // sL complete (first chunk); the previous chunk's monomials are read
    // monomials: thread t forms those of node t % 16 for m = t / 16, t / 16 + 32, ...
    {
      const int k = tid & (L2P_NCH - 1);
      float z[3] = {0.f, 0.f, 0.f};
      if (k < nk) {
        const int64_t i = i0 + k;
#pragma unroll
        for (int a = 0; a < 3; a++) z[a] = (float)((nodes_s[3 * i + a] - centre[3 * c + a]) * inv_s);
      }
      for (int m = tid / L2P_NCH; m < nc; m += L2P_THREADS / L2P_NCH) {
        int e[3];
        mi_decode(m, e[0], e[1], e[2]);
        float v = 1.f;
        for (int a = 0; a < 3; a++)
          for (int q = 1; q <= e[a]; q++) v = v * z[a] / q;
        sm[m * L2P_NCH + k] = v;
      }
    }
    __syncthreads();
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
    for (int m = 0; m < nc; m++) {
      const float l = sL[m * 128 + bl];
      const float4 w = smono[m * (L2P_NCH / 4) + grp];
      a0 = fmaf(l, w.x, a0);
      a1 = fmaf(l, w.y, a1);
      a2 = fmaf(l, w.z, a2);
      a3 = fmaf(l, w.w, a3);
    }
    if (live) {
      const int k0 = 4 * grp;
      if (k0 < nk) u[(int64_t)(i0 + k0) * B + b] = a0;
      if (k0 + 1 < nk) u[(int64_t)(i0 + k0 + 1) * B + b] = a1;
      if (k0 + 2 < nk) u[(int64_t)(i0 + k0 + 2) * B + b] = a2;
      if (k0 + 3 < nk) u[(int64_t)(i0 + k0 + 3) * B + b] = a3;
    }
  }
}

void launch_l2p32(Plan& P, int B, const float* L, float* u, cudaStream_t s) {
  const size_t smem = sizeof(float) * (size_t)P.nc * (128 + L2P_NCH);
  if (smem > 227 * 1024) {  // p = 12: the node-wise kernel
    k_l2p32<<<dim3((unsigned)P.nn, (unsigned)((B + 127) / 128)), 128, 0, s>>>(P.node_leaf, P.cell_level, P.nodes_s,
                                                                               P.cell_centre, P.side, P.nc, B, L, u);
    DM_LAUNCH("k_l2p32");
    return;
  }
  if (P.n_node_leaves == 0) return;
  smem_opt_in((const void*)k_l2p32_leaf, smem);
  const dim3 grid((unsigned)P.n_node_leaves, (unsigned)((B + 127) / 128));
  k_l2p32_leaf<<<grid, L2P_THREADS, smem, s>>>(P.node_leaves, P.cell_range, P.cell_level, P.nodes_s,
                                               P.cell_centre, P.side, P.nc, B, L, u);
  DM_LAUNCH("k_l2p32_leaf");
}

// u and the mass-lumped H of the mixed path, in the caller's layout: tiles of
// 32 original nodes x 32 states; reads coalesce over states, the transposed
// tile is written coalesced over nodes
__global__ void __launch_bounds__(256) k_out32(int64_t nn, int B, const int32_t* __restrict__ iperm,
                                               const int64_t* __restrict__ hoff, const int32_t* __restrict__ hcol,
                                               const float4* __restrict__ hw, const float* __restrict__ u32,
                                               double* u_out, double* H_out) {
  __shared__ float su[32][33];
  __shared__ float sh[32][97];
  const int64_t g0 = (int64_t)blockIdx.x * 32;
  const int b0 = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int b = b0 + lane;
  for (int r = w; r < 32; r += 8) {
    const int64_t g = g0 + r;
    float uu = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
    if (g < nn && b < B) {
      const int64_t i = iperm[g];
      uu = u32[i * B + b];
      if (H_out)
        for (int64_t e = hoff[i], e1 = hoff[i + 1]; e < e1; e++) {
          const float4 wv = hw[e];
          const float uj = u32[(int64_t)hcol[e] * B + b];
          hx = fmaf(wv.x, uj, hx);
          hy = fmaf(wv.y, uj, hy);
          hz = fmaf(wv.z, uj, hz);
        }
    }
    su[lane][r] = uu;
    sh[lane][3 * r] = hx;
    sh[lane][3 * r + 1] = hy;
    sh[lane][3 * r + 2] = hz;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * 32; q += blockDim.x) {
    const int bl = q >> 5, gl = q & 31;
    if (b0 + bl < B && g0 + gl < nn) u_out[(int64_t)(b0 + bl) * nn + g0 + gl] = (double)su[bl][gl];
  }
  if (H_out)
    for (int q = threadIdx.x; q < 32 * 96; q += blockDim.x) {
      const int bl = q / 96, rr = q - bl * 96;
      if (b0 + bl < B && g0 + rr / 3 < nn) H_out[((int64_t)(b0 + bl) * nn + g0) * 3 + rr] = (double)sh[bl][rr];
    }
}

__global__ void k_u32_to_64(int64_t n, const float* __restrict__ a, double* b) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

// coefficient lists of the FP32 translations (see the file header):
//   M2M  n <- k <= n,  j = n - k:  c = s_j(1/4) 2^-|k|, child centre - parent centre = +-s_P/4
//   L2L  m <- k = m + j, |k| <= p:  c = s_j(1/2) 2^-|k|, child centre - parent centre = +-s_C/2
// with the sign of s_j(d) for the child octant o: d_i = +h if bit i of o is set, else -h
static void build_translations(Plan& P) {
  const int p = P.p, nc = P.nc;
  std::vector<int> a(nc), b(nc), c(nc);
  for (int i = 0; i < nc; i++) mi_decode(i, a[i], b[i], c[i]);
  auto fact = [](int n) {
    double f = 1;
    for (int i = 2; i <= n; i++) f *= i;
    return f;
  };
  auto neg_bits = [](int ja, int jb, int jc) {
    int bits = 0;
    for (int o = 0; o < 8; o++) {
      int odd = ((o & 1) ? 0 : ja) + ((o & 2) ? 0 : jb) + ((o & 4) ? 0 : jc);
      if (odd & 1) bits |= 1 << o;
    }
    return (uint8_t)bits;
  };
  std::vector<int32_t> moff(nc + 1), loff(nc + 1);
  std::vector<TEnt> ment, lent;
  for (int n = 0; n < nc; n++) {
    moff[n] = (int32_t)ment.size();
    for (int k = 0; k < nc; k++) {
      if (a[k] > a[n] || b[k] > b[n] || c[k] > c[n]) continue;
      const int ja = a[n] - a[k], jb = b[n] - b[k], jc = c[n] - c[k], tj = ja + jb + jc, tk = a[k] + b[k] + c[k];
      const double cf = std::pow(0.25, tj) / (fact(ja) * fact(jb) * fact(jc)) * std::ldexp(1.0, -tk);
      ment.push_back(TEnt{(uint16_t)k, neg_bits(ja, jb, jc), 0, (float)cf});
    }
  }
  moff[nc] = (int32_t)ment.size();
  for (int m = 0; m < nc; m++) {
    loff[m] = (int32_t)lent.size();
    const int tm = a[m] + b[m] + c[m];
    for (int j = 0; j < nc; j++) {
      const int tj = a[j] + b[j] + c[j];
      if (tm + tj > p) continue;
      const int k = mi_index(a[m] + a[j], b[m] + b[j], c[m] + c[j]);
      const double cf = std::pow(0.5, tj) / (fact(a[j]) * fact(b[j]) * fact(c[j])) * std::ldexp(1.0, -(tm + tj));
      lent.push_back(TEnt{(uint16_t)k, neg_bits(a[j], b[j], c[j]), 0, (float)cf});
    }
  }
  loff[nc] = (int32_t)lent.size();
  cudaStream_t s = P.stream;
  P.m2m_eoff = dalloc<int32_t>(P, nc + 1);
  P.m2m_ent = dalloc<TEnt>(P, ment.size());
  P.l2l_eoff = dalloc<int32_t>(P, nc + 1);
  P.l2l_ent = dalloc<TEnt>(P, lent.size());
  DM_CUDA(cudaMemcpyAsync(P.m2m_eoff, moff.data(), moff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemcpyAsync(P.m2m_ent, ment.data(), ment.size() * sizeof(TEnt), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemcpyAsync(P.l2l_eoff, loff.data(), loff.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemcpyAsync(P.l2l_ent, lent.data(), lent.size() * sizeof(TEnt), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaStreamSynchronize(s));
}

// mass-lumped gradient (Sec. 4.1) as a sparse FP32 operator on u: row i holds,
// for every node j sharing a tet with i, -(1/V_i) sum_{t ni i, j} vol_t grad lambda_j^t
static void build_gradient_operator(Plan& P) {
  cudaStream_t s = P.stream;
  const int64_t nn = P.nn, nt = P.nt;
  std::vector<int32_t> tets(4 * nt), nt_tet(4 * nt), perm(nn);
  std::vector<double> grad(12 * nt), vol(nt);
  std::vector<int64_t> nt_off(nn + 1);
  DM_CUDA(cudaMemcpyAsync(tets.data(), P.tets_s, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(nt_tet.data(), P.nt_tet, sizeof(int32_t) * 4 * nt, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(perm.data(), P.node_perm, sizeof(int32_t) * nn, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(grad.data(), P.tet_grad, sizeof(double) * 12 * nt, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(vol.data(), P.tet_vol, sizeof(double) * nt, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(nt_off.data(), P.nt_off, sizeof(int64_t) * (nn + 1), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  std::vector<int64_t> off(nn + 1, 0);
  std::vector<int32_t> col;
  std::vector<float4> w;
  std::vector<std::pair<int32_t, std::array<double, 3>>> row;
  for (int64_t i = 0; i < nn; i++) {
    row.clear();
    double V = 0;
    for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) {
      const int64_t t = nt_tet[e];
      V += vol[t];
      for (int k = 0; k < 4; k++) {
        const int32_t j = tets[4 * t + k];
        auto it = std::find_if(row.begin(), row.end(), [&](const auto& x) { return x.first == j; });
        if (it == row.end()) {
          row.push_back({j, {0.0, 0.0, 0.0}});
          it = row.end() - 1;
        }
        for (int d = 0; d < 3; d++) it->second[d] += vol[t] * grad[12 * t + 3 * k + d];
      }
    }
    std::sort(row.begin(), row.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
    if (V > 0)
      for (auto& x : row) {
        col.push_back(x.first);
        w.push_back(make_float4((float)(-x.second[0] / V), (float)(-x.second[1] / V), (float)(-x.second[2] / V), 0.f));
      }
    off[i + 1] = (int64_t)col.size();
  }
  std::vector<int32_t> iperm(nn);
  for (int64_t i = 0; i < nn; i++) iperm[perm[i]] = (int32_t)i;
  P.hg_off = dalloc<int64_t>(P, nn + 1);
  P.hg_col = dalloc<int32_t>(P, std::max<size_t>(col.size(), 1));
  P.hg_w = dalloc<float4>(P, std::max<size_t>(w.size(), 1));
  P.node_iperm = dalloc<int32_t>(P, nn);
  DM_CUDA(cudaMemcpyAsync(P.hg_off, off.data(), sizeof(int64_t) * (nn + 1), cudaMemcpyHostToDevice, s));
  if (!col.empty()) {
    DM_CUDA(cudaMemcpyAsync(P.hg_col, col.data(), sizeof(int32_t) * col.size(), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.hg_w, w.data(), sizeof(float4) * w.size(), cudaMemcpyHostToDevice, s));
  }
  DM_CUDA(cudaMemcpyAsync(P.node_iperm, iperm.data(), sizeof(int32_t) * nn, cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaStreamSynchronize(s));
}

// cells with children, level by level (the M2M and L2L launches run over these only)
static void build_parent_lists(Plan& P) {
  cudaStream_t s = P.stream;
  std::vector<int32_t> nch(P.ncells), list;
  DM_CUDA(cudaMemcpyAsync(nch.data(), P.cell_nchild, sizeof(int32_t) * P.ncells, cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  P.par_start.assign(1, 0);
  for (int l = 0; l < P.nlevels; l++) {
    for (int64_t c = P.level_start[l]; c < P.level_start[l + 1]; c++)
      if (nch[c] > 0) list.push_back((int32_t)c);
    P.par_start.push_back((int64_t)list.size());
  }
  P.par_list = dalloc<int32_t>(P, std::max<size_t>(list.size(), 1));
  if (!list.empty())
    DM_CUDA(cudaMemcpyAsync(P.par_list, list.data(), sizeof(int32_t) * list.size(), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaStreamSynchronize(s));
}

void build_mixed_operators(Plan& P) {
  build_translations(P);
  build_gradient_operator(P);
  build_parent_lists(P);
  cudaStream_t s = P.stream;
  P.Ghat32 = dalloc<float>(P, std::max<int64_t>(P.n_sup, 1) * P.nc1);
  if (!P.h_src_leaves.empty()) {
    k_ghat32<<<(unsigned)P.h_src_leaves.size(), 128, 0, s>>>(P.src_leaves, P.cell_level, P.sup_off, P.Ghat, P.side,
                                                             P.nc1, P.Ghat32);
    DM_LAUNCH("k_ghat32");
  }
  if (P.n_m2l > 0) {
    const M2lKeys K = build_m2l_keys(P);
    build_m2l_tc(P, K);
    build_m2l_tab(P, K);
  }
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
  const int nc = P.nc;
  StageClock clk(P, s, profile_ok);
  clk.begin(DEMAG_STAGE_GATHER);
  k_gather_M32<<<dim3((unsigned)P.nn, (unsigned)((B + 127) / 128)), 128, 0, s>>>(P.nn, B, P.node_perm, Md, W.Ms32,
                                                                                 otf ? W.Ms : nullptr);
  DM_LAUNCH("k_gather_M32");
  clk.launched();
  clk.end();
  clk.begin(DEMAG_STAGE_P2M);
  DM_CUDA(cudaMemsetAsync(W.Q32, 0, sizeof(float) * P.ncells * nc * B, s));
  if (!P.h_src_leaves.empty()) {
    dim3 grid((unsigned)P.h_src_leaves.size(), (unsigned)((nc + P2M_NN - 1) / P2M_NN),
              (unsigned)((B + P2M_B - 1) / P2M_B));
    if (B > P2M_B) {  // two states per thread
      smem_opt_in((const void*)k_p2m32<2>, p2m_smem<2>());
      grid.z = (unsigned)((B + 2 * P2M_B - 1) / (2 * P2M_B));
      k_p2m32<2><<<grid, P2M_B, p2m_smem<2>(), s>>>(P.src_leaves, P.sup_off, P.sup_node, P.Ghat32, W.Ms32, nc, P.nc1,
                                                     B, W.Q32);
    } else {
      smem_opt_in((const void*)k_p2m32<1>, p2m_smem<1>());
      k_p2m32<1><<<grid, P2M_B, p2m_smem<1>(), s>>>(P.src_leaves, P.sup_off, P.sup_node, P.Ghat32, W.Ms32, nc, P.nc1,
                                                     B, W.Q32);
    }
    DM_LAUNCH("k_p2m32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_M2M);
  for (int l = P.nlevels - 2; l >= 0; l--) {
    const int64_t pb = P.par_start[l], np = P.par_start[l + 1] - pb;
    if (np == 0) continue;
    k_m2m32<<<nblk(np * nc * B, 256), 256, 0, s>>>(P.par_list + pb, np, P.cell_child0, P.cell_nchild, P.cell_prefix,
                                                   P.m2m_eoff, P.m2m_ent, nc, B, W.Q32);
    DM_LAUNCH("k_m2m32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_M2L);
  DM_CUDA(cudaMemsetAsync(W.L32, 0, sizeof(float) * P.ncells * nc * B, s));
  const bool tc_prec = P.opt.precision == DEMAG_MIXED_TF32 || P.opt.precision == DEMAG_MIXED_BF16X3 ||
                       P.opt.precision == DEMAG_MIXED_BF16X6;
  if (P.h_m2l_targets.empty()) {
  } else if (tc_prec && B > m2l_table_batch(P) && launch_m2l_tc(P, B, W.Q32, W.QP, W.L32, W.err, s)) {
    clk.launched(2);
  } else if ((!tc_prec || B <= m2l_table_batch(P)) && launch_m2l32_tab(P, B, W.Q32, W.L32, s)) {
    clk.launched();
  } else {
    launch_m2l32_fast(P, B, W.Q32, W.L32, W.err, s);  // orders without a derivative table
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_L2L);
  for (int l = 0; l + 1 < P.nlevels; l++) {  // parents at level l, children at l + 1
    const int64_t pb = P.par_start[l], np = P.par_start[l + 1] - pb;
    if (np == 0) continue;
    k_l2l32<<<nblk(np * nc * B, 256), 256, 0, s>>>(P.par_list + pb, np, P.cell_child0, P.cell_nchild, P.cell_range,
                                                   P.cell_prefix, P.l2l_eoff, P.l2l_ent, nc, B, W.L32);
    DM_LAUNCH("k_l2l32");
    clk.launched();
  }
  clk.end();
  clk.begin(DEMAG_STAGE_L2P);
  launch_l2p32(P, B, W.L32, W.u32, s);
  clk.launched();
  clk.end();
  if (otf) {
    k_u32_to_64<<<nblk(P.nn * B, 256), 256, 0, s>>>(P.nn * B, W.u32, W.u_s);
    DM_LAUNCH("k_u32_to_64");
    near_field_fp64(P, W, B, clk, s);
  } else {
    clk.begin(DEMAG_STAGE_P2P);
    if (P.nf_W) {
      launch_near_tc(P, W.Ms32, W.MP, B, W.u32, W.err, s);
      clk.launched();
    } else if (!P.h_p2p_targets.empty()) {
      launch_near_apply32(P, W.Ms32, B, W.u32, W.err, s);
      clk.launched();
    }
    clk.end();
  }
  clk.begin(DEMAG_STAGE_H);
  if (otf) {
    launch_lumped_H_out(P, B, W.u_s, ud, Hd, s);  // FP64 near field: u in FP64
  } else {
    k_out32<<<dim3((unsigned)((P.nn + 31) / 32), (unsigned)((B + 31) / 32)), 256, 0, s>>>(
        P.nn, B, P.node_iperm, P.hg_off, P.hg_col, P.hg_w, W.u32, ud, Hd);
    DM_LAUNCH("k_out32");
  }
  clk.launched();
  clk.end();
  clk.finish();
  eval_io_end(P, W, dev, B, u, H, s);
}

}  // namespace demag
