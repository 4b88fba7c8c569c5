// p2p.cu -- near field (Sec. 2.1): per-tet geometry, per-state records and
// the FP64 on-the-fly P2P kernel.
//
// P2P kernel layout: one warp per target leaf (blockIdx.x) and state
// (blockIdx.y).  The source tets of each P2P source leaf are contiguous in
// sorted tet order; chunks of up to 32 tets (their 66-double geometry records
// and 56-double state records) are staged in shared memory by TMA bulk copies
// (cp.async.bulk, completion on an mbarrier).  Lanes take (target node,
// source tet) pairs; each lane keeps a private partial sum per target node in
// shared memory and the partials are combined with warp shuffles.
#include "common.cuh"
#include "p2p.cuh"

namespace demag {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t > 0 ? (n + t - 1) / t : 1); }

// ---------------------------------------------------------------------------
// per-tet geometry (plan time)
// ---------------------------------------------------------------------------
__global__ void k_tet_geometry(int64_t nt, const double* __restrict__ nodes_s, int32_t* tets_s, double* geo,
                               double* grad, double* vol) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  int32_t g[4];
  double v[4][3];
  for (int k = 0; k < 4; k++) {
    g[k] = tets_s[4 * j + k];
    for (int c = 0; c < 3; c++) v[k][c] = nodes_s[3 * (int64_t)g[k] + c];
  }
  double e1[3], e2[3], e3[3];
  for (int c = 0; c < 3; c++) {
    e1[c] = v[1][c] - v[0][c];
    e2[c] = v[2][c] - v[0][c];
    e3[c] = v[3][c] - v[0][c];
  }
  double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2], e2[0] * e3[1] - e2[1] * e3[0]};
  double det = e1[0] * c23[0] + e1[1] * c23[1] + e1[2] * c23[2];
  if (det < 0) {  // store positively oriented: swap vertices 2 and 3
    int32_t t = g[2];
    g[2] = g[3];
    g[3] = t;
    tets_s[4 * j + 2] = g[2];
    tets_s[4 * j + 3] = g[3];
    for (int c = 0; c < 3; c++) {
      double x = v[2][c];
      v[2][c] = v[3][c];
      v[3][c] = x;
      x = e2[c];
      e2[c] = e3[c];
      e3[c] = x;
    }
    det = -det;
    c23[0] = e2[1] * e3[2] - e2[2] * e3[1];
    c23[1] = e2[2] * e3[0] - e2[0] * e3[2];
    c23[2] = e2[0] * e3[1] - e2[1] * e3[0];
  }
  double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2], e3[0] * e1[1] - e3[1] * e1[0]};
  double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  double inv = 1.0 / det;
  double* gr = grad + 12 * j;
  for (int c = 0; c < 3; c++) {
    gr[3 + c] = c23[c] * inv;
    gr[6 + c] = c31[c] * inv;
    gr[9 + c] = c12[c] * inv;
    gr[c] = -(gr[3 + c] + gr[6 + c] + gr[9 + c]);
  }
  vol[j] = det / 6.0;
  double* G = geo + (int64_t)TET_GEO * j;
  for (int k = 0; k < 4; k++)
    for (int c = 0; c < 3; c++) G[3 * k + c] = v[k][c];
  for (int F = 0; F < 4; F++) {
    int p = face_vertex(F, 0), q = face_vertex(F, 1), s = face_vertex(F, 2);
    double u1[3], u2[3];
    for (int c = 0; c < 3; c++) {
      u1[c] = v[q][c] - v[p][c];
      u2[c] = v[s][c] - v[p][c];
    }
    double n[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2], u1[0] * u2[1] - u1[1] * u2[0]};
    double ln = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int c = 0; c < 3; c++) n[c] /= ln;
    for (int c = 0; c < 3; c++) G[12 + 3 * F + c] = n[c];
    for (int e = 0; e < 3; e++) {
      int a0 = face_vertex(F, e), a1 = face_vertex(F, (e + 1) % 3);
      double t[3];
      for (int c = 0; c < 3; c++) t[c] = v[a1][c] - v[a0][c];
      double lt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2]);
      for (int c = 0; c < 3; c++) t[c] /= lt;
      double m[3] = {t[1] * n[2] - t[2] * n[1], t[2] * n[0] - t[0] * n[2], t[0] * n[1] - t[1] * n[0]};
      for (int c = 0; c < 3; c++) G[24 + 9 * F + 3 * e + c] = m[c];
    }
  }
  for (int e = 0; e < 6; e++) {
    int a0 = edge_v0(e), a1 = edge_v1(e);
    double dx = v[a1][0] - v[a0][0], dy = v[a1][1] - v[a0][1], dz = v[a1][2] - v[a0][2];
    G[60 + e] = sqrt(dx * dx + dy * dy + dz * dz);
  }
}

void build_tet_geometry(Plan& P) {
  P.tet_geo = dalloc<double>(P, (size_t)TET_GEO * P.nt);
  P.tet_grad = dalloc<double>(P, 12 * (size_t)P.nt);
  P.tet_vol = dalloc<double>(P, P.nt);
  k_tet_geometry<<<nblk(P.nt, 128), 128, 0, P.stream>>>(P.nt, P.nodes_s, P.tets_s, P.tet_geo, P.tet_grad, P.tet_vol);
  DM_LAUNCH("k_tet_geometry");
}

// ---------------------------------------------------------------------------
// per-tet, per-state record: M(v0), J = dM/dx and the r-independent
// contractions of the symmetric part Js of J used by pair_contract
// ---------------------------------------------------------------------------
__global__ void k_tet_state(int64_t nt, int B, const int32_t* __restrict__ tets_s, const double* __restrict__ geo,
                            const double* __restrict__ grad, const double* __restrict__ Ms, double* state) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int b = blockIdx.y;
  if (j >= nt) return;
  double Mk[4][3];
  for (int k = 0; k < 4; k++) {
    int64_t g = tets_s[4 * j + k];
    for (int c = 0; c < 3; c++) Mk[k][c] = Ms[(g * 3 + c) * B + b];
  }
  const double* gr = grad + 12 * j;
  double J[3][3];
  for (int x = 0; x < 3; x++)
    for (int y = 0; y < 3; y++) J[x][y] = Mk[0][x] * gr[y] + Mk[1][x] * gr[3 + y] + Mk[2][x] * gr[6 + y] + Mk[3][x] * gr[9 + y];
  double Js[3][3];
  for (int x = 0; x < 3; x++)
    for (int y = 0; y < 3; y++) Js[x][y] = 0.5 * (J[x][y] + J[y][x]);
  double* st = state + ((int64_t)b * nt + j) * TET_STATE;
  const double* G = geo + (int64_t)TET_GEO * j;
  for (int c = 0; c < 3; c++) st[c] = Mk[0][c];
  for (int x = 0; x < 3; x++)
    for (int y = 0; y < 3; y++) st[3 + 3 * x + y] = J[x][y];
  double trJ = J[0][0] + J[1][1] + J[2][2];
  for (int F = 0; F < 4; F++) {
    const double* n = G + 12 + 3 * F;
    double Jn[3];
    for (int x = 0; x < 3; x++) Jn[x] = Js[x][0] * n[0] + Js[x][1] * n[1] + Js[x][2] * n[2];
    double nJn = n[0] * Jn[0] + n[1] * Jn[1] + n[2] * Jn[2];
    st[48 + F] = trJ - nJn;
    st[52 + F] = nJn;
    for (int e = 0; e < 3; e++) {
      const double* m = G + 24 + 9 * F + 3 * e;
      double t[3] = {n[1] * m[2] - n[2] * m[1], n[2] * m[0] - n[0] * m[2], n[0] * m[1] - n[1] * m[0]};
      double Jm[3];
      for (int x = 0; x < 3; x++) Jm[x] = Js[x][0] * m[0] + Js[x][1] * m[1] + Js[x][2] * m[2];
      st[12 + 3 * F + e] = m[0] * Jm[0] + m[1] * Jm[1] + m[2] * Jm[2];
      st[24 + 3 * F + e] = t[0] * Jm[0] + t[1] * Jm[1] + t[2] * Jm[2];
      st[36 + 3 * F + e] = m[0] * Jn[0] + m[1] * Jn[1] + m[2] * Jn[2];
    }
  }
}

void launch_tet_state(Plan& P, const double* Ms, int B, double* state, cudaStream_t s) {
  dim3 grid(nblk(P.nt, 128), B);
  k_tet_state<<<grid, 128, 0, s>>>(P.nt, B, P.tets_s, P.tet_geo, P.tet_grad, Ms, state);
  DM_LAUNCH("k_tet_state");
}

// ---------------------------------------------------------------------------
// TMA bulk copy + mbarrier helpers (sm_90+ PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait: false if the barrier phase did not complete in time
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (long it = 0; it < (1l << 24); it++) {
    if (mbar_try_wait(bar, phase)) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

// ---------------------------------------------------------------------------
// FP64 on-the-fly P2P: one warp per (target leaf, state)
// ---------------------------------------------------------------------------
constexpr int P2P_CHUNK = 32;

__global__ void __launch_bounds__(32) k_p2p_fp64(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                                                 const int64_t* __restrict__ p2p_off,
                                                 const int32_t* __restrict__ p2p_src,
                                                 const double* __restrict__ nodes_s, const double* __restrict__ geo,
                                                 const double* __restrict__ state, int64_t nt, int B, double* u_s,
                                                 int* err) {
  __shared__ __align__(128) double s_geo[P2P_CHUNK * TET_GEO];
  __shared__ __align__(128) double s_st[P2P_CHUNK * TET_STATE];
  __shared__ double s_part[32][33];
  __shared__ __align__(8) uint64_t bar;
  const int lane = threadIdx.x;
  const int b = blockIdx.y;
  const int32_t T = targets[blockIdx.x];
  const int4 rT = range[T];
  if (lane == 0) mbar_init(&bar, 1);
  __syncwarp();
  uint32_t phase = 0;
  const double* st_b = state + (int64_t)b * nt * TET_STATE;
  for (int32_t i0 = rT.z; i0 < rT.w; i0 += 32) {  // chunks of 32 target nodes
    const int ntg = min(32, rT.w - i0);
    for (int i = 0; i < ntg; i++) s_part[i][lane] = 0.0;
    for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
      const int4 rS = range[p2p_src[e]];
      for (int32_t j0 = rS.x; j0 < rS.y; j0 += P2P_CHUNK) {
        const int ns = min(P2P_CHUNK, rS.y - j0);
        __syncwarp();
        if (lane == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          uint32_t bg = (uint32_t)(ns * TET_GEO * sizeof(double)), bs = (uint32_t)(ns * TET_STATE * sizeof(double));
          mbar_expect_tx(&bar, bg + bs);
          tma_bulk_g2s(s_geo, geo + (int64_t)j0 * TET_GEO, bg, &bar);
          tma_bulk_g2s(s_st, st_b + (int64_t)j0 * TET_STATE, bs, &bar);
        }
        if (!mbar_wait_bounded(&bar, phase)) {
          if (lane == 0) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
          mbar_wait_bounded(&bar, phase);  // let the copies in flight land before leaving
          return;
        }
        phase ^= 1;
        const int npair = ntg * ns;
        for (int q = lane; q < npair; q += 32) {
          const int i = q / ns, t = q - i * ns;
          const double* r = nodes_s + 3ll * (i0 + i);
          s_part[i][lane] += pair_contract(s_geo + t * TET_GEO, s_st + t * TET_STATE, r[0], r[1], r[2]);
        }
      }
    }
    __syncwarp();
    for (int i = 0; i < ntg; i++) {
      double v = s_part[i][lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) u_s[(int64_t)(i0 + i) * B + b] += v * (1.0 / (4.0 * M_PI));
    }
    __syncwarp();
  }
}

void launch_p2p_fp64(Plan& P, const double* state, int B, double* u_s, int* err, cudaStream_t s) {
  int64_t nT = (int64_t)P.h_p2p_targets.size();
  if (nT == 0) return;
  static_assert(sizeof(double) * P2P_CHUNK * TET_GEO % 16 == 0, "TMA size");
  dim3 grid((unsigned)nT, B);
  k_p2p_fp64<<<grid, 32, 0, s>>>(P.p2p_targets, P.cell_range, P.p2p_off, P.p2p_src, P.nodes_s, P.tet_geo, state,
                                 P.nt, B, u_s, err);
  DM_LAUNCH("k_p2p_fp64");
}

}  // namespace demag
