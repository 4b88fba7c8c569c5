// p2p.cu -- near field (Sec. 2.1): per-tet geometry and the FP64 on-the-fly
// P2P kernel.
//
// The source tets of each P2P source leaf are contiguous in sorted tet order;
// chunks of up to 32 tets (their 66-double geometry records) are staged in
// shared memory by bulk copies (cp.async.bulk, completion on an mbarrier).
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

constexpr int P2P_CHUNK = 32;

// ---------------------------------------------------------------------------
// FP64 on-the-fly P2P, one state at a time: one warp per (target leaf, state);
// lanes take (target node, source tet) pairs and contract the pair with the
// state's per-tet record (pair_contract)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32) k_p2p_fp64_state(const int32_t* __restrict__ targets, const int4* __restrict__ range,
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

// ---------------------------------------------------------------------------
// FP64 on-the-fly P2P, state-batched: one block of 4 warps per (target leaf,
// slice of FS states).  The state-independent part of every (target, tet)
// pair -- the vector a and the symmetric tensor T of the W-form (p2p.cuh) --
// is computed once and contracted with each state of the slice (16 states):
//     sum_k M_k . W_k = M(r) . a + (1/2) T : J,   J = dM/dx,  M(r) = M(v0) + J (r - v0).
// Chunks of 32 source tets: their geometry records are staged by a bulk copy,
// their per-state M(v0) and J (12 numbers) computed once by the block.  Warp w
// takes the target nodes w, w + 4, ... of the leaf, lane = tet of the chunk;
// the 32 lanes' terms are added by a fixed shuffle tree and then, by the
// warp that owns the target, into its shared-memory sum: no atomics, the
// result does not depend on timing.
// ---------------------------------------------------------------------------
constexpr int PA_FS = 16, PA_WARPS = 4, PA_NT = 64;  // states per block, warps, target nodes per pass
// dynamic shared memory: geometry records, per-state M(v0) and J of a chunk, per-target sums
constexpr size_t PA_SMEM = sizeof(double) * (P2P_CHUNK * (TET_GEO + PA_FS * 12) + PA_NT * PA_FS);

__global__ void __launch_bounds__(PA_WARPS * 32) k_p2p_fp64(
    const int32_t* __restrict__ targets, const int4* __restrict__ range, const int64_t* __restrict__ p2p_off,
    const int32_t* __restrict__ p2p_src, const double* __restrict__ nodes_s, const int32_t* __restrict__ tets_s,
    const double* __restrict__ geo, const double* __restrict__ grad, const double* __restrict__ Ms, int B,
    double* u_s, int* err) {
  extern __shared__ __align__(128) double pa_smem[];
  double* s_geo = pa_smem;                                                   // [tet][TET_GEO]
  double(*s_mj)[PA_FS][12] = (double(*)[PA_FS][12])(pa_smem + P2P_CHUNK * TET_GEO);  // M(v0) (3), J (9)
  double(*s_sum)[PA_FS] = (double(*)[PA_FS])(pa_smem + P2P_CHUNK * (TET_GEO + PA_FS * 12));
  __shared__ __align__(8) uint64_t bar;
  __shared__ bool s_ok;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int b0 = blockIdx.y * PA_FS;
  const int32_t T = targets[blockIdx.x];
  const int4 rT = range[T];
  if (tid == 0) mbar_init(&bar, 1);
  __syncthreads();
  uint32_t phase = 0;
  for (int32_t i0 = rT.z; i0 < rT.w; i0 += PA_NT) {  // passes of up to PA_NT target nodes
    const int ntg = min(PA_NT, rT.w - i0);
    for (int q = tid; q < PA_NT * PA_FS; q += blockDim.x) s_sum[q / PA_FS][q % PA_FS] = 0.0;
    for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
      const int4 rS = range[p2p_src[e]];
      for (int32_t j0 = rS.x; j0 < rS.y; j0 += P2P_CHUNK) {
        const int ns = min(P2P_CHUNK, rS.y - j0);
        __syncthreads();  // the previous chunk is no longer read
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          const uint32_t bg = (uint32_t)(ns * TET_GEO * sizeof(double));
          mbar_expect_tx(&bar, bg);
          tma_bulk_g2s(s_geo, geo + (int64_t)j0 * TET_GEO, bg, &bar);
        }
        // per tet and state: M(v0) and J = sum_k M_k (x) grad lambda_k
        for (int q = tid; q < ns * PA_FS; q += blockDim.x) {
          const int t = q / PA_FS, f = q - t * PA_FS, b = b0 + f;
          const int32_t* tv = tets_s + 4ll * (j0 + t);
          const double* g = grad + 12ll * (j0 + t);
          double mj[12] = {};
          if (b < B) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
              const int64_t node = tv[k];
              const double mx = Ms[(node * 3 + 0) * B + b], my = Ms[(node * 3 + 1) * B + b],
                           mz = Ms[(node * 3 + 2) * B + b];
              if (k == 0) {
                mj[0] = mx;
                mj[1] = my;
                mj[2] = mz;
              }
              const double m3[3] = {mx, my, mz};
#pragma unroll
              for (int x = 0; x < 3; x++)
#pragma unroll
                for (int y = 0; y < 3; y++) mj[3 + 3 * x + y] += m3[x] * g[3 * k + y];
            }
          }
#pragma unroll
          for (int c = 0; c < 12; c++) s_mj[t][f][c] = mj[c];
        }
        if (tid == 0) {
          const bool ok = mbar_wait_bounded(&bar, phase);
          if (!ok) {
            atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
            mbar_wait_bounded(&bar, phase);  // let the copy in flight land before leaving
          }
          s_ok = ok;
        }
        phase ^= 1;
        __syncthreads();  // s_geo landed (seen by thread 0), s_mj complete
        if (!s_ok) return;  // the whole block leaves together
        for (int i = warp; i < ntg; i += PA_WARPS) {
          const double* r = nodes_s + 3ll * (i0 + i);
          double acc[PA_FS];
#pragma unroll
          for (int f = 0; f < PA_FS; f++) acc[f] = 0.0;
          if (lane < ns) {
            const double* G = s_geo + lane * TET_GEO;
            PairAT at;
            pair_at(G, r[0], r[1], r[2], at);
            const double d0 = r[0] - G[0], d1 = r[1] - G[1], d2 = r[2] - G[2];
#pragma unroll
            for (int f = 0; f < PA_FS; f++) {
              const double* mj = s_mj[lane][f];
              const double* J = mj + 3;
              const double Mr0 = mj[0] + J[0] * d0 + J[1] * d1 + J[2] * d2;
              const double Mr1 = mj[1] + J[3] * d0 + J[4] * d1 + J[5] * d2;
              const double Mr2 = mj[2] + J[6] * d0 + J[7] * d1 + J[8] * d2;
              const double TJ = at.T[0] * J[0] + at.T[1] * J[4] + at.T[2] * J[8] + at.T[3] * (J[1] + J[3]) +
                                at.T[4] * (J[2] + J[6]) + at.T[5] * (J[5] + J[7]);
              acc[f] = Mr0 * at.a[0] + Mr1 * at.a[1] + Mr2 * at.a[2] + 0.5 * TJ;
            }
          }
#pragma unroll
          for (int f = 0; f < PA_FS; f++) {
            double v = acc[f];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) s_sum[i][f] += v;
          }
        }
      }
    }
    __syncthreads();
    for (int q = tid; q < ntg * PA_FS; q += blockDim.x) {
      const int i = q / PA_FS, f = q - i * PA_FS;
      if (b0 + f < B) u_s[(int64_t)(i0 + i) * B + b0 + f] += s_sum[i][f] * (1.0 / (4.0 * M_PI));
    }
    __syncthreads();  // s_sum is read before the next pass clears it
  }
}

void launch_p2p_fp64(Plan& P, const double* Ms, const double* state, int B, double* u_s, int* err, cudaStream_t s) {
  const int64_t nT = (int64_t)P.h_p2p_targets.size();
  if (nT == 0) return;
  static_assert(sizeof(double) * TET_GEO % 16 == 0 && sizeof(double) * TET_STATE % 16 == 0,
                "bulk copies of whole records");
  if (B < P2P_AT_MIN_B) {
    k_p2p_fp64_state<<<dim3((unsigned)nT, B), 32, 0, s>>>(P.p2p_targets, P.cell_range, P.p2p_off, P.p2p_src,
                                                          P.nodes_s, P.tet_geo, state, P.nt, B, u_s, err);
    DM_LAUNCH("k_p2p_fp64_state");
    return;
  }
  smem_opt_in((const void*)k_p2p_fp64, PA_SMEM);
  const dim3 grid((unsigned)nT, (unsigned)((B + PA_FS - 1) / PA_FS));
  k_p2p_fp64<<<grid, PA_WARPS * 32, PA_SMEM, s>>>(P.p2p_targets, P.cell_range, P.p2p_off, P.p2p_src, P.nodes_s,
                                             P.tets_s, P.tet_geo, P.tet_grad, Ms, B, u_s, err);
  DM_LAUNCH("k_p2p_fp64");
}


}  // namespace demag
