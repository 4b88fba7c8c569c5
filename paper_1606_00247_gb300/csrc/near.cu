// near.cu -- precomputed near field (near_mode = 1).
//
// Sec. 3.4 of the paper stores the direct-interaction coefficients instead of
// recomputing them.  Here, per P2P target leaf T, the columns are the unique
// nodes j of the tets of T's P2P source leaves, and
//     W[j][i][c] = 1/(4 pi) sum_{t in near(T), t ni j} int_t lambda_j(r') (r_i - r')_c / |r_i - r'|^3 dV'
// for every node i of T, so that u_near(r_i) = sum_j W[j][i] . M_j.  The
// integrals are the FP64 analytic pair integrals of p2p.cuh (W-form:
// W_k = lambda_k(r) a + T g_k / 2), computed once at plan time.  At every
// evaluation the near field is then a block-sparse product with the nodal M
// of all B states (FP64 for the FP64 path, FP32 for the mixed paths).
#include <cub/cub.cuh>
#include <cuda_bf16.h>

#include <algorithm>
#include <memory>

#include "common.cuh"
#include "p2p.cuh"

namespace demag {

namespace {

template <class T>
struct Tmp {
  T* p = nullptr;
  explicit Tmp(size_t n) {
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "near-field temporary allocation failed");
    }
  }
  ~Tmp() {
    if (p) cudaFree(p);
  }
};

__global__ void k_near_keys(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                            const int64_t* __restrict__ p2p_off, const int32_t* __restrict__ p2p_src,
                            const int32_t* __restrict__ tets_s, const int64_t* __restrict__ key_off, bool dipoles,
                            uint64_t* keys) {
  const int64_t ti = blockIdx.x;
  const int32_t T = targets[ti];
  int64_t o = key_off[ti];
  for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
    const int4 r = range[p2p_src[e]];
    if (dipoles) {  // the source leaf's own nodes
      const int64_t n = r.w - r.z;
      for (int64_t q = threadIdx.x; q < n; q += blockDim.x) keys[o + q] = ((uint64_t)ti << 32) | (uint32_t)(r.z + q);
      o += n;
    } else {  // the vertices of the source leaf's tets
      const int64_t n = 4ll * (r.y - r.x);
      for (int64_t q = threadIdx.x; q < n; q += blockDim.x)
        keys[o + q] = ((uint64_t)ti << 32) | (uint32_t)tets_s[4ll * r.x + q];
      o += n;
    }
  }
}

// point-dipole near field: W[col j][target i] = V_j (r_i - r_j) / (4 pi |r_i - r_j|^3), 0 for i = j
// (one block per target leaf; every (i, j) pair is written once)
__global__ void __launch_bounds__(128) k_near_build_dipole(const int32_t* __restrict__ targets,
                                                           const int4* __restrict__ range,
                                                           const int64_t* __restrict__ p2p_off,
                                                           const int32_t* __restrict__ p2p_src,
                                                           const double* __restrict__ nodes_s,
                                                           const double* __restrict__ V,
                                                           const int64_t* __restrict__ coloff,
                                                           const int32_t* __restrict__ cols,
                                                           const int64_t* __restrict__ woff, double* W) {
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], ncol = coloff[ti + 1] - c0;
  double* Wt = W + woff[ti];
  const double inv4pi = 1.0 / (4.0 * M_PI);
  for (int64_t e = p2p_off[targets[ti]]; e < p2p_off[targets[ti] + 1]; e++) {
    const int4 rS = range[p2p_src[e]];
    const int64_t nS = rS.w - rS.z;
    for (int64_t q = threadIdx.x; q < nS * nT; q += blockDim.x) {
      const int32_t j = rS.z + (int32_t)(q / nT);
      const int i = (int)(q % nT), gi = rT.z + i;
      if (gi == j) continue;
      int64_t lo = 0, hi = ncol;  // column of node j
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cols[c0 + mid] < j)
          lo = mid + 1;
        else
          hi = mid;
      }
      const double d0 = nodes_s[3 * gi] - nodes_s[3 * j], d1 = nodes_s[3 * gi + 1] - nodes_s[3 * j + 1],
                   d2 = nodes_s[3 * gi + 2] - nodes_s[3 * j + 2];
      const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
      const double f = V[j] * inv4pi / (r2 * sqrt(r2));
      double* dst = Wt + (lo * nT + i) * 3;
      dst[0] = f * d0;
      dst[1] = f * d1;
      dst[2] = f * d2;
    }
  }
}

// vertex-patch near field: W[col j][target i] = 1/(4 pi) sum_{t ni j} int_t lambda_j(r') (r_i - r') / |r_i - r'|^3 dV'
// over every tet around each own node j of the P2P source leaves (one block per
// target leaf; (target, tet around j) pairs over threads; a tet around several
// source nodes is integrated once per node).  W holds 64-bit integers in units
// of 1 / fix while it is being built (see k_fixed_to_double).
__global__ void __launch_bounds__(128) k_near_build_patch(
    const int32_t* __restrict__ targets, const int4* __restrict__ range, const int64_t* __restrict__ p2p_off,
    const int32_t* __restrict__ p2p_src, const double* __restrict__ nodes_s, const int32_t* __restrict__ tets_s,
    const double* __restrict__ geo, const double* __restrict__ grad, const int64_t* __restrict__ nt_off,
    const int32_t* __restrict__ nt_tet, const int64_t* __restrict__ coloff, const int32_t* __restrict__ cols,
    const int64_t* __restrict__ woff, double fix, unsigned long long* W) {
  const int64_t ti = blockIdx.x;
  const int32_t T = targets[ti];
  const int4 rT = range[T];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], ncol = coloff[ti + 1] - c0;
  unsigned long long* Wt = W + woff[ti];
  const double scl = fix / (4.0 * M_PI);
  for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
    const int4 rS = range[p2p_src[e]];
    for (int32_t j = rS.z; j < rS.w; j++) {
      int64_t lo = 0, hi = ncol;  // column of node j
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cols[c0 + mid] < j)
          lo = mid + 1;
        else
          hi = mid;
      }
      const int64_t t0 = nt_off[j];
      const int deg = (int)(nt_off[j + 1] - t0);
      for (int q = threadIdx.x; q < nT * deg; q += blockDim.x) {
        const int i = q / deg;
        const int32_t t = nt_tet[t0 + (q - i * deg)];
        const double* r = nodes_s + 3ll * (rT.z + i);
        const double* G = geo + (int64_t)t * TET_GEO;
        PairAT at;
        pair_at(G, r[0], r[1], r[2], at);
        int k = 0;
        while (k < 3 && tets_s[4ll * t + k] != j) k++;
        const double* g = grad + 12ll * t;
        const double d0 = r[0] - G[0], d1 = r[1] - G[1], d2 = r[2] - G[2];
        const double l1 = g[3] * d0 + g[4] * d1 + g[5] * d2, l2 = g[6] * d0 + g[7] * d1 + g[8] * d2,
                     l3 = g[9] * d0 + g[10] * d1 + g[11] * d2;
        const double lam = k == 0 ? 1.0 - l1 - l2 - l3 : (k == 1 ? l1 : (k == 2 ? l2 : l3));
        const double gx = g[3 * k], gy = g[3 * k + 1], gz = g[3 * k + 2];
        const double w0 = lam * at.a[0] + 0.5 * (at.T[0] * gx + at.T[3] * gy + at.T[4] * gz);
        const double w1 = lam * at.a[1] + 0.5 * (at.T[3] * gx + at.T[1] * gy + at.T[5] * gz);
        const double w2 = lam * at.a[2] + 0.5 * (at.T[4] * gx + at.T[5] * gy + at.T[2] * gz);
        unsigned long long* dst = Wt + (lo * nT + i) * 3;
        atomicAdd(dst, (unsigned long long)__double2ll_rn(w0 * scl));
        atomicAdd(dst + 1, (unsigned long long)__double2ll_rn(w1 * scl));
        atomicAdd(dst + 2, (unsigned long long)__double2ll_rn(w2 * scl));
      }
    }
  }
}

__global__ void k_col_offsets(const uint64_t* __restrict__ keys, int64_t n, int64_t nT, int64_t* off, int32_t* cols) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c <= nT) {
    uint64_t k = (uint64_t)c << 32;
    int64_t b = 0, e = n;
    while (b < e) {
      int64_t m = (b + e) >> 1;
      if (keys[m] < k)
        b = m + 1;
      else
        e = m;
    }
    off[c] = b;
  }
  if (cols && c < n) cols[c] = (int32_t)(keys[c] & 0xffffffffu);
}

constexpr int NB_CHUNK = 32;
constexpr int NB_COLCACHE = 4096;

// one block per P2P target leaf; (target node, source tet) pairs over threads.
// W holds 64-bit integers in units of 1 / fix while it is being built (see
// k_fixed_to_double)
__global__ void __launch_bounds__(128) k_near_build(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                                                    const int64_t* __restrict__ p2p_off,
                                                    const int32_t* __restrict__ p2p_src,
                                                    const double* __restrict__ nodes_s,
                                                    const int32_t* __restrict__ tets_s,
                                                    const double* __restrict__ geo, const double* __restrict__ grad,
                                                    const int64_t* __restrict__ coloff,
                                                    const int32_t* __restrict__ cols, const int64_t* __restrict__ woff,
                                                    double fix, unsigned long long* W) {
  __shared__ double s_geo[NB_CHUNK * TET_GEO];
  __shared__ double s_grad[NB_CHUNK * 12];
  __shared__ int32_t s_node[NB_CHUNK * 4];
  __shared__ int32_t s_cols[NB_COLCACHE];
  const int64_t ti = blockIdx.x;
  const int32_t T = targets[ti];
  const int4 rT = range[T];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], ncol = coloff[ti + 1] - c0;
  const bool cached = ncol <= NB_COLCACHE;
  if (cached)
    for (int64_t q = threadIdx.x; q < ncol; q += blockDim.x) s_cols[q] = cols[c0 + q];
  const int32_t* colv = cached ? s_cols : cols + c0;
  unsigned long long* Wt = W + woff[ti];
  const double scl = fix / (4.0 * M_PI);
  for (int64_t e = p2p_off[T]; e < p2p_off[T + 1]; e++) {
    const int4 rS = range[p2p_src[e]];
    for (int32_t j0 = rS.x; j0 < rS.y; j0 += NB_CHUNK) {
      const int ns = min(NB_CHUNK, rS.y - j0);
      __syncthreads();
      for (int q = threadIdx.x; q < ns * TET_GEO; q += blockDim.x) s_geo[q] = geo[(int64_t)j0 * TET_GEO + q];
      for (int q = threadIdx.x; q < ns * 12; q += blockDim.x) s_grad[q] = grad[(int64_t)j0 * 12 + q];
      for (int q = threadIdx.x; q < ns * 4; q += blockDim.x) s_node[q] = tets_s[4ll * j0 + q];
      __syncthreads();
      for (int q = threadIdx.x; q < nT * ns; q += blockDim.x) {
        const int i = q / ns, t = q - i * ns;
        const double* r = nodes_s + 3ll * (rT.z + i);
        const double* G = s_geo + t * TET_GEO;
        PairAT at;
        pair_at(G, r[0], r[1], r[2], at);
        const double* g = s_grad + 12 * t;
        const double d0 = r[0] - G[0], d1 = r[1] - G[1], d2 = r[2] - G[2];
        double lam[4];
        lam[1] = g[3] * d0 + g[4] * d1 + g[5] * d2;
        lam[2] = g[6] * d0 + g[7] * d1 + g[8] * d2;
        lam[3] = g[9] * d0 + g[10] * d1 + g[11] * d2;
        lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
        for (int k = 0; k < 4; k++) {
          const double gx = g[3 * k], gy = g[3 * k + 1], gz = g[3 * k + 2];
          const double w0 = lam[k] * at.a[0] + 0.5 * (at.T[0] * gx + at.T[3] * gy + at.T[4] * gz);
          const double w1 = lam[k] * at.a[1] + 0.5 * (at.T[3] * gx + at.T[1] * gy + at.T[5] * gz);
          const double w2 = lam[k] * at.a[2] + 0.5 * (at.T[4] * gx + at.T[5] * gy + at.T[2] * gz);
          // column of the vertex: binary search in the sorted column list
          const int32_t node = s_node[4 * t + k];
          int64_t lo = 0, hi = ncol;
          while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (colv[mid] < node)
              lo = mid + 1;
            else
              hi = mid;
          }
          // integer sums: exact and independent of the order of the threads' additions
          unsigned long long* dst = Wt + (lo * nT + i) * 3;
          atomicAdd(dst, (unsigned long long)__double2ll_rn(w0 * scl));
          atomicAdd(dst + 1, (unsigned long long)__double2ll_rn(w1 * scl));
          atomicAdd(dst + 2, (unsigned long long)__double2ll_rn(w2 * scl));
        }
      }
    }
  }
}


// u_s[i][b] += sum_col W[col][i] . M[node(col)][.][b]; one block per target leaf
template <class T>
__global__ void k_near_apply(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                             const int64_t* __restrict__ coloff, const int32_t* __restrict__ cols,
                             const int64_t* __restrict__ woff, const T* __restrict__ W, const T* __restrict__ Ms, int B,
                             T* u_s) {
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], c1 = coloff[ti + 1];
  const T* Wt = W + woff[ti];
  for (int item = threadIdx.x; item < nT * B; item += blockDim.x) {
    const int i = item / B, b = item - i * B;
    T acc = 0;
    for (int64_t c = c0; c < c1; c++) {
      const T* w = Wt + ((c - c0) * nT + i) * 3;
      const T* m = Ms + (int64_t)cols[c] * 3 * B + b;
      acc += w[0] * m[0] + w[1] * m[B] + w[2] * m[2 * B];
    }
    u_s[(int64_t)(rT.z + i) * B + b] += acc;
  }
}

// FP32 copy in the layout of the mixed apply: [col][target node][4] (x, y, z, 0)
__global__ void k_pack_w32(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                           const int64_t* __restrict__ coloff, const int64_t* __restrict__ woff,
                           const int64_t* __restrict__ woff32, const double* __restrict__ W, float* W32) {
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int64_t nT = rT.w - rT.z, n = (coloff[ti + 1] - coloff[ti]) * nT;
  const double* src = W + woff[ti];
  float4* dst = (float4*)(W32 + woff32[ti]);
  for (int64_t q = threadIdx.x; q < n; q += blockDim.x)
    dst[q] = make_float4((float)src[3 * q], (float)src[3 * q + 1], (float)src[3 * q + 2], 0.f);
}

// ---------------------------------------------------------------------------
// TMA bulk copy + mbarrier helpers (sm_90+ PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase) {
  for (long it = 0; it < (1l << 24); it++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}

constexpr int NA_COLS = 32;  // columns per staged chunk
constexpr int NA_NT = 32;    // target nodes per pass (registers)

// u[i][b] += sum_col W[col][i] . M[node(col)][.][b]
// one block of NA_WARPS warps per (target leaf, 32-state slice); lane =
// state; warp w takes the column chunks w, w + NA_WARPS, ...; each warp stages
// its chunk of W ([col][node][4] floats, contiguous) into its own shared-memory
// area with a TMA bulk copy, gathers M of the chunk's columns (4 columns in
// flight per lane) and keeps the partial sums of all target nodes of the pass
// in registers; the warps' partials are added in shared memory at the end.
constexpr int NA_WARPS = 8;

__global__ void __launch_bounds__(NA_WARPS * 32) k_near_apply32_v2(
    const int32_t* __restrict__ targets, const int4* __restrict__ range, const int64_t* __restrict__ coloff,
    const int32_t* __restrict__ cols, const int64_t* __restrict__ woff32, const float* __restrict__ W32,
    const float* __restrict__ Ms, int B, float* u_s, int* err) {
  extern __shared__ __align__(128) float4 sWv[];  // NA_WARPS x NA_COLS x NA_NT float4
  __shared__ __align__(8) uint64_t bar[NA_WARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], ncol = coloff[ti + 1] - c0;
  const float4* Wt = (const float4*)(W32 + woff32[ti]);
  const int b = blockIdx.y * 32 + lane;
  const bool live = b < B;
  const int bb = live ? b : 0;
  float4* myW = sWv + warp * NA_COLS * NA_NT;
  float* red = (float*)sWv;  // reused for the reduction: NA_WARPS x NA_NT x 32
  if (lane == 0) mbar_init(&bar[warp]);
  __syncwarp();
  uint32_t phase = 0;
  const int nchunk = (int)((ncol + NA_COLS - 1) / NA_COLS);
  for (int i0 = 0; i0 < nT; i0 += NA_NT) {
    const int ni = min(NA_NT, nT - i0);
    float acc[NA_NT];
#pragma unroll
    for (int i = 0; i < NA_NT; i++) acc[i] = 0.f;
    for (int k = warp; k < nchunk; k += NA_WARPS) {
      const int64_t cb = (int64_t)k * NA_COLS;
      const int cc = (ncol - cb < NA_COLS) ? (int)(ncol - cb) : NA_COLS;
      __syncwarp();
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (ni == nT) {
          tma_load(myW, Wt + cb * nT, (uint32_t)(cc * nT * sizeof(float4)), &bar[warp]);
        } else {
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[warp])),
                       "r"((uint32_t)(cc * ni * sizeof(float4)))
                       : "memory");
          for (int c = 0; c < cc; c++)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    smem_u32(&myW[c * ni])),
                "l"(Wt + (cb + c) * nT + i0), "r"((uint32_t)(ni * sizeof(float4))), "r"(smem_u32(&bar[warp]))
                : "memory");
        }
      }
      if (!mbar_wait(&bar[warp], phase)) {
        if (lane == 0) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
        mbar_wait(&bar[warp], phase);
        return;
      }
      phase ^= 1;
      for (int c = 0; c < cc; c += 4) {
        float m[4][3];
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const int cu = (c + u < cc) ? c + u : c;
          const float* mp = Ms + (int64_t)cols[c0 + cb + cu] * 3 * B + bb;
          m[u][0] = mp[0];
          m[u][1] = mp[B];
          m[u][2] = mp[2 * B];
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
          if (c + u >= cc) break;
          const float4* w = myW + (c + u) * ni;
#pragma unroll
          for (int i = 0; i < NA_NT; i++)
            if (i < ni) {
              const float4 wv = w[i];
              acc[i] = fmaf(wv.x, m[u][0], fmaf(wv.y, m[u][1], fmaf(wv.z, m[u][2], acc[i])));
            }
        }
      }
    }
    // add the warps' partial sums
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NA_NT; i++)
      if (i < ni) red[(warp * NA_NT + i) * 32 + lane] = acc[i];
    __syncthreads();
    for (int i = warp; i < ni; i += NA_WARPS) {
      float v = 0.f;
      for (int w = 0; w < NA_WARPS; w++) v += red[(w * NA_NT + i) * 32 + lane];
      if (live) u_s[(int64_t)(rT.z + i0 + i) * B + b] += v;
    }
    __syncthreads();
  }
}

// Batched form for B % 4 == 0: one block of NB_WARPS warps per (target leaf,
// 128 states), so W is streamed from HBM once per evaluation.  Lane = 4
// consecutive states (float4 loads of M), 16 target nodes per pass: 64
// accumulators per lane, 12 FMAs per broadcast shared-memory read of W.  Each
// warp stages its column chunks (NB_CW columns, <= 4 KB) into two buffers with
// bulk copies, the next chunk in flight while the current one is used; the
// warps' partial sums are added in shared memory at the end of the pass.
constexpr int NB_WARPS = 8, NB_CW = 16, NB_NT = 16, NB_STATES = 128;

__global__ void __launch_bounds__(NB_WARPS * 32, 2) k_near_apply32_v3(
    const int32_t* __restrict__ targets, const int4* __restrict__ range, const int64_t* __restrict__ coloff,
    const int32_t* __restrict__ cols, const int64_t* __restrict__ woff32, const float* __restrict__ W32,
    const float* __restrict__ Ms, int B, float* u_s, int* err) {
  extern __shared__ __align__(128) float4 sW[];  // NB_WARPS x 2 x (NB_CW * NB_NT) float4; then the reduction
  __shared__ __align__(8) uint64_t bar[NB_WARPS][2];
  __shared__ int s_bad;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti], ncol = coloff[ti + 1] - c0;
  const float4* Wt = (const float4*)(W32 + woff32[ti]);
  const int bs = blockIdx.y * NB_STATES + lane * 4;
  const bool live = bs < B;
  float4* const buf0 = sW + warp * 2 * NB_CW * NB_NT;  // buffer `slot` at buf0 + slot * NB_CW * NB_NT
  if (lane == 0) {
    mbar_init(&bar[warp][0]);
    mbar_init(&bar[warp][1]);
  }
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  uint32_t phases = 0u;  // bit s: parity of buffer s
  const int nchunk = (int)((ncol + NB_CW - 1) / NB_CW);
  for (int i0 = 0; i0 < nT; i0 += NB_NT) {
    bool bad = false;
    const int ni = min(NB_NT, nT - i0);
    // lane 0 issues chunk k into buffer `slot`
    auto issue = [&](int k, int slot) {
      if (lane != 0) return;
      const int64_t cb = (int64_t)k * NB_CW;
      const int cc = (ncol - cb < NB_CW) ? (int)(ncol - cb) : NB_CW;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      if (ni == nT) {
        tma_load(buf0 + slot * NB_CW * NB_NT, Wt + cb * nT, (uint32_t)(cc * nT * sizeof(float4)), &bar[warp][slot]);
      } else {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[warp][slot])),
                     "r"((uint32_t)(cc * ni * sizeof(float4)))
                     : "memory");
        for (int c = 0; c < cc; c++)
          asm volatile(
              "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                  smem_u32(buf0 + slot * NB_CW * NB_NT + c * ni)),
              "l"(Wt + (cb + c) * nT + i0), "r"((uint32_t)(ni * sizeof(float4))), "r"(smem_u32(&bar[warp][slot]))
              : "memory");
      }
    };
    float acc[NB_NT][4];
#pragma unroll
    for (int i = 0; i < NB_NT; i++) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    int q = 0;
    // column ids of the warp's current and next chunk: lane l holds column l of the chunk
    auto chunk_cols = [&](int k) {
      const int64_t cb = (int64_t)k * NB_CW;
      return (k < nchunk && lane < NB_CW && cb + lane < ncol) ? cols[c0 + cb + lane] : 0;
    };
    int colv = chunk_cols(warp);
    if (warp < nchunk) issue(warp, 0);
    for (int k = warp; k < nchunk && !bad; k += NB_WARPS, q++) {
      const int slot = q & 1;
      __syncwarp();  // every lane is done with the other buffer before it is refilled
      if (k + NB_WARPS < nchunk) issue(k + NB_WARPS, slot ^ 1);
      const int colv_next = chunk_cols(k + NB_WARPS);
      if (!mbar_wait(&bar[warp][slot], (phases >> slot) & 1u)) {
        if (lane == 0) {
          atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
          atomicExch(&s_bad, 1);
        }
        bad = true;
        break;
      }
      phases ^= 1u << slot;
      const int64_t cb = (int64_t)k * NB_CW;
      const int cc = (ncol - cb < NB_CW) ? (int)(ncol - cb) : NB_CW;
      const float4* w = buf0 + slot * NB_CW * NB_NT;
      // M of column c is loaded while column c - 1 is applied
      float4 mx = make_float4(0.f, 0.f, 0.f, 0.f), my = mx, mz = mx;
      {
        const int col = __shfl_sync(0xffffffffu, colv, 0);
        if (live) {
          const float* mp = Ms + (int64_t)col * 3 * B + bs;
          mx = *(const float4*)mp;
          my = *(const float4*)(mp + B);
          mz = *(const float4*)(mp + 2 * B);
        }
      }
      for (int c = 0; c < cc; c++) {
        float4 nx = make_float4(0.f, 0.f, 0.f, 0.f), ny = nx, nz = nx;
        const int coln = __shfl_sync(0xffffffffu, colv, (c + 1) & 31);
        if (live && c + 1 < cc) {
          const float* mp = Ms + (int64_t)coln * 3 * B + bs;
          nx = *(const float4*)mp;
          ny = *(const float4*)(mp + B);
          nz = *(const float4*)(mp + 2 * B);
        }
        const float4* wc = w + c * ni;
#pragma unroll
        for (int i = 0; i < NB_NT; i++)
          if (i < ni) {
            const float4 wv = wc[i];
            acc[i][0] = fmaf(wv.x, mx.x, fmaf(wv.y, my.x, fmaf(wv.z, mz.x, acc[i][0])));
            acc[i][1] = fmaf(wv.x, mx.y, fmaf(wv.y, my.y, fmaf(wv.z, mz.y, acc[i][1])));
            acc[i][2] = fmaf(wv.x, mx.z, fmaf(wv.y, my.z, fmaf(wv.z, mz.z, acc[i][2])));
            acc[i][3] = fmaf(wv.x, mx.w, fmaf(wv.y, my.w, fmaf(wv.z, mz.w, acc[i][3])));
          }
        mx = nx;
        my = ny;
        mz = nz;
      }
      colv = colv_next;
    }
    if (bad && lane == 0) {
      // a wait expired: let this warp's copies in flight land (bounded) before the buffers are reused
      mbar_wait(&bar[warp][0], phases & 1u);
      mbar_wait(&bar[warp][1], (phases >> 1) & 1u);
    }
    // add the warps' partial sums: red[warp][i][128 states]
    __syncthreads();
    if (s_bad) return;  // uniform: read after the barrier
    float4* red = sW;
#pragma unroll
    for (int i = 0; i < NB_NT; i++)
      if (i < ni) red[(warp * NB_NT + i) * 32 + lane] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
    __syncthreads();
    const float* redf = (const float*)sW;
    for (int idx = threadIdx.x; idx < ni * NB_STATES; idx += blockDim.x) {
      const int i = idx / NB_STATES, sl = idx - i * NB_STATES;
      float v = 0.f;
#pragma unroll
      for (int w2 = 0; w2 < NB_WARPS; w2++) v += redf[(w2 * NB_NT + i) * NB_STATES + sl];
      const int b = blockIdx.y * NB_STATES + sl;
      if (b < B) u_s[(int64_t)(rT.z + i0 + i) * B + b] += v;
    }
    __syncthreads();
  }
}

// fixed-point coefficients -> FP64 (in place): the near-field build adds its
// per-tet contributions as 64-bit integers in units of 1 / NEAR_FIX (exact,
// order-independent sums), so the coefficients do not depend on the order in
// which the threads add them
__global__ void k_fixed_to_double(int64_t n, double* W, double inv) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const long long v = __double_as_longlong(W[q]);
    W[q] = (double)v * inv;
  }
}

// keys (tile << 32 | node) of the columns of every leaf of the chunk's tiles:
// one block per tile, the leaves' (sorted, distinct) columns concatenated
__global__ void k_nf_tile_keys(const int64_t* __restrict__ tleaf, const int64_t* __restrict__ tkoff,
                               const int64_t* __restrict__ lcoloff, const uint64_t* __restrict__ lkeys, uint64_t* out) {
  const int64_t t = blockIdx.x;
  int64_t o = tkoff[t];
  for (int64_t l = tleaf[2 * t]; l < tleaf[2 * t + 1]; l++) {
    const int64_t c0 = lcoloff[l], n = lcoloff[l + 1] - c0;
    for (int64_t q = threadIdx.x; q < n; q += blockDim.x)
      out[o + q] = ((uint64_t)t << 32) | (uint32_t)(lkeys[c0 + q] & 0xffffffffu);
    o += n;
  }
}

// columns of each tile from its sorted distinct keys, padded to groups of 16 with the last column
__global__ void k_nf_tile_cols(const uint64_t* __restrict__ keys, const int64_t* __restrict__ kofft,
                               const int64_t* __restrict__ coff, int32_t* cols) {
  const int64_t t = blockIdx.x;
  const int64_t k0 = kofft[t], n = kofft[t + 1] - k0, npad = (n + 15) / 16 * 16;
  int32_t* dst = cols + coff[t];
  for (int64_t q = threadIdx.x; q < npad; q += blockDim.x)
    dst[q] = (int32_t)(keys[k0 + (q < n ? q : n - 1)] & 0xffffffffu);
}

// split-BF16 tile coefficients from the per-leaf FP64 ones: one block per leaf;
// every (row, column, component) of a tile is written by exactly one thread
__global__ void k_nf_pack(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                          const int64_t* __restrict__ lcoloff, const int32_t* __restrict__ lcols,
                          const int64_t* __restrict__ lwoff, const double* __restrict__ W,
                          const int32_t* __restrict__ ltile, const int32_t* __restrict__ lrow0,
                          const int64_t* __restrict__ twoff, const int64_t* __restrict__ tcoff,
                          const int32_t* __restrict__ tng, const int32_t* __restrict__ tnpad,
                          const int32_t* __restrict__ tcols, unsigned char* Wtc) {
  const int64_t l = blockIdx.x;
  const int4 rT = range[targets[l]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = lcoloff[l], ncol = lcoloff[l + 1] - c0;
  const double* Wl = W + lwoff[l];
  for (int64_t q = threadIdx.x; q < ncol * nT; q += blockDim.x) {
    const int64_t c = q / nT;
    const int i = (int)(q - c * nT);
    const int rr = lrow0[l] + i;
    const int64_t t = ltile[l] + rr / NF_ROWS;
    const int r = rr % NF_ROWS;
    const int32_t node = lcols[c0 + c];
    const int32_t* tc = tcols + tcoff[t];
    int64_t lo = 0, hi = (int64_t)tng[t] * 16;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (tc[mid] < node)
        lo = mid + 1;
      else
        hi = mid;
    }
    const int npad = tnpad[t];
    unsigned char* base = Wtc + twoff[t];
    for (int comp = 0; comp < 3; comp++) {
      const double v = Wl[(c * nT + i) * 3 + comp];
      const __nv_bfloat16 h = __float2bfloat16_rn((float)v);
      const __nv_bfloat16 s = __float2bfloat16_rn((float)(v - (double)__bfloat162float(h)));
      const int64_t ks = 3 * (lo / 16) + comp;
      const int k = (int)(lo % 16);
      unsigned char* kb = base + ks * 64 * npad + (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
      *(__nv_bfloat16*)kb = h;
      *(__nv_bfloat16*)(kb + 32 * npad) = s;
    }
  }
}

// row sums of the near-field coefficients, S_i = sum_j W_ij (FP64, columns in
// order), per sorted target node: the tensor-core near field applies W to
// M - Mbar and adds S_i . Mbar (near_tc.cu)
__global__ void k_nf_rowsum(const int32_t* __restrict__ targets, const int4* __restrict__ range,
                            const int64_t* __restrict__ lcoloff, const int64_t* __restrict__ lwoff,
                            const double* __restrict__ W, float* S) {
  const int64_t l = blockIdx.x;
  const int4 rT = range[targets[l]];
  const int nT = rT.w - rT.z;
  const int64_t ncol = lcoloff[l + 1] - lcoloff[l];
  const double* Wl = W + lwoff[l];
  for (int q = threadIdx.x; q < 3 * nT; q += blockDim.x) {
    const int i = q / 3, comp = q - 3 * i;
    double acc = 0.0;
    for (int64_t c = 0; c < ncol; c++) acc += Wl[(c * nT + i) * 3 + comp];
    S[(int64_t)(rT.z + i) * 3 + comp] = (float)acc;
  }
}

}  // namespace

// Tiles of the tensor-core near field over the P2P target leaves (already in
// order of their first node): consecutive leaves with at most NF_ROWS target
// nodes together; a leaf with more nodes gets tiles of its own, NF_ROWS rows
// each.
struct NfTiles {
  std::vector<int64_t> leaf;   // 2 per tile: its leaves [leaf0, leaf1)
  std::vector<int32_t> nrow;   // rows per tile
  std::vector<int32_t> ltile;  // per leaf: its first tile
  std::vector<int32_t> lrow0;  // per leaf: row of its first node in that tile
};

static NfTiles nf_make_tiles(const Plan& P) {
  NfTiles T;
  const int64_t nT = (int64_t)P.h_p2p_targets.size();
  T.ltile.resize(nT);
  T.lrow0.resize(nT);
  int64_t cur = -1;
  for (int64_t l = 0; l < nT; l++) {
    const int4 r = P.h_range[P.h_p2p_targets[l]];
    const int n = r.w - r.z;
    if (n > NF_ROWS) {
      T.ltile[l] = (int32_t)T.nrow.size();
      T.lrow0[l] = 0;
      for (int k = 0; k < n; k += NF_ROWS) {
        T.leaf.push_back(l);
        T.leaf.push_back(l + 1);
        T.nrow.push_back(std::min(NF_ROWS, n - k));
      }
      cur = -1;
      continue;
    }
    if (cur < 0 || T.nrow[cur] + n > NF_ROWS) {
      cur = (int64_t)T.nrow.size();
      T.leaf.push_back(l);
      T.leaf.push_back(l + 1);
      T.nrow.push_back(0);
    }
    T.leaf[2 * cur + 1] = l + 1;
    T.ltile[l] = (int32_t)cur;
    T.lrow0[l] = T.nrow[cur];
    T.nrow[cur] += n;
  }
  return T;
}

// the two-limb split precision; the three-limb one (24-bit operands) keeps the
// FP32 CUDA-core near field, whose rounding is finer than a two-limb product's
bool near_tc_wanted(const Plan& P) {
  return P.opt.near_mode == 1 && P.opt.near_tc >= 0 && P.opt.precision == DEMAG_MIXED_BF16X3;
}

// Plan-time near field, in chunks of consecutive target leaves (at most
// NEAR_KEYS_PER_CHUNK (target, source-node) candidates each; with tiles, a
// chunk ends only where a tile ends) so that large meshes never hold more than
// one chunk's keys and FP64 coefficients:
//   pass 1 -- per chunk, the distinct source nodes (columns) of every target
//             leaf, and with tiles the distinct columns of every tile;
//   pass 2 -- per chunk again, the columns, the FP64 coefficients integrated
//             (k_near_build, fixed-point sums) and, on the mixed path, packed:
//             to the FP32 per-leaf layout, or to the split-BF16 tiles of the
//             tensor-core near field.  Only the FP64 path keeps W64.
constexpr int64_t NEAR_KEYS_PER_CHUNK = int64_t(1) << 27;

void build_near_field(Plan& P) {
  cudaStream_t s = P.stream;
  const bool mixed = P.opt.precision != DEMAG_FP64, dip = P.opt.sources == DEMAG_SOURCES_DIPOLES;
  const bool patch = P.opt.sources == DEMAG_SOURCES_PATCHES;
  const bool nodesrc = dip || patch;  // columns: the source leaves' own nodes
  const bool tc = near_tc_wanted(P);
  if (tc) {  // tiles follow the Morton order of the target nodes
    std::stable_sort(P.h_p2p_targets.begin(), P.h_p2p_targets.end(),
                     [&](int32_t a, int32_t b) { return P.h_range[a].z < P.h_range[b].z; });
    DM_CUDA(cudaMemcpyAsync(P.p2p_targets, P.h_p2p_targets.data(), P.h_p2p_targets.size() * sizeof(int32_t),
                            cudaMemcpyHostToDevice, s));
  }
  const int64_t nT = (int64_t)P.h_p2p_targets.size();
  P.w_coloff = dalloc<int64_t>(P, nT + 1);
  P.w_off = dalloc<int64_t>(P, nT + 1);
  if (nT == 0) {
    DM_CUDA(cudaMemsetAsync(P.w_coloff, 0, sizeof(int64_t), s));
    DM_CUDA(cudaMemsetAsync(P.w_off, 0, sizeof(int64_t), s));
    P.w_cols = dalloc<int32_t>(P, 1);
    P.W64 = dalloc<double>(P, 1);
    if (mixed) {
      P.w_off32 = dalloc<int64_t>(P, 1);
      DM_CUDA(cudaMemsetAsync(P.w_off32, 0, sizeof(int64_t), s));
      P.W32 = dalloc<float>(P, 4);
    }
    return;
  }
  // candidate keys per target: 4 per source tet of its P2P list
  std::vector<int64_t> koff(nT + 1, 0);
  for (int64_t ti = 0; ti < nT; ti++) {
    int32_t T = P.h_p2p_targets[ti];
    int64_t n = 0;
    for (int64_t e = P.h_p2p_off[T]; e < P.h_p2p_off[T + 1]; e++) {
      int4 r = P.h_range[P.h_p2p_src[e]];
      n += nodesrc ? (int64_t)(r.w - r.z) : 4ll * (r.y - r.x);
    }
    if (n > NEAR_KEYS_PER_CHUNK) fail(DEMAG_ERR_UNSUPPORTED, "near field of one target leaf too large");
    koff[ti + 1] = koff[ti] + n;
  }
  NfTiles TL;
  if (tc) TL = nf_make_tiles(P);
  const int64_t ntiles = (int64_t)TL.nrow.size();
  auto tile_of = [&](int64_t l) -> int64_t { return l < nT ? TL.ltile[l] : ntiles; };  // first tile of leaf l
  std::vector<int64_t> chunk{0};
  for (int64_t ti = 0; ti < nT; ti++) {
    const bool may_cut = !tc || (TL.lrow0[ti] == 0 && (ti == 0 || TL.ltile[ti] != TL.ltile[ti - 1]));
    if (ti > chunk.back() && may_cut && koff[ti + 1] - koff[chunk.back()] > NEAR_KEYS_PER_CHUNK) chunk.push_back(ti);
  }
  chunk.push_back(nT);
  int64_t max_keys = 0;
  for (size_t c = 0; c + 1 < chunk.size(); c++) max_keys = std::max(max_keys, koff[chunk[c + 1]] - koff[chunk[c]]);
  Tmp<uint64_t> keys(max_keys), keys_s(max_keys);
  Tmp<int64_t> dkoff(nT + 1), doff(nT + 1);
  Tmp<int> nu(1);
  size_t tb = 0, tb2 = 0;
  cub::DeviceRadixSort::SortKeys(nullptr, tb, keys.p, keys_s.p, (int)max_keys, 0, 64, s);
  cub::DeviceSelect::Unique(nullptr, tb2, keys_s.p, keys.p, nu.p, (int)max_keys, s);
  Tmp<char> temp(std::max(tb, tb2));
  // the distinct columns of the targets [t0, t1), sorted by (target, node), in keys.p; returns their count
  auto columns = [&](int64_t t0, int64_t t1) -> int64_t {
    const int64_t nk = koff[t1] - koff[t0];
    std::vector<int64_t> rel(t1 - t0 + 1);
    for (int64_t t = t0; t <= t1; t++) rel[t - t0] = koff[t] - koff[t0];
    DM_CUDA(cudaMemcpyAsync(dkoff.p, rel.data(), rel.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_near_keys<<<(unsigned)(t1 - t0), 128, 0, s>>>(P.p2p_targets + t0, P.cell_range, P.p2p_off, P.p2p_src,
                                                     P.tets_s, dkoff.p, nodesrc, keys.p);
    DM_LAUNCH("k_near_keys");
    size_t t = tb;
    DM_CUDA(cub::DeviceRadixSort::SortKeys(temp.p, t, keys.p, keys_s.p, (int)nk, 0, 64, s));
    t = tb2;
    DM_CUDA(cub::DeviceSelect::Unique(temp.p, t, keys_s.p, keys.p, nu.p, (int)nk, s));
    int hnu = 0;
    DM_CUDA(cudaMemcpyAsync(&hnu, nu.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return hnu;
  };
  // tiles: the distinct columns of the tiles [q0, q1) of the chunk, whose leaves'
  // columns are in keys.p with chunk-relative offsets doff; returns the sorted
  // keys (tile - q0) << 32 | node and their per-tile offsets (host)
  auto tile_columns = [&](int64_t t0, int64_t q0, int64_t q1, const std::vector<int64_t>& lcnt,
                          std::vector<int64_t>& toff) -> std::unique_ptr<Tmp<uint64_t>> {
    std::vector<int64_t> tleaf(2 * (q1 - q0)), tkoff(q1 - q0 + 1, 0);
    for (int64_t q = q0; q < q1; q++) {
      tleaf[2 * (q - q0)] = TL.leaf[2 * q] - t0;
      tleaf[2 * (q - q0) + 1] = TL.leaf[2 * q + 1] - t0;
      int64_t n = 0;
      for (int64_t l = TL.leaf[2 * q]; l < TL.leaf[2 * q + 1]; l++) n += lcnt[l - t0];
      tkoff[q - q0 + 1] = tkoff[q - q0] + n;
    }
    const int64_t nk = tkoff[q1 - q0];
    Tmp<int64_t> dtleaf(tleaf.size()), dtkoff(tkoff.size());
    DM_CUDA(cudaMemcpyAsync(dtleaf.p, tleaf.data(), tleaf.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(dtkoff.p, tkoff.data(), tkoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    Tmp<uint64_t> tk(nk), tks(nk);
    std::unique_ptr<Tmp<uint64_t>> tu(new Tmp<uint64_t>(nk));
    k_nf_tile_keys<<<(unsigned)(q1 - q0), 128, 0, s>>>(dtleaf.p, dtkoff.p, doff.p, keys.p, tk.p);
    DM_LAUNCH("k_nf_tile_keys");
    size_t b1 = 0, b2 = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, b1, tk.p, tks.p, (int)nk, 0, 64, s);
    cub::DeviceSelect::Unique(nullptr, b2, tks.p, tu->p, nu.p, (int)nk, s);
    Tmp<char> tt(std::max(b1, b2));
    DM_CUDA(cub::DeviceRadixSort::SortKeys(tt.p, b1, tk.p, tks.p, (int)nk, 0, 64, s));
    DM_CUDA(cub::DeviceSelect::Unique(tt.p, b2, tks.p, tu->p, nu.p, (int)nk, s));
    int hnu = 0;
    DM_CUDA(cudaMemcpyAsync(&hnu, nu.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    Tmp<int64_t> dto(q1 - q0 + 1);
    k_col_offsets<<<(unsigned)((std::max<int64_t>(hnu, q1 - q0 + 1) + 255) / 256), 256, 0, s>>>(tu->p, hnu, q1 - q0,
                                                                                                 dto.p, nullptr);
    DM_LAUNCH("k_col_offsets(tiles)");
    toff.assign(q1 - q0 + 1, 0);
    DM_CUDA(cudaMemcpyAsync(toff.data(), dto.p, toff.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    return tu;
  };
  // pass 1: column counts per target leaf (and per tile)
  std::vector<int64_t> hcol(nT + 1, 0), tcol(ntiles, 0);
  for (size_t c = 0; c + 1 < chunk.size(); c++) {
    const int64_t t0 = chunk[c], t1 = chunk[c + 1];
    const int64_t nu_c = columns(t0, t1);
    k_col_offsets<<<(unsigned)((std::max<int64_t>(nu_c, t1 - t0 + 1) + 255) / 256), 256, 0, s>>>(
        keys.p, nu_c, t1 - t0, doff.p, nullptr);
    DM_LAUNCH("k_col_offsets");
    std::vector<int64_t> o(t1 - t0 + 1);
    DM_CUDA(cudaMemcpyAsync(o.data(), doff.p, o.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    for (int64_t t = t0; t < t1; t++) hcol[t + 1] = hcol[t0] + o[t - t0 + 1];
    if (tc) {
      std::vector<int64_t> lcnt(t1 - t0), toff;
      for (int64_t t = t0; t < t1; t++) lcnt[t - t0] = o[t - t0 + 1] - o[t - t0];
      const int64_t q0 = tile_of(t0), q1 = tile_of(t1);
      tile_columns(t0, q0, q1, lcnt, toff);
      for (int64_t q = q0; q < q1; q++) tcol[q] = toff[q - q0 + 1] - toff[q - q0];
    }
  }
  const int64_t ncols = hcol[nT];
  if (ncols > (int64_t)INT32_MAX) fail(DEMAG_ERR_UNSUPPORTED, "near field too large for the precomputed mode");
  std::vector<int64_t> hw(nT + 1, 0), hw32(nT + 1, 0);
  for (int64_t ti = 0; ti < nT; ti++) {
    int4 r = P.h_range[P.h_p2p_targets[ti]];
    hw[ti + 1] = hw[ti] + (hcol[ti + 1] - hcol[ti]) * (int64_t)(r.w - r.z) * 3;
    hw32[ti + 1] = hw32[ti] + (hcol[ti + 1] - hcol[ti]) * (int64_t)(r.w - r.z) * 4;
  }
  P.n_wcols = ncols;
  P.n_wentries = hw[nT];
  // per-leaf columns: kept by the FP64 and FP32 layouts, per chunk only for the tiles
  int64_t max_lcols = 0;
  for (size_t c = 0; c + 1 < chunk.size(); c++) max_lcols = std::max(max_lcols, hcol[chunk[c + 1]] - hcol[chunk[c]]);
  Tmp<int32_t> lcols_tmp(tc ? max_lcols : 0);
  P.w_cols = dalloc<int32_t>(P, tc ? 1 : std::max<int64_t>(ncols, 1));
  DM_CUDA(cudaMemcpyAsync(P.w_coloff, hcol.data(), (nT + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemcpyAsync(P.w_off, hw.data(), (nT + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  std::vector<int64_t> hcoff(ntiles + 1, 0), hwoff(ntiles + 1, 0);
  std::vector<int32_t> hng(ntiles), hnpad(ntiles);
  if (tc) {
    // tile shapes, row nodes and the split-BF16 coefficient array
    std::vector<int32_t> rown((size_t)std::max<int64_t>(ntiles, 1) * NF_ROWS, -1);
    for (int64_t q = 0; q < ntiles; q++) {
      hng[q] = (int32_t)((tcol[q] + 15) / 16);
      hnpad[q] = (TL.nrow[q] + 15) / 16 * 16;
      hcoff[q + 1] = hcoff[q] + 16ll * hng[q];
      hwoff[q + 1] = hwoff[q] + 3ll * hng[q] * 64 * hnpad[q];
    }
    for (int64_t l = 0; l < nT; l++) {
      const int4 r = P.h_range[P.h_p2p_targets[l]];
      for (int i = 0; i < r.w - r.z; i++) {
        const int rr = TL.lrow0[l] + i;
        rown[(size_t)(TL.ltile[l] + rr / NF_ROWS) * NF_ROWS + rr % NF_ROWS] = r.z + i;
      }
    }
    P.nf_ntiles = ntiles;
    P.nf_ncols = hcoff[ntiles];
    P.nf_wbytes = hwoff[ntiles];
    P.nf_woff = dalloc<int64_t>(P, ntiles);
    P.nf_coff = dalloc<int64_t>(P, ntiles);
    P.nf_ng = dalloc<int32_t>(P, ntiles);
    P.nf_npad = dalloc<int32_t>(P, ntiles);
    P.nf_rownode = dalloc<int32_t>(P, rown.size());
    P.nf_cols = dalloc<int32_t>(P, std::max<int64_t>(P.nf_ncols, 1));
    P.nf_W = dalloc<unsigned char>(P, std::max<int64_t>(P.nf_wbytes, 16));
    P.nf_S = dalloc<float>(P, 3 * (size_t)P.nn);
    DM_CUDA(cudaMemsetAsync(P.nf_S, 0, sizeof(float) * 3 * (size_t)P.nn, s));  // nodes in no P2P target leaf
    std::vector<int32_t> order(ntiles);
    for (int64_t q = 0; q < ntiles; q++) order[q] = (int32_t)q;
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return hng[a] > hng[b]; });
    P.nf_order = dalloc<int32_t>(P, std::max<int64_t>(ntiles, 1));
    DM_CUDA(cudaMemcpyAsync(P.nf_order, order.data(), ntiles * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.nf_woff, hwoff.data(), ntiles * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.nf_coff, hcoff.data(), ntiles * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.nf_ng, hng.data(), ntiles * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.nf_npad, hnpad.data(), ntiles * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.nf_rownode, rown.data(), rown.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemsetAsync(P.nf_W, 0, std::max<int64_t>(P.nf_wbytes, 16), s));
    DM_CUDA(cudaStreamSynchronize(s));
  } else if (mixed) {
    P.w_off32 = dalloc<int64_t>(P, nT + 1);
    DM_CUDA(cudaMemcpyAsync(P.w_off32, hw32.data(), (nT + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    P.W32 = dalloc<float>(P, std::max<int64_t>(hw32[nT], 4));
  }
  if (!mixed) P.W64 = dalloc<double>(P, std::max<int64_t>(hw[nT], 1));
  int64_t max_w = 0;
  for (size_t c = 0; c + 1 < chunk.size(); c++) max_w = std::max(max_w, hw[chunk[c + 1]] - hw[chunk[c]]);
  Tmp<double> wtmp(mixed ? max_w : 0);
  Tmp<int32_t> dltile(tc ? nT : 0), dlrow0(tc ? nT : 0);
  if (tc) {
    DM_CUDA(cudaMemcpyAsync(dltile.p, TL.ltile.data(), nT * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(dlrow0.p, TL.lrow0.data(), nT * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  const double fix = ldexp(1.0, 60) / P.side;  // |W| <= sqrt(3) side, so every partial sum fits in 63 bits
  // pass 2: columns, FP64 coefficients, FP32 or split-BF16 copy
  for (size_t c = 0; c + 1 < chunk.size(); c++) {
    const int64_t t0 = chunk[c], t1 = chunk[c + 1];
    const int64_t nu_c = columns(t0, t1);
    // per-leaf column offsets (chunk-relative in doff) and columns
    int32_t* lcols = tc ? lcols_tmp.p : P.w_cols + hcol[t0];
    k_col_offsets<<<(unsigned)((std::max<int64_t>(nu_c, t1 - t0 + 1) + 255) / 256), 256, 0, s>>>(
        keys.p, nu_c, t1 - t0, doff.p, lcols);
    DM_LAUNCH("k_col_offsets");
    std::vector<int64_t> rel(t1 - t0 + 1);
    for (int64_t t = t0; t <= t1; t++) rel[t - t0] = hcol[t] - hcol[t0];
    Tmp<int64_t> lcoloff(t1 - t0 + 1);
    DM_CUDA(cudaMemcpyAsync(lcoloff.p, rel.data(), rel.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    double* W = P.W64;
    const int64_t* woff = P.w_off + t0;
    Tmp<int64_t> wrel(t1 - t0 + 1);
    if (mixed) {  // chunk-relative offsets into the temporary FP64 block
      for (int64_t t = t0; t <= t1; t++) rel[t - t0] = hw[t] - hw[t0];
      DM_CUDA(cudaMemcpyAsync(wrel.p, rel.data(), rel.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      W = wtmp.p;
      woff = wrel.p;
    }
    const int64_t nw = std::max<int64_t>(hw[t1] - hw[t0], 1);
    double* Wc = W + (mixed ? 0 : hw[t0]);
    DM_CUDA(cudaMemsetAsync(Wc, 0, nw * sizeof(double), s));
    if (dip) {
      k_near_build_dipole<<<(unsigned)(t1 - t0), 128, 0, s>>>(P.p2p_targets + t0, P.cell_range, P.p2p_off,
                                                              P.p2p_src, P.nodes_s, P.node_vol_s, lcoloff.p, lcols,
                                                              woff, W);
      DM_LAUNCH("k_near_build_dipole");
    } else {
      if (patch) {
        k_near_build_patch<<<(unsigned)(t1 - t0), 128, 0, s>>>(
            P.p2p_targets + t0, P.cell_range, P.p2p_off, P.p2p_src, P.nodes_s, P.tets_s, P.tet_geo, P.tet_grad,
            P.nt_off, P.nt_tet, lcoloff.p, lcols, woff, fix, (unsigned long long*)W);
        DM_LAUNCH("k_near_build_patch");
      } else {
        k_near_build<<<(unsigned)(t1 - t0), 128, 0, s>>>(P.p2p_targets + t0, P.cell_range, P.p2p_off, P.p2p_src,
                                                         P.nodes_s, P.tets_s, P.tet_geo, P.tet_grad, lcoloff.p,
                                                         lcols, woff, fix, (unsigned long long*)W);
        DM_LAUNCH("k_near_build");
      }
      k_fixed_to_double<<<1024, 256, 0, s>>>(nw, Wc, 1.0 / fix);
      DM_LAUNCH("k_fixed_to_double");
    }
    if (tc) {
      std::vector<int64_t> lcnt(t1 - t0), toff;
      for (int64_t t = t0; t < t1; t++) lcnt[t - t0] = hcol[t + 1] - hcol[t];
      const int64_t q0 = tile_of(t0), q1 = tile_of(t1);
      // the leaf columns of this chunk again in keys.p for the tile keys
      std::unique_ptr<Tmp<uint64_t>> tu = tile_columns(t0, q0, q1, lcnt, toff);
      Tmp<int64_t> dto(q1 - q0 + 1);
      DM_CUDA(cudaMemcpyAsync(dto.p, toff.data(), toff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
      k_nf_tile_cols<<<(unsigned)(q1 - q0), 128, 0, s>>>(tu->p, dto.p, P.nf_coff + q0, P.nf_cols);
      DM_LAUNCH("k_nf_tile_cols");
      k_nf_pack<<<(unsigned)(t1 - t0), 256, 0, s>>>(P.p2p_targets + t0, P.cell_range, lcoloff.p, lcols, woff, W,
                                                    dltile.p + t0, dlrow0.p + t0, P.nf_woff, P.nf_coff, P.nf_ng,
                                                    P.nf_npad, P.nf_cols, P.nf_W);
      DM_LAUNCH("k_nf_pack");
      k_nf_rowsum<<<(unsigned)(t1 - t0), 128, 0, s>>>(P.p2p_targets + t0, P.cell_range, lcoloff.p, woff, W, P.nf_S);
      DM_LAUNCH("k_nf_rowsum");
      DM_CUDA(cudaStreamSynchronize(s));
    } else if (mixed) {
      // FP32 copy, [col][node][4] per target leaf (16-byte entries)
      k_pack_w32<<<(unsigned)(t1 - t0), 256, 0, s>>>(P.p2p_targets + t0, P.cell_range, lcoloff.p, woff,
                                                     P.w_off32 + t0, W, P.W32);
      DM_LAUNCH("k_pack_w32");
    }
    DM_CUDA(cudaStreamSynchronize(s));
  }
}

void launch_near_apply64(Plan& P, const double* Ms, int B, double* u_s, cudaStream_t s) {
  const int64_t nT = (int64_t)P.h_p2p_targets.size();
  if (!nT) return;
  k_near_apply<double><<<(unsigned)nT, 128, 0, s>>>(P.p2p_targets, P.cell_range, P.w_coloff, P.w_cols, P.w_off, P.W64,
                                                    Ms, B, u_s);
  DM_LAUNCH("k_near_apply<double>");
}

// Small batches: one block of 256 threads per (target leaf, slice of BS <= 8
// states), W streamed straight from HBM with one coalesced float4 load per
// (column, target node) element and no staging -- the W of a leaf is contiguous
// ([col][node]), so thread t = g NP + i (node i of a pass of NP nodes, column
// group g of G = 256 / NP) reads consecutive elements for consecutive t and
// the block sweeps the leaf's W front to back.  The NP threads of a column
// share its M (L1 broadcast).  Per-thread partial sums are added over the
// column groups in a fixed order, so the result does not depend on timing.
// The tiles of the batched kernels hold 32 or 128 states, so for small B this
// one reads W once per BS states instead of paying for the whole tile.
constexpr int NS_THREADS = 256;
constexpr int NEAR_SMALL_BATCH = 64;  // batches below this use k_near_apply32_s

template <int BS>
__device__ __forceinline__ void load_m(const float* __restrict__ mp, int B, int nlive, bool vec, float (&m)[3][BS]) {
  if (vec) {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      if constexpr (BS % 4 == 0) {
#pragma unroll
        for (int v = 0; v < BS / 4; v++) {
          const float4 x = *(const float4*)(mp + k * B + 4 * v);
          m[k][4 * v] = x.x;
          m[k][4 * v + 1] = x.y;
          m[k][4 * v + 2] = x.z;
          m[k][4 * v + 3] = x.w;
        }
      } else if constexpr (BS == 2) {
        const float2 x = *(const float2*)(mp + k * B);
        m[k][0] = x.x;
        m[k][1] = x.y;
      } else {
        m[k][0] = mp[k * B];
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 3; k++)
#pragma unroll
      for (int v = 0; v < BS; v++) m[k][v] = v < nlive ? mp[k * B + v] : 0.f;
  }
}

template <int BS>
__global__ void __launch_bounds__(NS_THREADS) k_near_apply32_s(
    const int32_t* __restrict__ targets, const int4* __restrict__ range, const int64_t* __restrict__ coloff,
    const int32_t* __restrict__ cols, const int64_t* __restrict__ woff32, const float* __restrict__ W32,
    const float* __restrict__ Ms, int B, float* u_s) {
  __shared__ float red[NS_THREADS * BS];
  const int64_t ti = blockIdx.x;
  const int4 rT = range[targets[ti]];
  const int nT = rT.w - rT.z;
  const int64_t c0 = coloff[ti];
  const int ncol = (int)(coloff[ti + 1] - c0);
  const float4* Wt = (const float4*)(W32 + woff32[ti]);
  const int b0 = blockIdx.y * BS;
  const int nlive = min(BS, B - b0);
  const bool vec = nlive == BS && (B % BS) == 0;  // M rows of this slice are BS-aligned vectors
  const int t = threadIdx.x;
  for (int i0 = 0; i0 < nT; i0 += NS_THREADS) {
    const int NP = min(NS_THREADS, nT - i0), G = NS_THREADS / NP;
    const int i = t % NP, g = t / NP;
    float acc[BS];
#pragma unroll
    for (int v = 0; v < BS; v++) acc[v] = 0.f;
    if (g < G) {
      const float4* w = Wt + i0 + i;
#pragma unroll 4
      for (int c = g; c < ncol; c += G) {
        const float4 wv = w[(int64_t)c * nT];
        float m[3][BS];
        load_m<BS>(Ms + (int64_t)cols[c0 + c] * 3 * B + b0, B, nlive, vec, m);
#pragma unroll
        for (int v = 0; v < BS; v++) acc[v] = fmaf(wv.x, m[0][v], fmaf(wv.y, m[1][v], fmaf(wv.z, m[2][v], acc[v])));
      }
    }
    __syncthreads();  // the previous pass's reduction has been read
#pragma unroll
    for (int v = 0; v < BS; v++) red[v * NS_THREADS + t] = acc[v];
    __syncthreads();
    for (int q = t; q < NP * BS; q += NS_THREADS) {
      const int ii = q % NP, v = q / NP;
      if (v < nlive) {
        float sum = 0.f;
        for (int gg = 0; gg < G; gg++) sum += red[v * NS_THREADS + gg * NP + ii];
        u_s[(int64_t)(rT.z + i0 + ii) * B + b0 + v] += sum;
      }
    }
  }
}

template <int BS>
void launch_near_small(Plan& P, const float* Ms, int B, float* u_s, cudaStream_t s) {
  dim3 grid((unsigned)P.h_p2p_targets.size(), (unsigned)((B + BS - 1) / BS));
  k_near_apply32_s<BS><<<grid, NS_THREADS, 0, s>>>(P.p2p_targets, P.cell_range, P.w_coloff, P.w_cols, P.w_off32,
                                                   P.W32, Ms, B, u_s);
  DM_LAUNCH("k_near_apply32_s");
}

void launch_near_apply32(Plan& P, const float* Ms, int B, float* u_s, int* err, cudaStream_t s) {
  const int64_t nT = (int64_t)P.h_p2p_targets.size();
  if (!nT) return;
  if (B < NEAR_SMALL_BATCH) {
    if (B == 1)
      launch_near_small<1>(P, Ms, B, u_s, s);
    else if (B == 2)
      launch_near_small<2>(P, Ms, B, u_s, s);
    else if (B <= 4)
      launch_near_small<4>(P, Ms, B, u_s, s);
    else
      launch_near_small<8>(P, Ms, B, u_s, s);
    return;
  }
  if (B % 4 == 0) {
    const size_t smem = sizeof(float4) * NB_WARPS * 2 * NB_CW * NB_NT;  // = the reduction area
    smem_opt_in((const void*)k_near_apply32_v3, smem);
    dim3 grid((unsigned)nT, (unsigned)((B + NB_STATES - 1) / NB_STATES));
    k_near_apply32_v3<<<grid, NB_WARPS * 32, smem, s>>>(P.p2p_targets, P.cell_range, P.w_coloff, P.w_cols,
                                                        P.w_off32, P.W32, Ms, B, u_s, err);
    DM_LAUNCH("k_near_apply32_v3");
    return;
  }
  const size_t smem = sizeof(float4) * NA_WARPS * NA_COLS * NA_NT;
  smem_opt_in((const void*)k_near_apply32_v2, smem);
  dim3 grid((unsigned)nT, (unsigned)((B + 31) / 32));
  k_near_apply32_v2<<<grid, NA_WARPS * 32, smem, s>>>(P.p2p_targets, P.cell_range, P.w_coloff, P.w_cols, P.w_off32,
                                                      P.W32, Ms, B, u_s, err);
  DM_LAUNCH("k_near_apply32_v2");
}

}  // namespace demag
