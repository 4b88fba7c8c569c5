// m2l_tc.cu -- M2L on the 5th-generation tensor cores (tcgen05) for batches
// of 128 states, with FP32 accumulation in tensor memory.
//
//   Lt^T_m = (-1)^|m| / (4 pi s_T) sum_S sum_{|n| <= p - |m|} b_{n+m}(v_S) f_S^|n| Qt^S_n
// (notation of fmm32.cu).  For one target cell T this is the matrix product
//   D[b][m] = sum_S sum_n A_S[b][n] K_S[m][n],   A_S[b][n] = Qt^S_n(state b),
//   K_S[m][n] = b_{n+m}(v_S) f_S^|n|  (0 where |n| + |m| > p),
// accumulated over all sources S of T in tensor memory (M = 128 states = TMEM
// lanes, N = rows m, K = n).  K_S is triangular in the degrees of (m, n); the
// rows are cut into level groups [ta, tb) (chosen on the host by a small
// dynamic programme), group g multiplying only the n with |n| <= p - ta, so
// that the dense tiles cover ~2.2x the useful entries at p = 8 instead of ~9x.
//
// Two operand formats:
//   TF32   : A and K_S rounded to TF32 by the tensor core, one MMA per k-step
//            (kind::tf32) -- fastest, ~2e-4 relative error on u;
//   BF16x3 : A = A_hi + A_lo, K = K_hi + K_lo with hi/lo in BF16 (16 significant
//            bits together), three MMAs per k-step (hi*hi + hi*lo + lo*hi,
//            kind::f16) -- ~1e-5 relative error on u.
//
// Per source the CTA (8 warps) writes A_S (moments of the 128 states) and the
// group tiles of K_S (operator values from the Taylor-coefficient recurrence of
// 1/|x|, built for 8 sources at a time) into shared memory in the no-swizzle
// K-major canonical layout (8-row x 16-byte core matrices, K-adjacent core
// matrices 128 bytes apart), one thread issues the tcgen05.mma instructions and
// commits them to an mbarrier, and the operands are rebuilt once the mbarrier
// reports that the tensor core has consumed them.  The epilogue reads the
// accumulators with tcgen05.ld and applies sign and scale.  Every wait is
// bounded: on expiry the kernel records DEMAG_ERR_TIMEOUT, waits once more for
// its own MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace demag {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;  // states per CTA = MMA M = TMEM lanes
constexpr int TC_BCH = 8;  // sources per operator batch
constexpr int TC_MAXG = 8;

struct TcGroups {
  int ng;
  int m0[TC_MAXG], nrow[TC_MAXG];  // rows [m0, m0 + nrow) of the graded order
  int N[TC_MAXG];                  // rows padded to a multiple of 16 (MMA N)
  int K[TC_MAXG];                  // n count padded to one MMA k-step (32 bytes of K)
  int col[TC_MAXG];                // first TMEM column of the group
  int boff[TC_MAXG];               // byte offset of the group's K_S tile in the B area
  int sbo[TC_MAXG];                // stride between 8-row core-matrix groups of that tile
  int kmax;                        // padded K of the A tile
  int sbo_a;                       // stride between 8-row groups of the A tile
  int a_bytes, b_bytes;            // one copy of the A tile / of all K_S tiles
  int tmem_cols;                   // power of two >= sum of N
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ int tri3(int t) { return t * (t + 1) * (t + 2) / 6; }
__device__ __forceinline__ int tri2(int j) { return j * (j + 1) / 2; }
__device__ __forceinline__ int idx3(int a, int b, int c) { return tri3(a + b + c) + tri2(b + c) + c; }

// shared-memory matrix descriptor: no swizzle, K-major canonical layout
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of this architecture
  return d;                // base offset 0, relative LBO, swizzle none
}
// instruction descriptors: D F32, A and B K-major; format 2 = TF32, 1 = BF16
__host__ __device__ constexpr uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
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
    if (it > 64) __nanosleep(32);
  }
  return false;
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t id, uint32_t acc) {
  if constexpr (BF16)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(acc)
        : "memory");
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(id), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// elements per 16-byte core-matrix row: 4 (TF32 in FP32 containers) or 8 (BF16)
template <bool BF16>
constexpr int EPR = BF16 ? 8 : 4;

// byte offset of element (row r, k) in a K-major no-swizzle tile
template <bool BF16>
__device__ __forceinline__ int tile_off(int r, int k, int sbo) {
  return (r >> 3) * sbo + (k / EPR<BF16>)*128 + (r & 7) * 16;
}

// one 16-byte row of a core matrix: EPR consecutive values of K; BF16x3
// writes the high part to `hi` and the rounding residual to `lo`
template <bool BF16>
__device__ __forceinline__ void store_row(unsigned char* hi, unsigned char* lo, const float* v) {
  if constexpr (BF16) {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      h[u] = __float2bfloat16_rn(v[u]);
      l[u] = __float2bfloat16_rn(v[u] - __bfloat162float(h[u]));
    }
    *(uint4*)hi = *(const uint4*)h;
    *(uint4*)lo = *(const uint4*)l;
  } else {
    (void)lo;
    *(float4*)hi = make_float4(v[0], v[1], v[2], v[3]);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(const int32_t* __restrict__ targets,
                                                        const int64_t* __restrict__ m2l_off,
                                                        const int32_t* __restrict__ m2l_src,
                                                        const double* __restrict__ centre,
                                                        const int32_t* __restrict__ level, double side, int p, int nc,
                                                        int B, const TcGroups G, const float* __restrict__ Q, float* L,
                                                        int* err) {
  constexpr int E = EPR<BF16>;
  constexpr int NCOPY = BF16 ? 2 : 1;  // hi (+ lo)
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As = sm;                               // A tile(s): 128 states x kmax
  unsigned char* Bs = As + NCOPY * G.a_bytes;           // group tiles of K_S (hi, then lo)
  float* bks = (float*)(Bs + NCOPY * G.b_bytes);        // TC_BCH x nc operator vectors
  float* fps = bks + TC_BCH * nc;                       // TC_BCH x 16
  float* geo = fps + TC_BCH * 16;                       // TC_BCH x 4
  int* mi = (int*)(geo + TC_BCH * 4);                   // nc packed multi-indices
  uint64_t* bar = (uint64_t*)(mi + ((nc + 1) & ~1));
  uint32_t* tmem_slot = (uint32_t*)(bar + 1);
  int* abort_flag = (int*)(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int32_t T = targets[blockIdx.x];
  const int b0 = blockIdx.y * TC_M;
  const double sT = ldexp(side, -level[T]);
  const double cx = centre[3 * T], cy = centre[3 * T + 1], cz = centre[3 * T + 2];
  for (int i = tid; i < nc; i += blockDim.x) {
    int a, b, c;
    mi_decode(i, a, b, c);
    mi[i] = a | (b << 8) | (c << 16) | ((a + b + c) << 24);
  }
  if (tid == 0) {
    mbar_init(bar);
    *abort_flag = 0;
  }
  if (warp == 0) {  // tensor memory for the accumulators of all groups
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(G.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  uint32_t phase = 0;
  bool first = true;
  const int64_t e0 = m2l_off[T], e1 = m2l_off[T + 1];
  for (int64_t ec = e0; ec < e1; ec += TC_BCH) {
    const int ns = (e1 - ec < TC_BCH) ? (int)(e1 - ec) : TC_BCH;
    if (tid < ns) {
      const int32_t S = m2l_src[ec + tid];
      const float x = (float)((cx - centre[3 * S]) / sT), y = (float)((cy - centre[3 * S + 1]) / sT),
                  z = (float)((cz - centre[3 * S + 2]) / sT);
      float* g = geo + 4 * tid;
      g[0] = x;
      g[1] = y;
      g[2] = z;
      g[3] = x * x + y * y + z * z;
      bks[tid * nc] = rsqrtf(g[3]);
      const int dl = level[T] - level[S];
      for (int t = 0; t <= p; t++) fps[tid * 16 + t] = ldexpf(1.f, dl * t);
    }
    __syncthreads();
    for (int t = 1; t <= p; t++) {
      const int o = tri3(t), cnt = (t + 1) * (t + 2) / 2;
      for (int q = tid; q < ns * cnt; q += blockDim.x) {
        const int s = q / cnt, k = o + (q - s * cnt);
        const int kk = mi[k], ka = kk & 255, kb = (kk >> 8) & 255, kz = (kk >> 16) & 255;
        const float* g = geo + 4 * s;
        const float* bb = bks + s * nc;
        float s1 = 0.f, s2 = 0.f;
        if (ka) s1 += ka * g[0] * bb[idx3(ka - 1, kb, kz)];
        if (kb) s1 += kb * g[1] * bb[idx3(ka, kb - 1, kz)];
        if (kz) s1 += kz * g[2] * bb[idx3(ka, kb, kz - 1)];
        if (ka > 1) s2 += ka * (ka - 1) * bb[idx3(ka - 2, kb, kz)];
        if (kb > 1) s2 += kb * (kb - 1) * bb[idx3(ka, kb - 2, kz)];
        if (kz > 1) s2 += kz * (kz - 1) * bb[idx3(ka, kb, kz - 2)];
        bks[s * nc + k] = ((2 * t - 1) * s1 - (t - 1) * s2) / (t * g[3]);
      }
      __syncthreads();
    }
    for (int s = 0; s < ns; s++) {
      const int32_t S = m2l_src[ec + s];
      // ---- A_S: moments of the 128 states, E consecutive n per 16-byte row
      {
        const float* Qs = Q + (int64_t)S * nc * B + b0;
        const int b = tid & (TC_M - 1);
        const bool live = b0 + b < B;
        for (int q = tid >> 7; q < G.kmax / E; q += TC_THREADS / TC_M) {
          float v[E];
#pragma unroll
          for (int u = 0; u < E; u++) {
            const int n = E * q + u;
            v[u] = (live && n < nc) ? Qs[(int64_t)n * B + b] : 0.f;
          }
          const int off = tile_off<BF16>(b, E * q, G.sbo_a);
          store_row<BF16>(As + off, As + G.a_bytes + off, v);
        }
      }
      // ---- K_S group tiles
      {
        const float* bk = bks + s * nc;
        const float* fp = fps + s * 16;
        for (int g = 0; g < G.ng; g++) {
          const int nq = G.K[g] / E, items = G.N[g] * nq;
          unsigned char* tile = Bs + G.boff[g];
          for (int it = tid; it < items; it += blockDim.x) {
            const int q = it / G.N[g], r = it - q * G.N[g];  // consecutive threads: consecutive rows
            float v[E];
#pragma unroll
            for (int u = 0; u < E; u++) v[u] = 0.f;
            if (r < G.nrow[g]) {
              const int mm = mi[G.m0[g] + r];
              const int ma = mm & 255, mb = (mm >> 8) & 255, mz = (mm >> 16) & 255, tm = mm >> 24;
#pragma unroll
              for (int u = 0; u < E; u++) {
                const int n = E * q + u;
                if (n < nc) {
                  const int nn = mi[n], tn = nn >> 24;
                  if (tn + tm <= p)
                    v[u] = bk[idx3((nn & 255) + ma, ((nn >> 8) & 255) + mb, ((nn >> 16) & 255) + mz)] * fp[tn];
                }
              }
            }
            const int off = tile_off<BF16>(r, E * q, G.sbo[g]);
            store_row<BF16>(tile + off, tile + G.b_bytes + off, v);
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> tensor-core reads
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        const uint32_t a_hi = smem_u32(As), b_hi = smem_u32(Bs);
        for (int g = 0; g < G.ng; g++) {
          const uint32_t id = idesc(BF16 ? 1 : 2, TC_M, G.N[g]);
          for (int ks = 0; ks < G.K[g] / (2 * E); ks++) {  // one k-step = 32 bytes of K = 2 core matrices
            const uint32_t ao = ks * 256, bo = G.boff[g] + ks * 256;
            const uint64_t ad = smem_desc(a_hi + ao, 128, G.sbo_a);
            const uint64_t bd = smem_desc(b_hi + bo, 128, G.sbo[g]);
            const uint32_t acc = (first && ks == 0) ? 0u : 1u;
            mma<BF16>(tmem + G.col[g], ad, bd, id, acc);
            if constexpr (BF16) {
              const uint64_t adl = smem_desc(a_hi + G.a_bytes + ao, 128, G.sbo_a);
              const uint64_t bdl = smem_desc(b_hi + G.b_bytes + bo, 128, G.sbo[g]);
              mma<BF16>(tmem + G.col[g], ad, bdl, id, 1u);  // hi x lo
              mma<BF16>(tmem + G.col[g], adl, bd, id, 1u);  // lo x hi
            }
          }
        }
        mma_commit(bar);
      }
      first = false;
      // the operands may be overwritten once the tensor core has read them
      const bool ok = mbar_wait(bar, phase);
      if (!ok) {
        if (tid == 0) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
        mbar_wait(bar, phase);  // once more, bounded, for the MMAs in flight
        *abort_flag = 1;
      }
      phase ^= 1;
      tc_fence_after();
      __syncthreads();
      if (*abort_flag) break;
    }
    if (*abort_flag) break;
  }
  // ---- epilogue: warps 0-3 read lanes 32w .. 32w+31 (states) of every group
  if (!*abort_flag && warp < 4 && !first) {
    const float inv = (float)(1.0 / (4.0 * M_PI * sT));
    const int b = b0 + warp * 32 + lane;
    for (int g = 0; g < G.ng; g++) {
      for (int c0 = 0; c0 < G.N[g]; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(G.col[g] + c0), r);
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const int row = c0 + i;
          if (row < G.nrow[g] && b < B) {
            const int m = G.m0[g] + row;
            const float sg = ((mi[m] >> 24) & 1) ? -inv : inv;
            L[((int64_t)T * nc + m) * B + b] = sg * __uint_as_float(r[i]);
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.tmem_cols) : "memory");
}

// level groups for order p: minimise the padded tile area sum N_g * K_g
// (epr = elements per 16 bytes: K is padded to one k-step of 2 * epr)
bool make_groups(int p, int epr, TcGroups& G) {
  auto cnc = [](int t) { return t < 0 ? 0 : (t + 1) * (t + 2) * (t + 3) / 6; };
  auto pad = [](int x, int m) { return (x + m - 1) / m * m; };
  const int T = p + 1, kstep = 2 * epr;
  std::vector<long> best(T + 1, -1);
  std::vector<int> from(T + 1, -1);
  best[0] = 0;
  for (int tb = 1; tb <= T; tb++)  // groups cover degrees [ta, tb)
    for (int ta = 0; ta < tb; ta++) {
      if (best[ta] < 0) continue;
      const long cost = (long)pad(cnc(tb - 1) - cnc(ta - 1), 16) * pad(cnc(p - ta), kstep) + 256;
      if (best[tb] < 0 || best[ta] + cost < best[tb]) {
        best[tb] = best[ta] + cost;
        from[tb] = ta;
      }
    }
  std::vector<std::pair<int, int>> gs;
  for (int tb = T; tb > 0; tb = from[tb]) gs.push_back({from[tb], tb});
  std::reverse(gs.begin(), gs.end());
  if ((int)gs.size() > TC_MAXG) return false;
  G.ng = (int)gs.size();
  int col = 0, boff = 0;
  G.kmax = 0;
  for (int g = 0; g < G.ng; g++) {
    const int ta = gs[g].first, tb = gs[g].second;
    G.m0[g] = cnc(ta - 1);
    G.nrow[g] = cnc(tb - 1) - cnc(ta - 1);
    G.N[g] = pad(G.nrow[g], 16);
    G.K[g] = pad(cnc(p - ta), kstep);
    G.col[g] = col;
    col += G.N[g];
    G.sbo[g] = (G.K[g] / epr) * 128 + 16;  // +16 bytes spreads the 8-row groups over the banks
    G.boff[g] = boff;
    boff = pad(boff + (G.N[g] / 8) * G.sbo[g], 128);
    G.kmax = std::max(G.kmax, G.K[g]);
  }
  G.sbo_a = (G.kmax / epr) * 128 + 16;
  G.a_bytes = pad((TC_M / 8) * G.sbo_a, 1024);
  G.b_bytes = pad(boff, 128);
  int tc = 32;
  while (tc < col) tc *= 2;
  if (tc > 512) return false;
  G.tmem_cols = tc;
  return true;
}

size_t tc_smem_bytes(const TcGroups& G, int nc, int ncopy) {
  return (size_t)ncopy * (G.a_bytes + G.b_bytes) + sizeof(float) * (TC_BCH * nc + TC_BCH * 16 + TC_BCH * 4) +
         sizeof(int) * ((nc + 1) & ~1) + sizeof(uint64_t) + 2 * sizeof(uint32_t) + 64;
}

template <bool BF16>
bool launch(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s) {
  TcGroups G;
  if (!make_groups(P.p, EPR<BF16>, G)) return false;
  const size_t smem = tc_smem_bytes(G, P.nc, BF16 ? 2 : 1);
  if (smem > 227 * 1024) return false;
  static size_t attr = 0;
  if (smem > attr) {
    DM_CUDA(cudaFuncSetAttribute(k_m2l_tc<BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((B + TC_M - 1) / TC_M));
  k_m2l_tc<BF16><<<grid, TC_THREADS, smem, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, P.cell_level,
                                                P.side, P.p, P.nc, B, G, Q, L, err);
  DM_LAUNCH("k_m2l_tc");
  return true;
}

}  // namespace

bool launch_m2l_tc(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s) {
  if (P.h_m2l_targets.empty()) return true;
  if (P.opt.precision == DEMAG_MIXED_BF16X3) return launch<true>(P, B, Q, L, err, s);
  return launch<false>(P, B, Q, L, err, s);
}

}  // namespace demag
