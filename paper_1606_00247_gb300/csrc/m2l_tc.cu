// m2l_tc.cu -- M2L on the 5th-generation tensor cores (tcgen05) for batches
// of 128 states, with FP32 accumulation in tensor memory.
//
//   Lt^T_m = (-1)^|m| / (4 pi s_T) sum_S sum_{|n| <= p - |m|} b_{n+m}(v_S) f_S^|n| Qt^S_n
// (notation of fmm32.cu).  For one target cell T this is the matrix product
//   D[b][m] = sum_S sum_n A_S[b][n] K_S[m][n],   A_S[b][n] = Qt^S_n(state b),
//   K_S[m][n] = b_{n+m}(v_S) f_S^|n|  (0 where |n| + |m| > p),
// accumulated over all sources S of T in tensor memory (M = 128 states = TMEM
// lanes, N = rows m, K = n).
//
// Translation operators.  Expansion centres are octree box centres, so
// v_S = (c_T - c_S) / s_T is fixed by the level difference and an integer
// lattice offset: 2 v = (2 k_T + 1) - (2 k_S + 1) 2^dl for dl = l_T - l_S >= 0,
// and 2^(1-dl) v = (2 k_T + 1) 2^-dl - (2 k_S + 1) otherwise (k = integer box
// coordinates).  A ball of 224k tets has ~8k distinct (dl, offset) keys for
// ~870k pairs, so every distinct K is built once per plan (FP64 b_k, rounded
// to the operand format) into a table, and each pair carries the index of its
// operator.  K is triangular in the degrees of (m, n): a row of degree t needs
// only the n with |n| <= p - t, so at k-step ks (n in [ks KW, (ks+1) KW)) the
// rows still needed are a prefix of the graded order; each k-step is one MMA
// over that prefix (N = its length padded to 16; the padding rows hold exact
// zeros of the operator), accumulating into TMEM column m for row m.
//
// Operand formats:
//   TF32   : one MMA per k-step (kind::tf32) -- ~2e-4 relative error on u;
//   BF16x3 : A = A_hi + A_lo, K = K_hi + K_lo in BF16 (16 significant bits
//            together), three MMAs per k-step (hi*hi + hi*lo + lo*hi,
//            kind::f16) -- ~3e-5 relative error on u.
//
// Data movement.  Before the M2L the moments are repacked (k_m2l_tc_pack)
// into the tensor-core tile layout, per cell and per 128 states, one 4 KB
// slice per k-step and operand copy; the operator table is stored in the same
// per-k-step order.  The M2L kernel is warp-specialised: one thread streams
// the A slices and the K slices of every source, a few k-steps at a time,
// into a ring of shared-memory slots with bulk copies (cp.async.bulk,
// completion on the slot's mbarrier); one thread issues the MMAs of each slot
// and releases it with tcgen05.commit; four warps read the accumulators at the
// end (tcgen05.ld) and write L with sign and scale.  The ring runs across
// source boundaries, so copies and MMAs overlap.  Tiles use the no-swizzle
// K-major canonical layout (8-row x 16-byte core matrices; the two core
// matrices of a k-step 128 bytes apart, 8-row groups 256 bytes apart).
//
// Issue costs shape the kernel.  On GB300 an M = 128, K = 16 BF16 MMA occupies
// its issuing CTA for ~60 cycles whatever N <= 112 (N/2 cycles above), and two
// CTAs per SM overlap about a third of that; one thread's loop overhead adds
// directly to it.  So the layout is a compile-time constant of the kernel
// (orders 4, 6, 8, 10): every MMA of a source is unrolled with constant
// descriptors offsets, and the ring shape (k-steps per slot, slots, CTAs per
// SM) is chosen at launch -- timed on the plan's own lists when the plan is
// autotuned.  Other orders run the FP32 CUDA-core M2L.
//
// Every wait is bounded: on expiry the kernel records DEMAG_ERR_TIMEOUT, stops
// issuing, waits (bounded) for its own copies and MMAs in flight, frees its
// tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <array>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace demag {

namespace {

constexpr int TC_THREADS = 256;
constexpr int TC_M = 128;              // states per CTA = MMA M = TMEM lanes
constexpr int TC_MAXKS = 48;
constexpr int TC_SLICE = TC_M * 32;    // one k-step of one operand copy: 128 rows x 32 bytes
constexpr int TC_MAXNC = 512;          // b_k table of the operator build (p <= 12)

template <class T>
struct Tmp {
  T* p = nullptr;
  explicit Tmp(size_t n) {
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "M2L tensor-core temporary allocation failed");
    }
  }
  ~Tmp() {
    if (p) cudaFree(p);
  }
};

// ---------------------------------------------------------------------------
// tile layout of one order and operand format (a compile-time constant of the
// kernels; also evaluated on the host for the operator table and the packing)
struct TcLayout {
  int valid, bf16;
  int ls;                           // split BF16 limb scheme: TC_LS_ALL2, TC_LS_ALL3 or a split degree (below)
  int lmax;                         // most limbs of any k-step (A slices are lmax x 4 KB apart)
  int E, KW;                        // elements per 16 bytes, per k-step (2E)
  int nc, ncp;                      // coefficients, padded to 16 (TMEM columns used)
  int KS;                           // k-steps of the A tile
  int Nks[TC_MAXKS];                // rows used at k-step ks (a prefix), padded to 16
  int N2[TC_MAXKS];                 // rows that also take the products with a second limb (a prefix of Nks)
  int L[TC_MAXKS];                  // limbs of k-step ks (A slices and operator rows)
  int ks_off[TC_MAXKS + 1];         // byte offset of k-step ks within one operator
  int op_bytes;                     // one operator, all k-steps, all limbs
  int a_off[TC_MAXKS + 1];          // byte offset of k-step ks within the A tile of one (cell, 128 states):
                                    // its L[ks] limb slices, 4 KB each, k-steps contiguous
  int a_bytes;                      // the whole A tile
  int tmem_cols;                    // power of two >= ncp
};

__host__ __device__ constexpr int cnc_of(int t) { return t < 0 ? 0 : (t + 1) * (t + 2) * (t + 3) / 6; }
__host__ __device__ constexpr int pad_to(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int tri3(int t) { return t * (t + 1) * (t + 2) / 6; }
// degree of the multi-index at position m of the graded order
__host__ __device__ constexpr int degree_of(int m) {
  int t = 0;
  while (tri3(t + 1) <= m) t++;
  return t;
}

// Split BF16 limb schemes.  Every product of the operator K (rows m) and the
// moments A (columns n) has a term degree |m| + |n| <= p.
//   TC_LS_ALL2: two limbs (16 significant bits) everywhere, three MMAs per
//               k-step (hi x hi, hi x lo, lo x hi) over all its rows;
//   TC_LS_ALL3: three limbs (24 bits), six MMAs per k-step;
//   d in 1..2p: the products hi x lo and lo x hi only where |m| + |n| <= d
//               (for the k-step's lowest |n|); the other terms take hi x hi
//               alone (8 significant bits per operand).  Terms of high degree
//               carry the smallest share of the expansion (they fall off like
//               the ratio of cell size to distance to that power), so their
//               8-bit products stay below the error of the low-degree terms;
//               k-steps with no such rows keep one limb and one MMA.
constexpr int TC_LS_ALL2 = 0, TC_LS_ALL3 = 99;
// default split degree: p - TC_SD_BELOW (the four highest term degrees of the
// expansion take hi x hi alone) from p = 8 on, p - 3 for lower orders (whose
// highest degrees carry a larger share)
constexpr int TC_SD_BELOW = 4;

__host__ __device__ constexpr TcLayout tc_layout(int p, bool bf16, int ls) {
  TcLayout G{};
  if (p < 1 || p > 12) return G;
  G.bf16 = bf16 ? 1 : 0;
  G.E = bf16 ? 8 : 4;
  G.KW = 2 * G.E;
  G.nc = cnc_of(p);
  G.ncp = pad_to(G.nc, 16);
  G.KS = pad_to(G.nc, G.KW) / G.KW;
  if (G.KS > TC_MAXKS) return TcLayout{};
  G.ls = bf16 ? ls : TC_LS_ALL2;
  G.lmax = 1;
  G.ks_off[0] = 0;
  for (int ks = 0; ks < G.KS; ks++) {
    int rows = 0;  // rows of degree t need n < cnc(p - t)
    for (int t = 0; t <= p; t++)
      if (cnc_of(p - t) > ks * G.KW) rows = cnc_of(t);
    G.Nks[ks] = pad_to(rows, 16);
    if (!bf16) {
      G.L[ks] = 1;
      G.N2[ks] = 0;
    } else if (ls == TC_LS_ALL3) {
      G.L[ks] = 3;
      G.N2[ks] = G.Nks[ks];
    } else if (ls == TC_LS_ALL2) {
      G.L[ks] = 2;
      G.N2[ks] = G.Nks[ks];
    } else {
      const int r = ls - degree_of(ks * G.KW);  // rows of degree <= r take the second limb
      const int n2 = r < 0 ? 0 : pad_to(cnc_of(r), 16);
      G.N2[ks] = n2 < G.Nks[ks] ? n2 : G.Nks[ks];
      G.L[ks] = G.N2[ks] > 0 ? 2 : 1;
    }
    if (G.L[ks] > G.lmax) G.lmax = G.L[ks];
    // the chunk of a k-step: hi rows (Nks), then each further limb's rows (N2)
    G.ks_off[ks + 1] = G.ks_off[ks] + 32 * (G.Nks[ks] + (G.L[ks] - 1) * G.N2[ks]);
  }
  G.op_bytes = G.ks_off[G.KS];
  G.a_off[0] = 0;
  for (int ks = 0; ks < G.KS; ks++) G.a_off[ks + 1] = G.a_off[ks] + G.L[ks] * TC_SLICE;
  G.a_bytes = G.a_off[G.KS];
  int tc = 32;
  while (tc < G.ncp) tc *= 2;
  if (tc > 512) return TcLayout{};
  G.tmem_cols = tc;
  G.valid = 1;
  return G;
}

// the orders with a compiled tensor-core kernel; split BF16 is compiled with
// the default split degree of the order and with two limbs on every k-step
// (DEMAG_MIXED_BF16X3), and with three limbs (DEMAG_MIXED_BF16X6)
constexpr bool tc_order(int p) { return p == 4 || p == 6 || p == 8 || p == 10; }
__host__ __device__ constexpr int tc_split_degree(int p) { return p >= 8 ? p - TC_SD_BELOW : p - 3; }

// launch shape: `nt` targets per CTA sharing each source's moments, `kps`
// k-steps of one source per ring slot (A slices, then one K region per target)
struct TcRing {
  int nt, kps, nsteps, amax, kmax, slot_bytes, nslots;
  int prom_group, prom_chunks;                  // promote the first prom_chunks x 16 columns every prom_group sources
  int step_koff[TC_MAXKS], step_kb[TC_MAXKS];  // K bytes of step st within one operator
  int step_aoff[TC_MAXKS], step_ab[TC_MAXKS];  // A bytes of step st within one A tile
};

bool make_ring(const TcLayout& G, int nt, int kps, int budget, TcRing& R) {
  if (!G.valid || kps < 1 || kps > G.KS || nt < 1 || nt > 2) return false;
  if (nt == 2 && (G.tmem_cols > 256 || G.ls == TC_LS_ALL3)) return false;  // two accumulators in 512 columns
  R = TcRing{};
  R.nt = nt;
  R.kps = kps;
  R.nsteps = (G.KS + kps - 1) / kps;
  int maxk = 0, maxa = 0;
  for (int st = 0; st < R.nsteps; st++) {
    const int k0 = st * kps, k1 = std::min(k0 + kps, G.KS);
    R.step_koff[st] = G.ks_off[k0];
    R.step_kb[st] = G.ks_off[k1] - G.ks_off[k0];
    R.step_aoff[st] = G.a_off[k0];
    R.step_ab[st] = G.a_off[k1] - G.a_off[k0];
    maxk = std::max(maxk, R.step_kb[st]);
    maxa = std::max(maxa, R.step_ab[st]);
  }
  R.kmax = maxk;
  R.amax = maxa;
  R.slot_bytes = pad_to(maxa + nt * maxk, 1024);
  R.nslots = std::min(32, budget / R.slot_bytes);
  return R.nslots >= 2;
}

size_t ring_smem(const TcRing& R) { return (size_t)R.nslots * R.slot_bytes + sizeof(uint64_t) * (2 * R.nslots + 3) + 64; }

// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__host__ __device__ constexpr int idx3(int a, int b, int c) {
  return tri3(a + b + c) + (b + c) * (b + c + 1) / 2 + c;
}

// shared-memory matrix descriptor, no swizzle, K-major canonical layout:
// LBO = 128 bytes between the two core matrices of a k-step, SBO = 256 bytes
// between 8-row groups, descriptor version 1 (bit 46); the start address
// (>> 4, 14 bits) is or-ed in
constexpr uint64_t DESC_FIXED = ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) | ((uint64_t)1 << 46);
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) { return DESC_FIXED | (uint64_t)((saddr & 0x3FFFFu) >> 4); }

// instruction descriptor: D F32, A and B K-major; format 2 = TF32, 1 = BF16
__host__ __device__ constexpr uint32_t idesc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(phase)
      : "memory");
  return ok != 0;
}
// bounded wait; gives up early when another role has aborted
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, volatile int* abort_flag) {
  if (mbar_test(bar, phase)) return true;
  for (int it = 0; it < (1 << 24); it++) {
    if (mbar_test(bar, phase)) return true;
    if (abort_flag && *abort_flag) return false;
    if (it > 64) __nanosleep(64);
  }
  return false;
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
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

// zero 16 accumulator columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(0u)
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// one 16-byte row of a core matrix (E consecutive values of K) in nl limbs,
// limb c at dst + c * stride: TF32 stores the FP32 values (rounded by the
// tensor core); split BF16 stores hi = BF16(v), then the BF16 roundings of the
// successive residuals
template <bool BF16>
__device__ __forceinline__ void store_row(unsigned char* dst, int stride, int nl, const float* v) {
  if constexpr (BF16) {
    float r[8];
#pragma unroll
    for (int u = 0; u < 8; u++) r[u] = v[u];
    for (int c = 0; c < nl; c++) {
      uint32_t h[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const __nv_bfloat162 hh = __floats2bfloat162_rn(r[2 * u], r[2 * u + 1]);
        const float2 hf = __bfloat1622float2(hh);
        r[2 * u] -= hf.x;  // exact: the residual of a BF16 rounding of an FP32 value is an FP32 value
        r[2 * u + 1] -= hf.y;
        h[u] = *(const uint32_t*)&hh;
      }
      *(uint4*)(dst + c * stride) = make_uint4(h[0], h[1], h[2], h[3]);
    }
  } else {
    (void)stride;
    (void)nl;
    *(float4*)dst = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// the same from FP64 values, the residuals taken in FP64
template <bool BF16>
__device__ __forceinline__ void store_row64(unsigned char* dst, int stride, int nl, const double* v) {
  if constexpr (BF16) {
    double r[8];
#pragma unroll
    for (int u = 0; u < 8; u++) r[u] = v[u];
    for (int c = 0; c < nl; c++) {
      __nv_bfloat16 h[8];
#pragma unroll
      for (int u = 0; u < 8; u++) {
        h[u] = __float2bfloat16_rn((float)r[u]);
        r[u] -= (double)__bfloat162float(h[u]);
      }
      *(uint4*)(dst + c * stride) = *(const uint4*)h;
    }
  } else {
    (void)stride;
    (void)nl;
    *(float4*)dst = make_float4((float)v[0], (float)v[1], (float)v[2], (float)v[3]);
  }
}

// ---------------------------------------------------------------------------
// moments -> tile layout: QP[cell][sb] = A tile (k-step ks at a_off[ks]: [limb][128 rows x 32 bytes])
template <bool BF16>
__global__ void __launch_bounds__(TC_M) k_m2l_tc_pack(const float* __restrict__ Q, int nc, int B, int nsb,
                                                      const TcLayout G, unsigned char* __restrict__ QP) {
  const int KS = G.KS;
  constexpr int E = BF16 ? 8 : 4;
  const int64_t cell = blockIdx.x;
  const int sb = blockIdx.y, b = threadIdx.x, bb = sb * TC_M + b;
  const bool alive = bb < B;
  const float* q = Q + cell * nc * (int64_t)B + bb;
  unsigned char* out = QP + (cell * nsb + sb) * (int64_t)G.a_bytes;
  for (int qq = 0; qq < 2 * KS; qq++) {
    float v[E];
#pragma unroll
    for (int u = 0; u < E; u++) {
      const int n = qq * E + u;
      v[u] = (alive && n < nc) ? q[(int64_t)n * B] : 0.f;
    }
    const int off = G.a_off[qq >> 1] + (b >> 3) * 256 + (qq & 1) * 128 + (b & 7) * 16;
    store_row<BF16>(out + off, TC_SLICE, G.L[qq >> 1], v);
  }
}

// ---------------------------------------------------------------------------
// operator table: key = (dl, I) with v = I * 2^-(max(0, -dl) + 1), f = 2^dl
template <bool BF16>
__global__ void __launch_bounds__(128) k_m2l_tc_ops(const int4* __restrict__ keys, int p, int nc, const TcLayout G,
                                                    unsigned char* __restrict__ ops) {
  constexpr int E = BF16 ? 8 : 4;
  __shared__ double b[TC_MAXNC];
  const int tid = threadIdx.x;
  const int4 key = keys[blockIdx.x];
  const int dl = key.x;
  const double sc = ldexp(1.0, -((dl < 0 ? -dl : 0) + 1));
  const double vx = key.y * sc, vy = key.z * sc, vz = key.w * sc, r2 = vx * vx + vy * vy + vz * vz;
  if (tid == 0) b[0] = 1.0 / sqrt(r2);
  __syncthreads();
  // b_k = (-1)^|k| d^k (1/|x|) at v:  |k| r^2 b_k = (2|k|-1) sum k_i v_i b_{k-e_i} - (|k|-1) sum k_i (k_i-1) b_{k-2e_i}
  for (int t = 1; t <= p; t++) {
    for (int k = tri3(t) + tid; k < tri3(t + 1); k += blockDim.x) {
      int ka, kb, kz;
      mi_decode(k, ka, kb, kz);
      double s1 = 0.0, s2 = 0.0;
      if (ka) s1 += ka * vx * b[idx3(ka - 1, kb, kz)];
      if (kb) s1 += kb * vy * b[idx3(ka, kb - 1, kz)];
      if (kz) s1 += kz * vz * b[idx3(ka, kb, kz - 1)];
      if (ka > 1) s2 += ka * (ka - 1) * b[idx3(ka - 2, kb, kz)];
      if (kb > 1) s2 += kb * (kb - 1) * b[idx3(ka, kb - 2, kz)];
      if (kz > 1) s2 += kz * (kz - 1) * b[idx3(ka, kb, kz - 2)];
      b[k] = ((2 * t - 1) * s1 - (t - 1) * s2) / (t * r2);
    }
    __syncthreads();
  }
  unsigned char* out = ops + (int64_t)blockIdx.x * G.op_bytes;
  for (int ks = 0; ks < G.KS; ks++) {
    unsigned char* chunk = out + G.ks_off[ks];
    const int N = G.Nks[ks];
    for (int it = tid; it < 2 * N; it += blockDim.x) {
      const int r = it >> 1, kc = it & 1;  // row m = r, 16-byte column group kc of the k-step
      double v[E];
      for (int u = 0; u < E; u++) {
        v[u] = 0.0;
        const int n = ks * G.KW + kc * E + u;
        if (r < nc && n < nc) {
          int ma, mb, mz, na, nb, nz;
          mi_decode(r, ma, mb, mz);
          mi_decode(n, na, nb, nz);
          const int tn = na + nb + nz;
          if (tn + ma + mb + mz <= p) v[u] = b[idx3(na + ma, nb + mb, nz + mz)] * ldexp(1.0, dl * tn);
        }
      }
      const int off = (r >> 3) * 256 + kc * 128 + (r & 7) * 16;
      store_row64<BF16>(chunk + off, 32 * N, r < G.N2[ks] ? G.L[ks] : 1, v);
    }
  }
}

// ---------------------------------------------------------------------------
// one CTA per group of NT targets (NT = 2: two consecutive targets, most often
// siblings) and 128 states.  The group's sources are the union of the
// targets' lists; gop[e * NT + t] is target t's operator for source e, or -1
// when e is not in its list.  Warp 0 lane 0 streams each source's A slices
// once, plus the K slices of every target that uses it; warp 1 (target 0) and
// warp 3 (target 1) issue the MMAs into their own 256-column halves of TMEM.
template <int P, bool BF16, int NT, int LS>
__global__ void __launch_bounds__(TC_THREADS, NT == 1 ? 2 : 1)
    k_m2l_tc(const int32_t* __restrict__ gtarget, const int64_t* __restrict__ goff,
             const int32_t* __restrict__ gsrc, const int32_t* __restrict__ gop, const int32_t* __restrict__ level,
             double side, int nc, int B, int nsb, const TcRing R, const unsigned char* __restrict__ QP,
             const unsigned char* __restrict__ ops, float* L, int* err) {
  constexpr TcLayout G = tc_layout(P, BF16, LS);
  static_assert(G.valid, "no tensor-core layout for this order");
  static_assert(NT == 1 || G.tmem_cols <= 256, "two targets need two 256-column accumulators");
  constexpr int TMEM_COLS = NT == 1 ? G.tmem_cols : 512;
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* full = (uint64_t*)(sm + (size_t)R.nslots * R.slot_bytes);
  uint64_t* empty = full + R.nslots;
  uint64_t* done = empty + R.nslots;
  uint64_t* gdone = done + 1;  // promotion: MMAs of a source group complete
  uint64_t* gfree = done + 2;  // promotion: the promoted columns are read and zeroed
  uint32_t* tmem_slot = (uint32_t*)(done + 3);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* counts = (int*)(tmem_slot + 2);  // slots issued, slots consumed by each issuer
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the state blocks of a group are neighbours in launch order, so the second
  // finds the group's translation operators in L2
  const int64_t grp = blockIdx.x / nsb;
  const int sb = (int)(blockIdx.x - grp * nsb);
  const int64_t e0 = goff[grp], e1 = goff[grp + 1];
  if (tid == 0) {
    for (int i = 0; i < R.nslots; i++) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], NT);  // one commit per issuer
    }
    mbar_init(done, NT);
    mbar_init(gdone, 1);
    mbar_init(gfree, 4);  // the four epilogue warps
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    *abort_flag = 0;
    counts[0] = counts[1] = counts[2] = 0;
  }
  if (warp == 2) {  // tensor memory for the accumulators
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t ring0 = smem_u32(sm), full0 = smem_u32(full), empty0 = smem_u32(empty);

  if (warp == 0) {
    // ---- producer: A slices of every (source, step) once, K slices per target using it
    if (lane == 0) {
      int slot = 0, n = 0;
      uint32_t phase = 0;
      int32_t S = gsrc[e0], O[NT];
#pragma unroll
      for (int t = 0; t < NT; t++) O[t] = gop[e0 * NT + t];
      for (int64_t e = e0; e < e1 && !*abort_flag; e++) {
        int32_t Sn = 0, On[NT];
#pragma unroll
        for (int t = 0; t < NT; t++) On[t] = -1;
        if (e + 1 < e1) {  // next source's indices, ahead of their use
          Sn = gsrc[e + 1];
#pragma unroll
          for (int t = 0; t < NT; t++) On[t] = gop[(e + 1) * NT + t];
        }
        const unsigned char* a = QP + ((int64_t)S * nsb + sb) * (int64_t)G.a_bytes;
        for (int st = 0; st < R.nsteps; st++) {
          if (n >= R.nslots && !mbar_wait(empty0 + 8 * slot, phase ^ 1u, abort_flag)) {
            if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
            *abort_flag = 1;
            break;
          }
          const uint32_t fb = full0 + 8 * slot, dst = ring0 + slot * R.slot_bytes;
          const uint32_t kb = (uint32_t)R.step_kb[st], ab = (uint32_t)R.step_ab[st];
          uint32_t bytes = ab;  // the step's A slices (contiguous), then the K slices of each target
#pragma unroll
          for (int t = 0; t < NT; t++) bytes += O[t] >= 0 ? kb : 0u;
          expect_tx(fb, bytes);
          bulk_load(dst, a + R.step_aoff[st], ab, fb);
#pragma unroll
          for (int t = 0; t < NT; t++)
            if (O[t] >= 0)
              bulk_load(dst + R.amax + t * R.kmax, ops + (int64_t)O[t] * G.op_bytes + R.step_koff[st], kb, fb);
          n++;
          if (++slot == R.nslots) {
            slot = 0;
            phase ^= 1u;
          }
        }
        S = Sn;
#pragma unroll
        for (int t = 0; t < NT; t++) O[t] = On[t];
      }
      counts[0] = n;
    }
    __syncwarp();
  } else if (warp == 1 || (NT == 2 && warp == 3)) {
    // ---- MMA issue for target t: one thread; the MMAs of a source are unrolled
    const int t = warp == 1 ? 0 : 1;
    if (lane == 0) {
      int slot = 0, n = 0;
      uint32_t phase = 0, acc = 0;  // acc = 0 until the first source of this target has started D
      uint32_t pphase = 0;          // promotion handshakes done
      bool bad = false;
      // one target per CTA: every source is in its list, no operator index is needed here
      int32_t O = NT == 1 ? 0 : gop[e0 * NT + t];
      for (int64_t e = e0; e < e1 && !bad; e++) {
        const int32_t On = NT == 1 ? 0 : (e + 1 < e1 ? gop[(e + 1) * NT + t] : -1);
        int j = 0;
        uint32_t sa = 0, kb0 = 0, a0 = 0;
#pragma unroll
        for (int ks = 0; ks < G.KS; ks++) {
          if (!bad && j == 0) {
            if (!mbar_wait(full0 + 8 * slot, phase, abort_flag)) {
              if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
              *abort_flag = 1;
              bad = true;
            }
            tc_fence_after();
            sa = ring0 + slot * R.slot_bytes;
            kb0 = sa + R.amax + t * R.kmax - G.ks_off[ks];
            a0 = sa - G.a_off[ks];
          }
          if (!bad) {
            if (O >= 0) {
              const uint32_t as = a0 + G.a_off[ks];
              const uint64_t ad = sdesc(as);
              const uint32_t kc = kb0 + G.ks_off[ks];  // k-step chunk: hi rows, then lo rows
              const int nl = G.L[ks];  // 1, 2 or 3 (compile-time after unrolling)
#pragma unroll
              for (int r0 = 0; r0 < 512; r0 += 256) {
                if (r0 < G.Nks[ks]) {
                  const int nrow = (G.Nks[ks] - r0 < 256) ? G.Nks[ks] - r0 : 256;  // MMA N <= 256
                  const uint32_t id = idesc(BF16 ? 1 : 2, TC_M, nrow);
                  const uint32_t dcol = tmem + t * 256 + r0;
                  const uint32_t kl = 32 * G.Nks[ks];  // the second limb's rows follow the hi rows
                  const uint64_t bd = sdesc(kc + 32 * r0);
                  mma<BF16>(dcol, ad, bd, id, ks == 0 ? acc : 1u);
                  if (nl >= 2 && r0 < G.N2[ks]) {  // products of limb orders 1 on the rows that take them
                    const int nrow2 = (G.N2[ks] - r0 < 256) ? G.N2[ks] - r0 : 256;
                    const uint32_t id2 = idesc(1, TC_M, nrow2);
                    mma<BF16>(dcol, ad, sdesc(kc + kl + 32 * r0), id2, 1u);
                    mma<BF16>(dcol, sdesc(as + TC_SLICE), bd, id2, 1u);
                  }
                  if (nl >= 3) {  // limb order 2 (three limbs: N2 = Nks): hi x lo, mid x mid, lo x hi
                    mma<BF16>(dcol, ad, sdesc(kc + 2 * kl + 32 * r0), id, 1u);
                    mma<BF16>(dcol, sdesc(as + TC_SLICE), sdesc(kc + kl + 32 * r0), id, 1u);
                    mma<BF16>(dcol, sdesc(as + 2 * TC_SLICE), bd, id, 1u);
                  }
                }
              }
            }
            if (++j == R.kps || ks == G.KS - 1) {
              mma_commit(empty0 + 8 * slot);  // the slot is free once both issuers' MMAs have read it
              n++;
              j = 0;
              if (++slot == R.nslots) {
                slot = 0;
                phase ^= 1u;
              }
            }
          }
        }
        if (O >= 0) acc = 1u;
        O = On;
        // promotion: hand the leading columns to the epilogue warps every prom_group sources
        if (NT == 1 && R.prom_group > 0 && !bad && ((e - e0 + 1) % R.prom_group) == 0 && e + 1 < e1) {
          mma_commit(smem_u32(gdone));
          if (!mbar_wait(smem_u32(gfree), pphase, abort_flag)) {
            if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
            *abort_flag = 1;
            bad = true;
          }
          pphase ^= 1u;
          tc_fence_after();
        }
      }
      counts[1 + t] = n;
      mma_commit(smem_u32(done));  // arrives when every MMA issued above has completed
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- epilogue: warp 4 + q reads TMEM lanes 32q .. 32q + 31 (states)
    const int q = warp - 4;
    // promotion: the leading columns are summed here in FP32 (round to nearest)
    // and zeroed in TMEM every prom_group sources, so that the accumulator
    // never carries a large running value of the cancelling low-degree terms
    float tot[64];
#pragma unroll
    for (int i = 0; i < 64; i++) tot[i] = 0.f;
    const int nprom = (NT == 1 && R.prom_group > 0) ? (int)((e1 - e0 - 1) / R.prom_group) : 0;
    for (int g = 0; g < nprom; g++) {
      if (!mbar_wait(smem_u32(gdone), (uint32_t)(g & 1), abort_flag)) {
        if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 4; c++) {
        if (c < R.prom_chunks) {
          uint32_t r[16];
          const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(16 * c);
          tmem_ld16(ta, r);
#pragma unroll
          for (int i = 0; i < 16; i++) tot[16 * c + i] += __uint_as_float(r[i]);
          tmem_zero16(ta);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(smem_u32(gfree));
    }
    const bool ok = mbar_wait(smem_u32(done), 0, nullptr);
    if (!ok) {
      atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
      *abort_flag = 1;
      mbar_wait(smem_u32(done), 0, nullptr);  // once more, bounded, for the MMAs in flight
    }
    tc_fence_after();
    if (ok && !*abort_flag) {
      const int b = sb * TC_M + q * 32 + lane;
#pragma unroll
      for (int t = 0; t < NT; t++) {
        const int32_t T = gtarget[grp * NT + t];
        if (T < 0) continue;
        const float inv = (float)(1.0 / (4.0 * M_PI * ldexp(side, -level[T])));
        float* Lt = L + (int64_t)T * nc * B + b;
#pragma unroll
        for (int c0 = 0; c0 < G.ncp; c0 += 16) {
          uint32_t r[16];
          tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(t * 256 + c0), r);
          if (b < B) {
#pragma unroll
            for (int i = 0; i < 16; i++) {
              const int m = c0 + i;
              float v = __uint_as_float(r[i]);
              if (c0 < 64 && t == 0) v += tot[(c0 < 64 ? c0 : 0) + i];  // promoted part (zero when not promoting)
              if (m < G.nc) Lt[(int64_t)m * B] = ((degree_of(m) & 1) ? -inv : inv) * v;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0 && *abort_flag) {
    // copies issued but not consumed by both issuers still land in the ring: wait for them
    const int consumed = NT == 1 ? counts[1] : min(counts[1], counts[2]);
    for (int it = consumed; it < counts[0]; it++)
      mbar_wait(full0 + 8 * (it % R.nslots), (uint32_t)((it / R.nslots) & 1), nullptr);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ---------------------------------------------------------------------------
// host side
void cell_coords(uint64_t prefix, int level, int64_t* k) {  // integer box coordinates (x bit at 3b)
  k[0] = k[1] = k[2] = 0;
  for (int b = 0; b < level; b++)
    for (int a = 0; a < 3; a++) k[a] |= (int64_t)((prefix >> (3 * b + a)) & 1ull) << b;
}

struct KeyHash {
  size_t operator()(const std::array<int64_t, 4>& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int64_t v : k) h = (h ^ (uint64_t)v) * 1099511628211ull;
    return (size_t)h;
  }
};

bool split_bf16(const Plan& P) {
  return P.opt.precision == DEMAG_MIXED_BF16X3 || P.opt.precision == DEMAG_MIXED_BF16X6;
}
TcLayout layout_of(const Plan& P) { return tc_layout(P.p, split_bf16(P), P.tc_ls); }

template <int PP, bool BF16, int NT, int LS>
void launch_fixed(Plan& P, const TcRing& R, int B, const unsigned char* QP, float* L, int* err, cudaStream_t s) {
  const size_t smem = ring_smem(R);
  smem_opt_in((const void*)k_m2l_tc<PP, BF16, NT, LS>, smem);
  const int nsb = (B + TC_M - 1) / TC_M;
  if (NT == 1) {
    dim3 grid((unsigned)(nsb * P.h_m2l_targets.size()));
    k_m2l_tc<PP, BF16, NT, LS><<<grid, TC_THREADS, smem, s>>>(P.m2l_targets, P.tc_g1_off, P.m2l_src, P.m2l_op,
                                                              P.cell_level, P.side, P.nc, B, nsb, R, QP, P.tc_ops, L,
                                                              err);
  } else {
    dim3 grid((unsigned)(nsb * P.tc_n_g2));
    k_m2l_tc<PP, BF16, NT, LS><<<grid, TC_THREADS, smem, s>>>(P.tc_g2_tgt, P.tc_g2_off, P.tc_g2_src, P.tc_g2_op,
                                                              P.cell_level, P.side, P.nc, B, nsb, R, QP, P.tc_ops, L,
                                                              err);
  }
  DM_LAUNCH("k_m2l_tc");
}

// compiled variants: TF32, and split BF16 with the order's default split
// degree or two limbs everywhere, with one or two targets per CTA; three-limb
// split BF16 with one target per CTA
template <int PP, bool BF16, int LS>
void launch_ls(Plan& P, const TcRing& R, int B, const unsigned char* QP, float* L, int* err, cudaStream_t s) {
  if constexpr (tc_layout(PP, BF16, LS).tmem_cols <= 256) {
    if (R.nt == 2) return launch_fixed<PP, BF16, 2, LS>(P, R, B, QP, L, err, s);
  }
  launch_fixed<PP, BF16, 1, LS>(P, R, B, QP, L, err, s);
}

template <int PP, bool BF16>
void launch_nt(Plan& P, const TcRing& R, int B, const unsigned char* QP, float* L, int* err, cudaStream_t s) {
  if constexpr (BF16) {
    if (P.tc_ls == TC_LS_ALL3) return launch_fixed<PP, BF16, 1, TC_LS_ALL3>(P, R, B, QP, L, err, s);
    if (P.tc_ls == tc_split_degree(PP)) return launch_ls<PP, BF16, tc_split_degree(PP)>(P, R, B, QP, L, err, s);
  }
  launch_ls<PP, BF16, TC_LS_ALL2>(P, R, B, QP, L, err, s);
}

template <bool BF16>
void launch_order(Plan& P, const TcRing& R, int B, const unsigned char* QP, float* L, int* err, cudaStream_t s) {
  switch (P.p) {
    case 4: launch_nt<4, BF16>(P, R, B, QP, L, err, s); break;
    case 6: launch_nt<6, BF16>(P, R, B, QP, L, err, s); break;
    case 8: launch_nt<8, BF16>(P, R, B, QP, L, err, s); break;
    case 10: launch_nt<10, BF16>(P, R, B, QP, L, err, s); break;
    default: fail(DEMAG_ERR_UNSUPPORTED, "no tensor-core M2L for this order");
  }
}

void launch_main(Plan& P, const TcRing& R, int B, const unsigned char* QP, float* L, int* err, cudaStream_t s) {
  if (split_bf16(P))
    launch_order<true>(P, R, B, QP, L, err, s);
  else
    launch_order<false>(P, R, B, QP, L, err, s);
}

// ring budgets: ~100 KB lets two CTAs share an SM (when their tensor memory
// fits), ~200 KB gives one CTA the whole shared memory
constexpr int TC_BUDGET_2 = 100 * 1024, TC_BUDGET_1 = 200 * 1024;

// default launch shape (the fastest measured on GB300 for a ball of 224k tets
// at p = 8): one target per CTA, 2 k-steps per slot, and a ring small enough
// for two CTAs per SM when their tensor memory fits; nt / kps override it
void default_ring(const TcLayout& G, int nt, int kps, TcRing& R) {
  if (nt == 0) nt = 1;
  if (kps == 0) kps = std::min(G.KS, 2);
  const int budget = (nt == 1 && G.tmem_cols <= 256) ? TC_BUDGET_2 : TC_BUDGET_1;
  for (; kps >= 1; kps--)
    if (make_ring(G, nt, kps, budget, R) || make_ring(G, nt, kps, TC_BUDGET_1, R)) return;
  R.nslots = 0;
}

// autotune: time every launch shape on the plan's own lists (zero moments,
// 128 states) and keep the fastest
void tune_ring(Plan& P, const TcLayout& G) {
  cudaStream_t s = P.stream;
  const int B = TC_M;
  Tmp<unsigned char> qp((size_t)P.ncells * G.a_bytes);
  Tmp<float> L((size_t)P.ncells * P.nc * B);
  Tmp<int> err(1);
  DM_CUDA(cudaMemsetAsync(qp.p, 0, (size_t)P.ncells * G.a_bytes, s));
  DM_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
  cudaEvent_t a, b;
  DM_CUDA(cudaEventCreate(&a));
  DM_CUDA(cudaEventCreate(&b));
  float best = 1e30f;
  // two-target groups carry no accumulator promotion: with promotion on (the
  // default) the tuner keeps one target per CTA, whose accuracy it must not trade
  const int nt_max = P.tc_prom_group > 0 ? 1 : 2;
  for (int nt = 1; nt <= nt_max; nt++)
    for (int budget : {TC_BUDGET_2, TC_BUDGET_1}) {
      if (budget == TC_BUDGET_2 && (nt == 2 || G.tmem_cols > 256)) continue;  // one CTA per SM anyway
      for (int kps = 1; kps <= std::min(G.KS, 8); kps++) {
        TcRing R;
        if (!make_ring(G, nt, kps, budget, R)) continue;
        if (ring_smem(R) > 227 * 1024) continue;
        launch_main(P, R, B, qp.p, L.p, err.p, s);  // warm-up
        DM_CUDA(cudaEventRecord(a, s));
        launch_main(P, R, B, qp.p, L.p, err.p, s);
        DM_CUDA(cudaEventRecord(b, s));
        DM_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        DM_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (ms < best) {
          best = ms;
          P.tc_nt = nt;
          P.tc_kps = kps;
          P.tc_budget = budget;
        }
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  int h_err = 0;
  DM_CUDA(cudaMemcpy(&h_err, err.p, sizeof(int), cudaMemcpyDeviceToHost));
  if (h_err) fail(DEMAG_ERR_TIMEOUT, "tensor-core M2L timed out while tuning");
}

bool current_ring(const Plan& P, const TcLayout& G, TcRing& R) {
  if (!(P.tc_kps > 0 && make_ring(G, P.tc_nt, P.tc_kps, P.tc_budget, R)))
    default_ring(G, P.opt.m2l_targets_per_cta, P.opt.m2l_kps, R);
  R.prom_group = R.nt == 1 ? P.tc_prom_group : 0;
  R.prom_chunks = std::min(4, std::max(1, (P.tc_prom_rows + 15) / 16));
  return R.nslots >= 2;
}

template <bool BF16>
void build_ops(Plan& P, const TcLayout& G, const std::vector<int4>& keys) {
  cudaStream_t s = P.stream;
  P.tc_ops = dalloc<unsigned char>(P, (size_t)keys.size() * G.op_bytes);
  Tmp<int4> dkeys(keys.size());
  DM_CUDA(cudaMemcpyAsync(dkeys.p, keys.data(), keys.size() * sizeof(int4), cudaMemcpyHostToDevice, s));
  k_m2l_tc_ops<BF16><<<(unsigned)keys.size(), 128, 0, s>>>(dkeys.p, P.p, P.nc, G, P.tc_ops);
  DM_LAUNCH("k_m2l_tc_ops");
  DM_CUDA(cudaStreamSynchronize(s));
}

bool tc_enabled(const Plan& P) { return (P.opt.precision == DEMAG_MIXED_TF32 || split_bf16(P)) && P.tc_ops != nullptr; }

}  // namespace

M2lKeys build_m2l_keys(Plan& P) {
  M2lKeys K;
  if (P.n_m2l == 0) return K;
  cudaStream_t s = P.stream;
  const int64_t nc = P.ncells;
  std::vector<uint64_t> prefix(nc);
  std::vector<int32_t> lev(nc);
  K.off.resize(nc + 1);
  K.src.resize(P.n_m2l);
  DM_CUDA(cudaMemcpyAsync(prefix.data(), P.cell_prefix, nc * sizeof(uint64_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(lev.data(), P.cell_level, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(K.off.data(), P.m2l_off, (nc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(K.src.data(), P.m2l_src, P.n_m2l * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  std::vector<std::array<int64_t, 3>> kc(nc);
  for (int64_t c = 0; c < nc; c++) cell_coords(prefix[c], lev[c], kc[c].data());
  std::unordered_map<std::array<int64_t, 4>, int32_t, KeyHash> index;
  K.op.resize(P.n_m2l);
  for (int64_t T = 0; T < nc; T++)
    for (int64_t e = K.off[T]; e < K.off[T + 1]; e++) {
      const int32_t S = K.src[e];
      const int dl = lev[T] - lev[S];
      std::array<int64_t, 4> key{dl, 0, 0, 0};
      for (int a = 0; a < 3; a++)
        key[1 + a] = dl >= 0 ? (2 * kc[T][a] + 1) - ((2 * kc[S][a] + 1) << dl)
                             : ((2 * kc[T][a] + 1) << (-dl)) - (2 * kc[S][a] + 1);
      auto f = index.find(key);
      if (f == index.end()) {
        for (int a = 1; a < 4; a++)
          if (key[a] > INT32_MAX || key[a] < INT32_MIN) return M2lKeys{};  // beyond the table's key range
        f = index.emplace(key, (int32_t)K.keys.size()).first;
        K.keys.push_back(make_int4(dl, (int)key[1], (int)key[2], (int)key[3]));
      }
      K.op[e] = f->second;
    }
  P.m2l_op = dalloc<int32_t>(P, P.n_m2l);
  DM_CUDA(cudaMemcpyAsync(P.m2l_op, K.op.data(), P.n_m2l * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaStreamSynchronize(s));
  P.n_tc_ops = (int64_t)K.keys.size();
  K.ok = true;
  return K;
}

void build_m2l_tc(Plan& P, const M2lKeys& K) {
  if (P.opt.precision != DEMAG_MIXED_TF32 && !split_bf16(P)) return;
  if (!K.ok || !tc_order(P.p)) return;  // the CUDA-core M2L runs instead
  P.tc_prom_group = P.opt.m2l_promote < 0 ? 0 : (P.opt.m2l_promote == 0 ? 8 : P.opt.m2l_promote);
  P.tc_prom_rows = P.opt.m2l_promote_rows > 0 ? P.opt.m2l_promote_rows : 16;
  P.tc_ls = P.opt.precision == DEMAG_MIXED_BF16X6
                ? TC_LS_ALL3
                : (P.opt.m2l_split_degree < 0 ? TC_LS_ALL2 : tc_split_degree(P.p));
  const TcLayout G = layout_of(P);
  if (!G.valid) return;
  cudaStream_t s = P.stream;
  const std::vector<int64_t>& off = K.off;
  const std::vector<int32_t>& src = K.src;
  const std::vector<int32_t>& op = K.op;
  if (G.bf16)
    build_ops<true>(P, G, K.keys);
  else
    build_ops<false>(P, G, K.keys);
  // groups of one target: the target's own list
  const int64_t nT = (int64_t)P.h_m2l_targets.size();
  std::vector<int64_t> g1(nT + 1);
  for (int64_t i = 0; i < nT; i++) g1[i] = off[P.h_m2l_targets[i]];
  g1[nT] = nT ? off[P.h_m2l_targets[nT - 1] + 1] : 0;
  P.tc_g1_off = dalloc<int64_t>(P, nT + 1);
  DM_CUDA(cudaMemcpyAsync(P.tc_g1_off, g1.data(), (nT + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  // groups of two consecutive targets: the union of their (ascending) lists
  if (G.tmem_cols <= 256) {
    const int64_t ng = (nT + 1) / 2;
    std::vector<int32_t> tgt(2 * ng, -1), usrc, uop;
    std::vector<int64_t> uoff(ng + 1, 0);
    usrc.reserve(P.n_m2l);
    uop.reserve(2 * P.n_m2l);
    for (int64_t g = 0; g < ng; g++) {
      const int32_t T0 = P.h_m2l_targets[2 * g], T1 = 2 * g + 1 < nT ? P.h_m2l_targets[2 * g + 1] : -1;
      tgt[2 * g] = T0;
      tgt[2 * g + 1] = T1;
      int64_t i = off[T0], ie = off[T0 + 1], j = T1 >= 0 ? off[T1] : 0, je = T1 >= 0 ? off[T1 + 1] : 0;
      while (i < ie || j < je) {
        const int32_t si = i < ie ? src[i] : INT32_MAX, sj = j < je ? src[j] : INT32_MAX;
        const int32_t sm = std::min(si, sj);
        usrc.push_back(sm);
        uop.push_back(si == sm ? op[i++] : -1);
        uop.push_back(sj == sm ? op[j++] : -1);
      }
      uoff[g + 1] = (int64_t)usrc.size();
    }
    P.tc_n_g2 = ng;
    P.tc_g2_tgt = dalloc<int32_t>(P, 2 * ng);
    P.tc_g2_off = dalloc<int64_t>(P, ng + 1);
    P.tc_g2_src = dalloc<int32_t>(P, usrc.size());
    P.tc_g2_op = dalloc<int32_t>(P, uop.size());
    DM_CUDA(cudaMemcpyAsync(P.tc_g2_tgt, tgt.data(), tgt.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.tc_g2_off, uoff.data(), uoff.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.tc_g2_src, usrc.data(), usrc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.tc_g2_op, uop.data(), uop.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  DM_CUDA(cudaStreamSynchronize(s));
  P.tc_nt = 1;
  P.tc_kps = 0;
  P.tc_budget = 0;
  if ((P.opt.autotune & 1) && P.opt.m2l_targets_per_cta == 0 && P.opt.m2l_kps == 0) {
    const bool preset = P.tc_preset_kps >= 1 && P.tc_preset_kps <= 8 &&
                        (P.tc_preset_nt == 1 || (P.tc_preset_nt == 2 && P.tc_prom_group == 0));
    if (preset) {  // a shape this tuner chose before on the same mesh and options
      P.tc_nt = P.tc_preset_nt;
      P.tc_kps = P.tc_preset_kps;
      P.tc_budget = P.tc_preset_budget;
    } else {
      tune_ring(P, G);
    }
  }
  TcRing R;
  if (!current_ring(P, G, R)) fail(DEMAG_ERR_UNSUPPORTED, "no ring shape fits the tensor-core M2L");
  P.tc_nt = R.nt;
  P.tc_kps = R.kps;
  P.tc_budget = R.nslots * R.slot_bytes;
}

size_t m2l_tc_pack_bytes(const Plan& P, int B) {
  if (!tc_enabled(P)) return 0;
  if (B <= m2l_table_batch(P) && P.m2l_tab != nullptr) return 0;  // the table-driven M2L runs instead
  const TcLayout G = layout_of(P);
  const size_t nsb = (size_t)(B + TC_M - 1) / TC_M;
  return (size_t)P.ncells * nsb * G.a_bytes;
}

bool launch_m2l_tc(Plan& P, int B, const float* Q, unsigned char* QP, float* L, int* err, cudaStream_t s) {
  if (P.h_m2l_targets.empty()) return true;
  if (!tc_enabled(P) || QP == nullptr) return false;
  const TcLayout G = layout_of(P);
  TcRing R;
  if (!current_ring(P, G, R)) return false;
  const int nsb = (B + TC_M - 1) / TC_M;
  const dim3 grid((unsigned)P.ncells, (unsigned)nsb);
  if (G.bf16)
    k_m2l_tc_pack<true><<<grid, TC_M, 0, s>>>(Q, P.nc, B, nsb, G, QP);
  else
    k_m2l_tc_pack<false><<<grid, TC_M, 0, s>>>(Q, P.nc, B, nsb, G, QP);
  DM_LAUNCH("k_m2l_tc_pack");
  launch_main(P, R, B, QP, L, err, s);
  return true;
}

}  // namespace demag
