// m2l32.cu -- FP32 M2L on CUDA cores for batches of states (mixed path).
//
//   Lt^T_m = (-1)^|m| / (4 pi s_T) sum_S sum_{|n| <= p - |m|} b_{n+m}(v_S) f_S^|n| Qt^S_n
// (v_S = (c_T - c_S)/s_T, f_S = s_S/s_T, notation of fmm32.cu).
//
// Layout: one block per (target cell, slice of 32 states).  Thread = one output
// row m and SPT = 16 states held in registers, so every operator value
// b_{n+m} read from shared memory feeds 16 FMAs and the 16 moments of a given n
// are read with four 16-byte shared-memory broadcasts.  Sources are staged
// CHUNK at a time (their moments for the slice and their operator vectors
// b_k(v), computed in the block by the Taylor-coefficient recurrence of 1/|x|).
// All threads run the same short loop (no per-warp code paths).
#include <algorithm>
#include <utility>

#include "common.cuh"

namespace demag {

namespace {

constexpr int SPT = 16;    // states per thread
constexpr int SLICE = 32;  // states per block

__device__ __forceinline__ int idx3(int a, int b, int c) {
  const int t = a + b + c, j = b + c;
  return t * (t + 1) * (t + 2) / 6 + j * (j + 1) / 2 + c;
}

__global__ void __launch_bounds__(1024) k_m2l32_rows(const int32_t* __restrict__ targets,
                                                    const int64_t* __restrict__ m2l_off,
                                                    const int32_t* __restrict__ m2l_src,
                                                    const double* __restrict__ centre,
                                                    const int32_t* __restrict__ level, double side, int p, int nc,
                                                    int B, int CHUNK, const float* __restrict__ Q, float* L) {
  extern __shared__ __align__(16) float smem[];
  float* Qs = smem;                              // CHUNK x nc x SLICE
  float* bks = Qs + CHUNK * nc * SLICE;          // CHUNK x nc
  float* fps = bks + CHUNK * nc;                 // CHUNK x 16
  float* geo = fps + CHUNK * 16;                 // CHUNK x 4
  int* mi = (int*)(geo + CHUNK * 4);             // nc packed (a | b<<8 | c<<16 | t<<24)
  const int32_t T = targets[blockIdx.x];
  const int b0 = blockIdx.y * SLICE;
  const double sT = ldexp(side, -level[T]);
  const double cx = centre[3 * T], cy = centre[3 * T + 1], cz = centre[3 * T + 2];
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    int a, b, c;
    mi_decode(i, a, b, c);
    mi[i] = a | (b << 8) | (c << 16) | ((a + b + c) << 24);
  }
  // thread -> (row m, half of the slice)
  const int m = threadIdx.x % nc, half = threadIdx.x / nc;
  const bool active = threadIdx.x < 2 * nc;
  float acc[SPT];
#pragma unroll
  for (int r = 0; r < SPT; r++) acc[r] = 0.f;
  __syncthreads();
  const int mm = mi[active ? m : 0];
  const int ma = mm & 255, mb = (mm >> 8) & 255, mz = (mm >> 16) & 255, tm = mm >> 24;
  const int nmax = ncoef_of(p - tm);  // n runs over |n| <= p - |m|, a prefix of the graded order
  const int64_t e0 = m2l_off[T], e1 = m2l_off[T + 1];
  for (int64_t ec = e0; ec < e1; ec += CHUNK) {
    const int ns = (e1 - ec < CHUNK) ? (int)(e1 - ec) : CHUNK;
    __syncthreads();  // the previous chunk is consumed
    for (int q = threadIdx.x; q < ns * nc * SLICE; q += blockDim.x) {
      const int s = q / (nc * SLICE), r = q - s * nc * SLICE, n = r / SLICE, l = r - n * SLICE;
      const int32_t S = m2l_src[ec + s];
      Qs[q] = (b0 + l < B) ? Q[((int64_t)S * nc + n) * B + b0 + l] : 0.f;
    }
    if (threadIdx.x < ns) {
      const int32_t S = m2l_src[ec + threadIdx.x];
      const float x = (float)((cx - centre[3 * S]) / sT), y = (float)((cy - centre[3 * S + 1]) / sT),
                  z = (float)((cz - centre[3 * S + 2]) / sT);
      float* g = geo + 4 * threadIdx.x;
      g[0] = x;
      g[1] = y;
      g[2] = z;
      g[3] = x * x + y * y + z * z;
      bks[threadIdx.x * nc] = rsqrtf(g[3]);
      const int dl = level[T] - level[S];
      for (int t = 0; t <= p; t++) fps[threadIdx.x * 16 + t] = ldexpf(1.f, dl * t);
    }
    __syncthreads();
    for (int t = 1; t <= p; t++) {
      const int o = t * (t + 1) * (t + 2) / 6, cnt = (t + 1) * (t + 2) / 2;
      for (int q = threadIdx.x; q < ns * cnt; q += blockDim.x) {
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
    if (active) {
      for (int s = 0; s < ns; s++) {
        const float* bk = bks + s * nc;
        const float* fp = fps + s * 16;
        const float4* qs = (const float4*)(Qs + s * nc * SLICE + half * SPT);
        int n = 0;
        for (int t = 0; n < nmax; t++) {
          const float f = fp[t];
          const int tt = t + tm;
          const int base = tt * (tt + 1) * (tt + 2) / 6;
          for (int j = 0; j <= t; j++) {
            const int jb = j + mb + mz;  // (n_b + n_c) + (m_b + m_c)
            const int jbase = base + jb * (jb + 1) / 2 + mz;
            for (int c = 0; c <= j; c++, n++) {
              const float w = bk[jbase + c] * f;
              const float4* qn = qs + n * (SLICE / 4);
              const float4 q0 = qn[0], q1 = qn[1], q2 = qn[2], q3 = qn[3];
              acc[0] = fmaf(w, q0.x, acc[0]);
              acc[1] = fmaf(w, q0.y, acc[1]);
              acc[2] = fmaf(w, q0.z, acc[2]);
              acc[3] = fmaf(w, q0.w, acc[3]);
              acc[4] = fmaf(w, q1.x, acc[4]);
              acc[5] = fmaf(w, q1.y, acc[5]);
              acc[6] = fmaf(w, q1.z, acc[6]);
              acc[7] = fmaf(w, q1.w, acc[7]);
              acc[8] = fmaf(w, q2.x, acc[8]);
              acc[9] = fmaf(w, q2.y, acc[9]);
              acc[10] = fmaf(w, q2.z, acc[10]);
              acc[11] = fmaf(w, q2.w, acc[11]);
              acc[12] = fmaf(w, q3.x, acc[12]);
              acc[13] = fmaf(w, q3.y, acc[13]);
              acc[14] = fmaf(w, q3.z, acc[14]);
              acc[15] = fmaf(w, q3.w, acc[15]);
            }
          }
        }
      }
    }
  }
  if (!active) return;
  const float inv = (float)(1.0 / (4.0 * M_PI * sT));
  const float sg = (tm & 1) ? -inv : inv;
  (void)ma;
#pragma unroll
  for (int r = 0; r < SPT; r++) {
    const int b = b0 + half * SPT + r;
    if (b < B) L[((int64_t)T * nc + m) * B + b] = sg * acc[r];
  }
}

}  // namespace

bool launch_m2l32_fast(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s) {
  (void)err;
  if (P.h_m2l_targets.empty()) return true;
  const int nc = P.nc;
  const int threads = ((2 * nc + 31) / 32) * 32;
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(4, (200u << 10) / (sizeof(float) * nc * SLICE)));
  const size_t smem = sizeof(float) * (chunk * nc * SLICE + chunk * nc + chunk * 16 + chunk * 4) + sizeof(int) * nc;
  static size_t attr = 0;
  if (smem > attr) {
    DM_CUDA(cudaFuncSetAttribute(k_m2l32_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((B + SLICE - 1) / SLICE));
  k_m2l32_rows<<<grid, threads, smem, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, P.cell_level, P.side,
                                           P.p, nc, B, chunk, Q, L);
  DM_LAUNCH("k_m2l32_rows");
  return true;
}


// ---------------------------------------------------------------------------
// Table-driven FP32 M2L for small batches (k_m2l32_tab).
//
// The same sum, with b_k(v_S) read from a per-plan table: one row of nc FP32
// values per distinct translation key (dl, lattice offset), keyed as for the
// tensor-core M2L, so each pair costs a table row instead of the recurrence.
// Two facts shape the work.  Qt_0 = 0 (the degree-0 moment vanishes: P2M
// integrates gradients of the monomials), so n runs over degrees 1 .. p - |m|
// and the rows of degree p stay zero.  And the entries with |m| = tm, |n| = tn
// form a dense cnt(tm) x cnt(tn) block (cnt(t) = (t+1)(t+2)/2) whose values
// are the b_k of degree tm + tn: within a degree, the graded position of
// m + n is J(J+1)/2 + C with J = j_m + j_n, C = c_m + c_n (j = b + c).
//
// Layout: one CTA per (target, slice of SB states), SB = the batch rounded up
// to a power of two, at most 32.  Lane = (source slot j, state b), so a warp
// covers 32/SB sources at once and needs no broadcast between lanes.  Each
// warp owns a fixed set of row degrees (assigned at compile time, balanced on
// FMA count), keeps their accumulators in registers over all sources of the
// target, and runs its blocks fully unrolled with every multi-index position
// a compile-time constant: ~0.4 shared-memory loads per FMA.  Sources are
// staged 32/SB at a time (cp.async, two buffers; rows of odd length so the 32
// lanes' reads fall in distinct banks); f_S^|n| is applied to the staged
// moments of sources on another level.  At the end the lanes of a state add
// their per-source partial sums by a fixed shuffle tree, so results do not
// depend on timing.
namespace tab {

__host__ __device__ constexpr int cnt(int t) { return (t + 1) * (t + 2) / 2; }
__host__ __device__ constexpr int tri(int t) { return t * (t + 1) * (t + 2) / 6; }
__host__ __device__ constexpr int work(int p, int tm) { return cnt(tm) * (tri(p - tm + 1) - 1); }
__host__ __device__ constexpr int band_j(int r) {
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= r) j++;
  return j;
}
// position within degree tm + tn of (i-th multi-index of degree tm) + (j-th of degree tn)
__host__ __device__ constexpr int band_sum(int i, int j) {
  const int ji = band_j(i), jj = band_j(j);
  const int J = ji + jj, C = (i - ji * (ji + 1) / 2) + (j - jj * (jj + 1) / 2);
  return J * (J + 1) / 2 + C;
}

constexpr int MAXR = 4, MAXBLK = 24, MAXDEG = 12;

struct Roles {
  int nblk[MAXR] = {}, tm[MAXR][MAXBLK] = {}, tn[MAXR][MAXBLK] = {}, aoff[MAXR][MAXBLK] = {};
  int nacc[MAXR] = {}, ndeg[MAXR] = {}, deg[MAXR][MAXDEG] = {}, dacc[MAXR][MAXDEG] = {}, load[MAXR] = {};
};

// row degrees 0 .. p-1 to nr warps, heaviest first onto the least loaded warp;
// blocks ordered by column degree, then row degree
__host__ __device__ constexpr Roles make_roles(int p, int nr) {
  Roles R{};
  bool used[MAXDEG] = {};
  for (int it = 0; it < p; it++) {
    int best = -1;
    for (int t = 0; t < p; t++)
      if (!used[t] && (best < 0 || work(p, t) > work(p, best))) best = t;
    used[best] = true;
    int r = 0;
    for (int q = 1; q < nr; q++)
      if (R.load[q] < R.load[r]) r = q;
    R.load[r] += work(p, best);
    R.deg[r][R.ndeg[r]++] = best;
  }
  for (int r = 0; r < nr; r++) {
    for (int a = 1; a < R.ndeg[r]; a++)
      for (int b = a; b > 0 && R.deg[r][b - 1] > R.deg[r][b]; b--) {
        const int t = R.deg[r][b];
        R.deg[r][b] = R.deg[r][b - 1];
        R.deg[r][b - 1] = t;
      }
    for (int d = 0; d < R.ndeg[r]; d++) {
      R.dacc[r][d] = R.nacc[r];
      R.nacc[r] += cnt(R.deg[r][d]);
    }
    for (int tn = 1; tn <= p; tn++)
      for (int d = 0; d < R.ndeg[r]; d++)
        if (R.deg[r][d] + tn <= p) {
          const int k = R.nblk[r]++;
          R.tm[r][k] = R.deg[r][d];
          R.tn[r][k] = tn;
          R.aoff[r][k] = R.dacc[r][d];
        }
  }
  return R;
}

template <int V>
struct C_ {
  static constexpr int v = V;
};

// one dense block, column-major so consecutive FMAs go to different accumulators.
// f_S^tn is applied to whichever side is shorter: the cnt(tn) moments, or the
// cnt(tm) partial sums (these in R interleaved partials when cnt(tm) is small,
// to keep the dependent chains short).
template <int TM, int TN, int AOFF, int NA, int... IJ>
__device__ __forceinline__ void block_fmas(float (&acc)[NA], const float* __restrict__ bs,
                                           const float* __restrict__ qs, float fs, std::integer_sequence<int, IJ...>) {
  constexpr int CM = cnt(TM), CN = cnt(TN), BT = tri(TM + TN), QT = tri(TN);
  if constexpr (CM >= CN) {
    float q[CN];
#pragma unroll
    for (int j = 0; j < CN; j++) q[j] = qs[(QT + j) * 32] * fs;
    ((acc[AOFF + IJ % CM] = fmaf(bs[C_<BT + band_sum(IJ % CM, IJ / CM)>::v], q[IJ / CM], acc[AOFF + IJ % CM])), ...);
  } else {
    constexpr int R = CM == 1 ? 4 : (CM <= 3 ? 2 : 1);
    float t[CM * R];
#pragma unroll
    for (int i = 0; i < CM * R; i++) t[i] = 0.f;
    ((t[(IJ % CM) * R + (IJ / CM) % R] = fmaf(bs[C_<BT + band_sum(IJ % CM, IJ / CM)>::v], qs[(QT + IJ / CM) * 32],
                                              t[(IJ % CM) * R + (IJ / CM) % R])),
     ...);
#pragma unroll
    for (int i = 0; i < CM; i++) {
      float s = t[i * R];
#pragma unroll
      for (int r = 1; r < R; r++) s += t[i * R + r];
      acc[AOFF + i] = fmaf(fs, s, acc[AOFF + i]);
    }
  }
}

template <int P, int NR, int R, int BI, int NA>
__device__ __forceinline__ void role_blocks(float (&acc)[NA], const float* __restrict__ bs,
                                            const float* __restrict__ qs, const float (&fp)[P + 1]) {
  constexpr Roles RT = make_roles(P, NR);
  if constexpr (BI < RT.nblk[R]) {
    constexpr int TM = RT.tm[R][BI], TN = RT.tn[R][BI];
    block_fmas<TM, TN, RT.aoff[R][BI]>(acc, bs, qs, fp[TN], std::make_integer_sequence<int, cnt(TM) * cnt(TN)>{});
    role_blocks<P, NR, R, BI + 1>(acc, bs, qs, fp);
  }
}

// the target's rows of degree DEG(role, D): scale, sign and store
template <int P, int NR, int R, int D, int NA>
__device__ __forceinline__ void role_store(const float (&acc)[NA], float inv, float* L, int64_t row0, int B) {
  constexpr Roles RT = make_roles(P, NR);
  if constexpr (D < RT.ndeg[R]) {
    constexpr int TM = RT.deg[R][D], A0 = RT.dacc[R][D];
    const float sg = (TM & 1) ? -inv : inv;
#pragma unroll
    for (int i = 0; i < cnt(TM); i++) L[(row0 + tri(TM) + i) * B] = sg * acc[A0 + i];
    role_store<P, NR, R, D + 1>(acc, inv, L, row0, B);
  }
}

struct Ctx {
  const int32_t* src;
  const int32_t* opdl;  // per pair: key index | (dl & 255) << 24
  const float* tab;
  const float* Q;
  int64_t e0, e1;
  int B, b0, SB, lsb, NJ, nsteps;
};

// a lane's source for one step: slot j = lane >> lsb
struct Meta {
  int32_t S, opdl;
  bool valid;
};

__device__ __forceinline__ Meta load_meta(const Ctx& c, int s, int lane) {
  Meta m;
  const int64_t e = c.e0 + (int64_t)s * c.NJ + (lane >> c.lsb);
  m.valid = s < c.nsteps && e < c.e1;
  m.S = m.valid ? c.src[e] : 0;
  m.opdl = m.valid ? c.opdl[e] : 0;
  return m;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cta_sync(int nthreads) { asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory"); }

// stage one step into buf: NJ operator rows of RS floats (slot j at j RS), then
// the moments as nc rows of 32 lanes (n at NJ RS + 32 n, lane j SB + b).  Warp
// w copies the operator rows of slots w, w + NR, ...; every lane copies its own
// moments for n = w, w + NR, ...  The slots' keys come from the lanes that own
// them (lane j SB).
template <int P, int NR>
__device__ __forceinline__ void stage(const Ctx& c, const Meta& m, float* buf, int warp, int lane) {
  constexpr int NC = tri(P + 1), RS = NC | 1;
  for (int j = warp; j < c.NJ; j += NR) {
    const int opdl = __shfl_sync(0xffffffffu, m.opdl, j << c.lsb);
    const bool valid = __shfl_sync(0xffffffffu, (int)m.valid, j << c.lsb) != 0;
    float* brow = buf + j * RS;
    if (valid) {
      const float* trow = c.tab + (int64_t)(opdl & 0xFFFFFF) * NC;
      for (int k = lane; k < NC; k += 32) cp_async4(brow + k, trow + k);
    } else {
      for (int k = lane; k < NC; k += 32) brow[k] = 0.f;
    }
  }
  float* qcol = buf + c.NJ * RS + lane;
  const int b = lane & (c.SB - 1);
  if (m.valid && c.b0 + b < c.B) {
    const float* q = c.Q + (int64_t)m.S * NC * c.B + c.b0 + b;
    for (int n = warp; n < NC; n += NR) cp_async4(qcol + 32 * n, q + (int64_t)n * c.B);
  } else {
    for (int n = warp; n < NC; n += NR) qcol[32 * n] = 0.f;
  }
}

template <int P, int NR, int R>
__device__ __forceinline__ void role_run(const Ctx& c, float* sm, float* L, int32_t T, float inv) {
  constexpr int NC = tri(P + 1), RS = NC | 1;
  constexpr Roles RT = make_roles(P, NR);
  constexpr int NA = RT.nacc[R] > 0 ? RT.nacc[R] : 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int bufsz = c.NJ * RS + 32 * NC;
  float acc[NA];
#pragma unroll
  for (int i = 0; i < NA; i++) acc[i] = 0.f;
  Meta cur = load_meta(c, 0, lane);
  Meta nxt = load_meta(c, 1, lane);
  stage<P, NR>(c, cur, sm, warp, lane);
  cp_async_commit();
  const int j = lane >> c.lsb;
  for (int s = 0; s < c.nsteps; s++) {
    cp_async_wait_all();
    cta_sync(32 * NR);  // step s staged; step s - 1 consumed by every warp
    const float* buf = sm + (s & 1) * bufsz;
    if (s + 1 < c.nsteps) stage<P, NR>(c, nxt, sm + ((s + 1) & 1) * bufsz, warp, lane);
    cp_async_commit();
    const Meta after = load_meta(c, s + 2, lane);  // consumed by the next step's staging
    // f_S^t = 2^(dl t), exact powers of two
    float fp[P + 1];
    fp[0] = 1.f;
    fp[1] = ldexpf(1.f, cur.opdl >> 24);
#pragma unroll
    for (int t = 2; t <= P; t++) fp[t] = fp[t - 1] * fp[1];
    role_blocks<P, NR, R, 0>(acc, buf + j * RS, buf + c.NJ * RS + lane, fp);
    cur = nxt;
    nxt = after;
  }
  // sum over the source slots of each state (lanes b, b + SB, ...)
  for (int o = c.SB; o < 32; o <<= 1) {
#pragma unroll
    for (int i = 0; i < NA; i++) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  }
  if (lane < c.SB && c.b0 + lane < c.B) role_store<P, NR, R, 0>(acc, inv, L + c.b0 + lane, (int64_t)T * NC, c.B);
}

template <int P, int NR>
__global__ void __launch_bounds__(32 * NR) k_m2l32_tab(const int32_t* __restrict__ targets,
                                                       const int64_t* __restrict__ m2l_off,
                                                       const int32_t* __restrict__ m2l_src,
                                                       const int32_t* __restrict__ m2l_opdl,
                                                       const float* __restrict__ tab,
                                                       const int32_t* __restrict__ level, double side, int B,
                                                       int lsb, const float* __restrict__ Q, float* L) {
  extern __shared__ __align__(16) float sm[];
  const int32_t T = targets[blockIdx.x];
  Ctx c;
  c.src = m2l_src;
  c.opdl = m2l_opdl;
  c.tab = tab;
  c.Q = Q;
  c.e0 = m2l_off[T];
  c.e1 = m2l_off[T + 1];
  c.B = B;
  c.lsb = lsb;
  c.SB = 1 << lsb;
  c.NJ = 32 >> lsb;
  c.b0 = blockIdx.y * c.SB;
  c.nsteps = (int)((c.e1 - c.e0 + c.NJ - 1) / c.NJ);
  const float inv = (float)(1.0 / (4.0 * M_PI * ldexp(side, -level[T])));
  const int warp = threadIdx.x >> 5;
  if (warp == 0) role_run<P, NR, 0>(c, sm, L, T, inv);
  if constexpr (NR > 1) if (warp == 1) role_run<P, NR, 1>(c, sm, L, T, inv);
  if constexpr (NR > 2) if (warp == 2) role_run<P, NR, 2>(c, sm, L, T, inv);
  if constexpr (NR > 3) if (warp == 3) role_run<P, NR, 3>(c, sm, L, T, inv);
}

// b_k(v) for one key per block, FP64 recurrence, rounded to FP32
__global__ void __launch_bounds__(128) k_m2l_tab_ops(const int4* __restrict__ keys, int p, int nc, float* tab) {
  __shared__ double b[MAX_NCOEF];
  const int4 key = keys[blockIdx.x];
  const int dl = key.x;
  const double sc = ldexp(1.0, -((dl < 0 ? -dl : 0) + 1));
  const double vx = key.y * sc, vy = key.z * sc, vz = key.w * sc, r2 = vx * vx + vy * vy + vz * vz;
  if (threadIdx.x == 0) b[0] = 1.0 / sqrt(r2);
  __syncthreads();
  // b_k = (-1)^|k| d^k (1/|x|) at v:  |k| r^2 b_k = (2|k|-1) sum k_i v_i b_{k-e_i} - (|k|-1) sum k_i (k_i-1) b_{k-2e_i}
  for (int t = 1; t <= p; t++) {
    for (int k = tri(t) + threadIdx.x; k < tri(t + 1); k += blockDim.x) {
      int ka, kb, kz;
      mi_decode(k, ka, kb, kz);
      double s1 = 0.0, s2 = 0.0;
      if (ka) s1 += ka * vx * b[mi_index(ka - 1, kb, kz)];
      if (kb) s1 += kb * vy * b[mi_index(ka, kb - 1, kz)];
      if (kz) s1 += kz * vz * b[mi_index(ka, kb, kz - 1)];
      if (ka > 1) s2 += ka * (ka - 1) * b[mi_index(ka - 2, kb, kz)];
      if (kb > 1) s2 += kb * (kb - 1) * b[mi_index(ka, kb - 2, kz)];
      if (kz > 1) s2 += kz * (kz - 1) * b[mi_index(ka, kb, kz - 2)];
      b[k] = ((2 * t - 1) * s1 - (t - 1) * s2) / (t * r2);
    }
    __syncthreads();
  }
  for (int k = threadIdx.x; k < nc; k += blockDim.x) tab[(int64_t)blockIdx.x * nc + k] = (float)b[k];
}

constexpr bool tab_order(int p) { return p == 4 || p == 6 || p == 8; }
constexpr int tab_warps(int) { return 4; }

template <int P>
size_t tab_smem(int lsb) {
  constexpr int NC = tri(P + 1), RS = NC | 1;
  return sizeof(float) * 2 * (size_t)((32 >> lsb) * RS + 32 * NC);
}

template <int P>
void launch_tab(Plan& P_, int B, const float* Q, float* L, cudaStream_t s) {
  constexpr int NR = tab_warps(P);
  int lsb = 0;
  while ((1 << lsb) < B && lsb < 5) lsb++;
  const size_t smem = tab_smem<P>(lsb);
  static size_t attr = 0;
  if (smem > attr) {
    DM_CUDA(cudaFuncSetAttribute(k_m2l32_tab<P, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tab_smem<P>(0)));
    attr = tab_smem<P>(0);
  }
  const dim3 grid((unsigned)P_.h_m2l_targets.size(), (unsigned)((B + (1 << lsb) - 1) >> lsb));
  k_m2l32_tab<P, NR><<<grid, 32 * NR, smem, s>>>(P_.m2l_targets, P_.m2l_off, P_.m2l_src, P_.m2l_tab_opdl, P_.m2l_tab,
                                                 P_.cell_level, P_.side, B, lsb, Q, L);
  DM_LAUNCH("k_m2l32_tab");
}

}  // namespace tab

void build_m2l_tab(Plan& P, const M2lKeys& K) {
  if (!K.ok || !tab::tab_order(P.p) || K.keys.empty() || K.keys.size() >= (1u << 24)) return;
  std::vector<int32_t> opdl(K.op.size());
  for (size_t e = 0; e < K.op.size(); e++) {
    const int dl = K.keys[K.op[e]].x;
    if (dl < -128 || dl > 127) return;
    opdl[e] = K.op[e] | (int32_t)((uint32_t)(dl & 255) << 24);
  }
  cudaStream_t s = P.stream;
  P.m2l_tab_opdl = dalloc<int32_t>(P, opdl.size());
  DM_CUDA(cudaMemcpyAsync(P.m2l_tab_opdl, opdl.data(), opdl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  P.m2l_tab = dalloc<float>(P, K.keys.size() * (size_t)P.nc);
  int4* dkeys = nullptr;
  if (cudaMalloc(&dkeys, K.keys.size() * sizeof(int4)) != cudaSuccess) {
    cudaGetLastError();
    fail(DEMAG_ERR_OUT_OF_MEMORY, "M2L table temporary allocation failed");
  }
  cudaError_t e = cudaMemcpyAsync(dkeys, K.keys.data(), K.keys.size() * sizeof(int4), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    tab::k_m2l_tab_ops<<<(unsigned)K.keys.size(), 128, 0, s>>>(dkeys, P.p, P.nc, P.m2l_tab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dkeys);
  if (e != cudaSuccess) fail(DEMAG_ERR_CUDA, std::string("M2L table build: ") + cudaGetErrorString(e));
}

bool launch_m2l32_tab(Plan& P, int B, const float* Q, float* L, cudaStream_t s) {
  if (P.m2l_tab == nullptr || P.m2l_tab_opdl == nullptr) return false;
  if (P.h_m2l_targets.empty()) return true;
  switch (P.p) {
    case 4: tab::launch_tab<4>(P, B, Q, L, s); return true;
    case 6: tab::launch_tab<6>(P, B, Q, L, s); return true;
    case 8: tab::launch_tab<8>(P, B, Q, L, s); return true;
    default: return false;
  }
}

}  // namespace demag
