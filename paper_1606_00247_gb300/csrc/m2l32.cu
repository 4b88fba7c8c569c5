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
  smem_opt_in((const void*)k_m2l32_rows, smem);
  dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((B + SLICE - 1) / SLICE));
  k_m2l32_rows<<<grid, threads, smem, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, P.cell_level, P.side,
                                           P.p, nc, B, chunk, Q, L);
  DM_LAUNCH("k_m2l32_rows");
  return true;
}


// ---------------------------------------------------------------------------
// Table-driven FP32 M2L for small batches (k_m2l32_rc).
//
// The same sum, with b_k(v_S) read from a per-plan table: one row of nc FP32
// values per distinct translation key (dl, lattice offset), keyed as for the
// tensor-core M2L, so a pair costs a table row instead of the recurrence.
// Qt_0 = 0 (the degree-0 moment vanishes: P2M integrates gradients of the
// monomials), so n runs over 1 <= n < C(p - |m| + 3, 3) and the rows of degree
// p have no terms.
//
// Thread = work item (row m, chunk c of CH consecutive n in the graded order):
// it owns the accumulators of row m for the SB <= 8 states of its slice and
// adds, over every source of the target, b_{m+n} f^|n| Qt_n for the n of its
// chunk.  The CH table positions of b_{m+n} are computed once and held in
// registers; items are ordered chunk-major, so the lanes of a warp read the
// same moments (shared-memory broadcast, SB states as float4s) and gather b
// from one table row.  No position is a compile-time constant, so the code is
// small: a fully unrolled variant with one source per lane and compile-time
// positions was bound by instruction fetch (~16 KB of straight-line code per
// warp).  KS = 8 sources are staged per step by eight warps (cp.async, two
// buffers, each warp's next two sources prefetched in registers); f_S^|n| is
// applied in shared memory to the staged moments of sources on another level.
// The chunks of a row are added in a fixed order at the end, so results do
// not depend on timing.
namespace rc {

constexpr int KS = 8;  // sources per step

// (m, c) items of order p with chunk length ch, chunk-major: m | c << 16
std::vector<uint32_t> items(int p, int ch) {
  std::vector<uint32_t> it;
  const int nc = ncoef_of(p);
  for (int c = 0; c * ch < nc; c++)
    for (int m = 0; m < nc; m++) {
      int a, b, z;
      mi_decode(m, a, b, z);
      const int t = a + b + z, nmax = t < p ? ncoef_of(p - t) : 0;  // n < nmax, n >= 1
      const int lo = std::max(1, c * ch), hi = std::min(nmax, (c + 1) * ch);
      if (lo < hi) it.push_back((uint32_t)m | ((uint32_t)c << 16));
    }
  return it;
}

__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// one buffer: KS operator rows (nc floats), KS moment blocks (nc x SB floats), KS level differences
template <int SB>
__host__ __device__ constexpr size_t buf_floats(int nc) {
  return (size_t)KS * nc * (1 + SB) + KS;
}

template <int CH, int SB>
__global__ void __launch_bounds__(1024) k_m2l32_rc(const int32_t* __restrict__ targets,
                                                   const int64_t* __restrict__ m2l_off,
                                                   const int32_t* __restrict__ m2l_src,
                                                   const int32_t* __restrict__ m2l_opdl,
                                                   const float* __restrict__ tab, const uint32_t* __restrict__ items,
                                                   int nitems, const int32_t* __restrict__ level, double side, int p,
                                                   int nc, int B, const float* __restrict__ Q, float* L) {
  extern __shared__ __align__(16) float sm[];
  const int32_t T = targets[blockIdx.x];
  const int b0 = blockIdx.y * SB, nlive = min(SB, B - b0);
  const bool vec = SB % 4 == 0 && nlive == SB && B % 4 == 0;
  const int64_t e0 = m2l_off[T], nsrc = m2l_off[T + 1] - e0;
  const int nsteps = (int)((nsrc + KS - 1) / KS);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t bufsz = buf_floats<SB>(nc);
  int* deg = (int*)(sm + 2 * bufsz);  // degree of every n
  for (int n = tid; n < nc; n += blockDim.x) {
    int a, b, z;
    mi_decode(n, a, b, z);
    deg[n] = a + b + z;
  }
  // this thread's row and table positions
  const bool has = tid < nitems;
  const uint32_t it = has ? items[tid] : 0u;
  const int m = (int)(it & 0xFFFFu), c = (int)(it >> 16);
  int ma, mb, mz;
  mi_decode(m, ma, mb, mz);
  const int nmax = has && ma + mb + mz < p ? ncoef_of(p - ma - mb - mz) : 0;
  int idx[CH];
  bool ok[CH];
#pragma unroll
  for (int j = 0; j < CH; j++) {
    const int n = c * CH + j;
    ok[j] = n >= 1 && n < nmax;
    int na = 0, nb = 0, nz = 0;
    if (ok[j]) mi_decode(n, na, nb, nz);
    idx[j] = ok[j] ? mi_index(ma + na, mb + nb, mz + nz) : 0;
  }
  float acc[SB];
#pragma unroll
  for (int b = 0; b < SB; b++) acc[b] = 0.f;
  // staging: warp w < KS owns source slot w of every step
  auto meta = [&](int s, int k, int32_t& S, int32_t& od) {
    const int64_t e = (int64_t)s * KS + k;
    const bool v = s < nsteps && e < nsrc;
    S = v ? m2l_src[e0 + e] : -1;
    od = v ? m2l_opdl[e0 + e] : 0;
  };
  auto stage = [&](float* buf, int k, int32_t S, int32_t od) {
    float* brow = buf + (size_t)k * nc;
    float* qblk = buf + (size_t)KS * nc + (size_t)k * nc * SB;
    if (S < 0) {
      for (int i = lane; i < nc; i += 32) brow[i] = 0.f;
      for (int i = lane; i < nc * SB; i += 32) qblk[i] = 0.f;
      if (lane == 0) buf[(size_t)KS * nc * (1 + SB) + k] = 0.f;
      return;
    }
    const float* trow = tab + (int64_t)(od & 0xFFFFFF) * nc;
    for (int i = lane; i < nc; i += 32) cp_async4(brow + i, trow + i);
    const float* q = Q + (int64_t)S * nc * B + b0;
    bool done = false;
    if constexpr (SB % 4 == 0) {
      if (vec) {
        for (int i = lane; i < nc * (SB / 4); i += 32) {
          const int n = i / (SB / 4), v4 = i % (SB / 4);
          cp_async16(qblk + n * SB + 4 * v4, q + (int64_t)n * B + 4 * v4);
        }
        done = true;
      }
    }
    if (!done)
      for (int i = lane; i < nc * SB; i += 32) {
        const int n = i / SB, b = i % SB;
        if (b < nlive)
          cp_async4(qblk + i, q + (int64_t)n * B + b);
        else
          qblk[i] = 0.f;
      }
    if (lane == 0) buf[(size_t)KS * nc * (1 + SB) + k] = (float)(od >> 24);  // level difference
  };
  int32_t S0 = -1, od0 = 0, S1 = -1, od1 = 0;
  const int kw = warp < KS ? warp : -1;
  if (kw >= 0) {
    meta(0, kw, S0, od0);
    meta(1, kw, S1, od1);
  }
  __syncthreads();  // degrees
  if (kw >= 0) stage(sm, kw, S0, od0);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int s = 0; s < nsteps; s++) {
    float* buf = sm + (size_t)(s & 1) * bufsz;
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();  // step s staged; step s - 1 consumed
    // f_S^|n| = 2^(dl |n|) on the staged moments of sources on another level
    const float* dls = buf + (size_t)KS * nc * (1 + SB);
    for (int k = 0; k < KS; k++) {
      const int dl = (int)dls[k];
      if (dl == 0) continue;
      float* qblk = buf + (size_t)KS * nc + (size_t)k * nc * SB;
      for (int i = tid; i < nc * SB; i += blockDim.x) qblk[i] = ldexpf(qblk[i], dl * deg[i / SB]);
    }
    int32_t S2 = -1, od2 = 0;
    if (kw >= 0) {
      if (s + 1 < nsteps) stage(sm + (size_t)((s + 1) & 1) * bufsz, kw, S1, od1);
      meta(s + 2, kw, S2, od2);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    __syncthreads();  // scaled moments visible
    if (has) {
#pragma unroll 1
      for (int k = 0; k < KS; k++) {
        const float* bs = buf + (size_t)k * nc;
        const float* qs = buf + (size_t)KS * nc + (size_t)k * nc * SB + (size_t)c * CH * SB;
#pragma unroll
        for (int j = 0; j < CH; j++) {
          if (!ok[j]) continue;
          const float bv = bs[idx[j]];
          if constexpr (SB % 4 == 0) {
#pragma unroll
            for (int v4 = 0; v4 < SB / 4; v4++) {
              const float4 q4 = *(const float4*)(qs + j * SB + 4 * v4);
              acc[4 * v4] = fmaf(bv, q4.x, acc[4 * v4]);
              acc[4 * v4 + 1] = fmaf(bv, q4.y, acc[4 * v4 + 1]);
              acc[4 * v4 + 2] = fmaf(bv, q4.z, acc[4 * v4 + 2]);
              acc[4 * v4 + 3] = fmaf(bv, q4.w, acc[4 * v4 + 3]);
            }
          } else {
#pragma unroll
            for (int b = 0; b < SB; b++) acc[b] = fmaf(bv, qs[j * SB + b], acc[b]);
          }
        }
      }
    }
    S1 = S2;
    od1 = od2;
  }
  // add the chunks of each row in chunk order: partial sums staged in shared memory
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  float* part = sm;  // nitems x SB
  if (has)
#pragma unroll
    for (int b = 0; b < SB; b++) part[tid * SB + b] = acc[b];
  __syncthreads();
  const float inv = (float)(1.0 / (4.0 * M_PI * ldexp(side, -level[T])));
  // the items of row mm, in chunk order: rowitem[rowoff[mm] .. rowoff[mm + 1])
  const uint32_t* rowoff = items + nitems;
  const uint32_t* rowitem = rowoff + nc + 1;
  for (int q = tid; q < nc * SB; q += blockDim.x) {
    const int mm = q / SB, b = q % SB;
    if (b >= nlive) continue;
    float v = 0.f;
    for (uint32_t i = rowoff[mm]; i < rowoff[mm + 1]; i++) v += part[rowitem[i] * SB + b];
    int a2, b2, z2;
    mi_decode(mm, a2, b2, z2);
    L[((int64_t)T * nc + mm) * B + b0 + b] = ((a2 + b2 + z2) & 1) ? -inv * v : inv * v;
  }
}

template <int CH, int SB>
void launch_rc(Plan& P, int B, const float* Q, float* L, cudaStream_t s) {
  const int nthreads = std::max(32 * KS, (P.m2l_rc_nitems + 31) / 32 * 32);  // every source slot has a warp
  const size_t smem = std::max(sizeof(float) * 2 * buf_floats<SB>(P.nc) + sizeof(int) * P.nc,
                               sizeof(float) * (size_t)nthreads * SB);
  smem_opt_in((const void*)k_m2l32_rc<CH, SB>, smem);
  const dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((B + SB - 1) / SB));
  k_m2l32_rc<CH, SB><<<grid, nthreads, smem, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.m2l_tab_opdl, P.m2l_tab,
                                                  P.m2l_rc_items, P.m2l_rc_nitems, P.cell_level, P.side, P.p, P.nc, B,
                                                  Q, L);
  DM_LAUNCH("k_m2l32_rc");
}

template <int CH>
void launch_rc_ch(Plan& P, int B, const float* Q, float* L, cudaStream_t s) {
  if (B == 1)
    launch_rc<CH, 1>(P, B, Q, L, s);
  else if (B == 2)
    launch_rc<CH, 2>(P, B, Q, L, s);
  else if (B <= 4)
    launch_rc<CH, 4>(P, B, Q, L, s);
  else
    launch_rc<CH, 8>(P, B, Q, L, s);
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
    for (int k = ncoef_of(t - 1) + threadIdx.x; k < ncoef_of(t); k += blockDim.x) {
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


}  // namespace rc

void build_m2l_tab(Plan& P, const M2lKeys& K) {
  if (!K.ok || K.keys.empty() || K.keys.size() >= (1u << 24)) return;
  if (P.p > 10) return;  // two staging buffers of 8 sources x 8 states exceed shared memory
  std::vector<int32_t> opdl(K.op.size());
  for (size_t e = 0; e < K.op.size(); e++) {
    const int dl = K.keys[K.op[e]].x;
    if (dl < -128 || dl > 127) return;
    opdl[e] = K.op[e] | (int32_t)((uint32_t)(dl & 255) << 24);
  }
  // work items: the shortest chunk (8, 16, 32) with at most 1024 items, then per row the
  // list of its items in chunk order (CSR)
  std::vector<uint32_t> it;
  int ch = 0;
  for (int c : {8, 16, 32}) {
    it = rc::items(P.p, c);
    if (it.size() <= 1024) {
      ch = c;
      break;
    }
  }
  if (!ch) return;
  const int nit = (int)it.size();
  std::vector<uint32_t> rows(nit + P.nc + 1 + nit);
  std::copy(it.begin(), it.end(), rows.begin());
  std::vector<uint32_t> cntr(P.nc + 1, 0);
  for (uint32_t v : it) cntr[(v & 0xFFFFu) + 1]++;
  for (int m = 0; m < P.nc; m++) cntr[m + 1] += cntr[m];
  std::copy(cntr.begin(), cntr.end(), rows.begin() + nit);
  std::vector<uint32_t> fill(cntr.begin(), cntr.end() - 1);
  for (int i = 0; i < nit; i++) rows[nit + P.nc + 1 + fill[it[i] & 0xFFFFu]++] = (uint32_t)i;
  cudaStream_t s = P.stream;
  P.m2l_rc_items = dalloc<uint32_t>(P, rows.size());
  P.m2l_rc_nitems = nit;
  P.m2l_rc_ch = ch;
  DM_CUDA(cudaMemcpyAsync(P.m2l_rc_items, rows.data(), rows.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
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
    rc::k_m2l_tab_ops<<<(unsigned)K.keys.size(), 128, 0, s>>>(dkeys, P.p, P.nc, P.m2l_tab);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(dkeys);
  if (e != cudaSuccess) fail(DEMAG_ERR_CUDA, std::string("M2L table build: ") + cudaGetErrorString(e));
}

bool launch_m2l32_tab(Plan& P, int B, const float* Q, float* L, cudaStream_t s) {
  if (P.m2l_tab == nullptr || P.m2l_tab_opdl == nullptr || P.m2l_rc_items == nullptr) return false;
  if (P.h_m2l_targets.empty()) return true;
  switch (P.m2l_rc_ch) {
    case 8: rc::launch_rc_ch<8>(P, B, Q, L, s); return true;
    case 16: rc::launch_rc_ch<16>(P, B, Q, L, s); return true;
    case 32: rc::launch_rc_ch<32>(P, B, Q, L, s); return true;
    default: return false;
  }
}

}  // namespace demag
