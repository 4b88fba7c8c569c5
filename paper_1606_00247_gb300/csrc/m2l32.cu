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

}  // namespace demag
