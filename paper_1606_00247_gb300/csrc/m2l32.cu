// m2l32.cu -- FP32 M2L on CUDA cores for batches of states (mixed path).
//
//   Lt^T_m = (-1)^|m| / (4 pi s_T) sum_S sum_{|n| <= p - |m|} b_{n+m}(v_S) f_S^|n| Qt^S_n
// (v_S = (c_T - c_S)/s_T, f_S = s_S/s_T, notation of fmm32.cu).
//
// Work layout.  One block per (target cell, slice of 32*SPL states); lane =
// SPL consecutive states.  Row m of the output has C(p - |m| + 3, 3) terms
// (1 ... 165 at p = 8), so rows are bin-packed on the host into NW warp
// schedules of at most RMAX rows with nearly equal term counts; a warp walks
// n in graded order once per source and updates all of its rows, so every
// operator value b_{n+m} (a warp-uniform shared-memory broadcast) feeds SPL
// FMAs, every moment vector Q_n[lane states] is loaded once per n, and no lane
// of a warp diverges from the others.  Source moments are staged in shared
// memory one source ahead with TMA bulk copies; the operator vectors b_k(v)
// of 8 sources at a time are built by the block with the Taylor-coefficient
// recurrence of 1/|x|.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace demag {

namespace {

constexpr int NW = 16;     // warps per block
constexpr int RMAX = 12;   // rows per warp (NW * RMAX >= 165 rows at p = 8)
constexpr int BCH = 8;     // sources per operator batch

__device__ __forceinline__ int tri3(int t) { return t * (t + 1) * (t + 2) / 6; }
__device__ __forceinline__ int tri2(int j) { return j * (j + 1) / 2; }
__device__ __forceinline__ int idx3(int a, int b, int c) { return tri3(a + b + c) + tri2(b + c) + c; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
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
    if (it > 64) __nanosleep(32);
  }
  return false;
}

// one row's description, packed: tm | sm<<4 | mz<<8 | (number of n terms)<<12 | m<<21
struct RowInfo {
  int tm, sm, mz, w, m;
};
__device__ __forceinline__ RowInfo unpack(int v) {
  return RowInfo{v & 15, (v >> 4) & 15, (v >> 8) & 15, (v >> 12) & 511, v >> 21};
}

template <int SPL>
__global__ void __launch_bounds__(NW * 32, 1) k_m2l32_v3(const int32_t* __restrict__ targets,
                                                       const int64_t* __restrict__ m2l_off,
                                                       const int32_t* __restrict__ m2l_src,
                                                       const double* __restrict__ centre,
                                                       const int32_t* __restrict__ level, double side, int p, int nc,
                                                       int B, const int* __restrict__ sched,
                                                       const float* __restrict__ Q, float* L, int* err) {
  constexpr int SLICE = 32 * SPL;
  extern __shared__ __align__(128) float smem[];
  float* Qs = smem;                        // 2 x nc x SLICE (double buffer)
  float* bks = Qs + 2 * nc * SLICE;        // BCH x nc
  float* fps = bks + BCH * nc;             // BCH x 16
  float* geo = fps + BCH * 16;             // BCH x 4
  int* srow = (int*)(geo + BCH * 4);       // NW x RMAX packed rows (0 = empty)
  int* mi = srow + NW * RMAX;              // nc packed multi-indices
  uint64_t* bar = (uint64_t*)(mi + ((nc + 3) & ~3));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int32_t T = targets[blockIdx.x];
  const int b0 = blockIdx.y * SLICE;
  const double sT = ldexp(side, -level[T]);
  const double cx = centre[3 * T], cy = centre[3 * T + 1], cz = centre[3 * T + 2];
  for (int i = threadIdx.x; i < nc; i += blockDim.x) {
    int a, b, c;
    mi_decode(i, a, b, c);
    mi[i] = a | (b << 8) | (c << 16);
  }
  for (int i = threadIdx.x; i < NW * RMAX; i += blockDim.x) srow[i] = sched[i];
  if (threadIdx.x == 0) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
  }
  float acc[RMAX][SPL];
#pragma unroll
  for (int r = 0; r < RMAX; r++)
#pragma unroll
    for (int k = 0; k < SPL; k++) acc[r][k] = 0.f;
  const int64_t e0 = m2l_off[T], e1 = m2l_off[T + 1];
  const bool whole = (b0 == 0 && B == SLICE);  // the slice is contiguous in global memory
  auto issue = [&](int64_t e, int buf) {       // stage the moments of source e (thread 0)
    const int32_t S = m2l_src[e];
    const float* src = Q + (int64_t)S * nc * B + b0;
    if (whole) {
      mbar_expect(&bar[buf], (uint32_t)(nc * SLICE * sizeof(float)));
      bulk_g2s(Qs + buf * nc * SLICE, src, (uint32_t)(nc * SLICE * sizeof(float)), &bar[buf]);
    } else {
      const int w = min(SLICE, B - b0);  // states present in this slice
      const uint32_t bytes = (uint32_t)(((w * sizeof(float)) + 15) & ~size_t(15));
      mbar_expect(&bar[buf], (uint32_t)(nc * bytes));
      for (int n = 0; n < nc; n++) bulk_g2s(Qs + (buf * nc + n) * SLICE, src + (int64_t)n * B, bytes, &bar[buf]);
    }
  };
  __syncthreads();
  if (threadIdx.x == 0 && e1 > e0) issue(e0, 0);
  uint32_t ph0 = 0, ph1 = 0;
  for (int64_t ec = e0; ec < e1; ec += BCH) {
    const int ns = (e1 - ec < BCH) ? (int)(e1 - ec) : BCH;
    // operator vectors of this batch of sources
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
      const int o = tri3(t), cnt = (t + 1) * (t + 2) / 2;
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
    for (int s = 0; s < ns; s++) {
      const int64_t e = ec + s;
      const int buf = (int)((e - e0) & 1);
      // prefetch the next source into the other buffer (released by the sync at the end of the previous step)
      if (threadIdx.x == 0 && e + 1 < e1) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        issue(e + 1, buf ^ 1);
      }
      const uint32_t ph = buf ? ph1 : ph0;
      if (!mbar_wait(&bar[buf], ph)) {
        if (threadIdx.x == 0) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
        mbar_wait(&bar[buf], ph);
        return;
      }
      if (buf)
        ph1 ^= 1;
      else
        ph0 ^= 1;
      const float* bk = bks + s * nc;
      const float* fp = fps + s * 16;
      const float* qb = Qs + buf * nc * SLICE + lane * SPL;
      const int* myrows = srow + warp * RMAX;
      int n = 0;
      for (int t = 0; t <= p; t++) {
        const float f = fp[t];
        for (int j = 0; j <= t; j++) {
          int base[RMAX];
#pragma unroll
          for (int r = 0; r < RMAX; r++) {
            const RowInfo ri = unpack(myrows[r]);
            base[r] = tri3(t + ri.tm) + tri2(j + ri.sm) + ri.mz;
          }
          for (int c = 0; c <= j; c++, n++) {
            float q[SPL];
            if constexpr (SPL == 4) {
              const float4 v = *(const float4*)(qb + n * SLICE);
              q[0] = v.x * f;
              q[1] = v.y * f;
              q[2] = v.z * f;
              q[3] = v.w * f;
            } else {
#pragma unroll
              for (int k = 0; k < SPL; k++) q[k] = qb[n * SLICE + k] * f;
            }
#pragma unroll
            for (int r = 0; r < RMAX; r++) {
              const int v = myrows[r];
              if (((v >> 12) & 511) > n) {  // row r still has terms at this n (warp-uniform)
                const float w = bk[base[r] + c];
#pragma unroll
                for (int k = 0; k < SPL; k++) acc[r][k] = fmaf(w, q[k], acc[r][k]);
              }
            }
          }
        }
      }
      __syncthreads();  // buffer `buf` is free again
    }
  }
  const float inv = (float)(1.0 / (4.0 * M_PI * sT));
  const int* myrows = srow + warp * RMAX;
#pragma unroll
  for (int r = 0; r < RMAX; r++) {
    const int v = myrows[r];
    if (v == 0) continue;
    const RowInfo ri = unpack(v);
    const float sg = (ri.tm & 1) ? -inv : inv;
#pragma unroll
    for (int k = 0; k < SPL; k++) {
      const int b = b0 + lane * SPL + k;
      if (b < B) L[((int64_t)T * nc + ri.m) * B + b] = sg * acc[r][k];
    }
  }
}

// bin-pack the rows of order p into NW warps of <= RMAX rows with balanced term counts
std::vector<int> make_schedule(int p) {
  const int nc = ncoef_of(p);
  std::vector<int> rows(nc);
  for (int m = 0; m < nc; m++) rows[m] = m;
  auto work = [&](int m) {
    int a, b, c;
    mi_decode(m, a, b, c);
    return ncoef_of(p - (a + b + c));
  };
  std::stable_sort(rows.begin(), rows.end(), [&](int x, int y) { return work(x) > work(y); });
  std::vector<int> load(NW, 0), count(NW, 0), sched(NW * RMAX, 0);
  for (int m : rows) {
    int best = -1;
    for (int w = 0; w < NW; w++)
      if (count[w] < RMAX && (best < 0 || load[w] < load[best])) best = w;
    if (best < 0) return {};
    int a, b, c;
    mi_decode(m, a, b, c);
    const int wk = work(m);
    sched[best * RMAX + count[best]++] = (a + b + c) | ((b + c) << 4) | (c << 8) | (wk << 12) | (m << 21);
    load[best] += wk;
  }
  // rows of a warp in decreasing term count (the row test then fails for a suffix)
  for (int w = 0; w < NW; w++)
    std::stable_sort(sched.begin() + w * RMAX, sched.begin() + w * RMAX + count[w],
                     [](int x, int y) { return ((x >> 12) & 511) > ((y >> 12) & 511); });
  return sched;
}

template <int SPL>
void launch_v3(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s, const int* sched) {
  const int nc = P.nc;
  constexpr int SLICE = 32 * SPL;
  const size_t smem = sizeof(float) * (2 * nc * SLICE + BCH * nc + BCH * 16 + BCH * 4) +
                      sizeof(int) * (NW * RMAX + ((nc + 3) & ~3)) + 2 * sizeof(uint64_t) + 16;
  static size_t attr = 0;
  if (smem > attr) {
    DM_CUDA(cudaFuncSetAttribute(k_m2l32_v3<SPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = smem;
  }
  dim3 grid((unsigned)P.h_m2l_targets.size(), (unsigned)((B + SLICE - 1) / SLICE));
  k_m2l32_v3<SPL><<<grid, NW * 32, smem, s>>>(P.m2l_targets, P.m2l_off, P.m2l_src, P.cell_centre, P.cell_level,
                                              P.side, P.p, nc, B, sched, Q, L, err);
  DM_LAUNCH("k_m2l32_v3");
}

}  // namespace

void build_m2l32_schedule(Plan& P) {
  if (P.p > 8) return;
  std::vector<int> h = make_schedule(P.p);
  if (h.empty()) return;
  P.m2l_sched = dalloc<int>(P, h.size());
  DM_CUDA(cudaMemcpyAsync(P.m2l_sched, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, P.stream));
  DM_CUDA(cudaStreamSynchronize(P.stream));
}

bool launch_m2l32_fast(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s) {
  if (P.h_m2l_targets.empty()) return true;
  // needs the row schedule (p <= 8) and 16-byte aligned state rows for the bulk copies
  if (!P.m2l_sched || (B & 3)) return false;
  if (B > 64)
    launch_v3<4>(P, B, Q, L, err, s, P.m2l_sched);
  else if (B > 32)
    launch_v3<2>(P, B, Q, L, err, s, P.m2l_sched);
  else
    launch_v3<1>(P, B, Q, L, err, s, P.m2l_sched);
  return true;
}

}  // namespace demag
