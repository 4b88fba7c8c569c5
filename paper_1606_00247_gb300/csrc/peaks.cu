// peaks.cu -- microbenchmarks of the arithmetic peaks the roofline fractions
// of the evaluation stages are stated against (a service of the library; the
// paper has no counterpart):
//   FP64 and FP32 FMA on the CUDA cores: every thread runs 8 independent FMA
//   chains in registers (2 flops per FMA);
//   BF16 and TF32 tcgen05.mma, M = 128, N = 256, FP32 accumulation in tensor
//   memory: one CTA per SM, one thread issues a long sequence of MMAs on
//   shared-memory operands (2 M N K flops each).
// Timed with CUDA events on a private stream after a warm-up; the best of
// three runs is returned.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace demag {

namespace {

using namespace tcx;

template <class T>
__global__ void __launch_bounds__(256) k_fma_peak(int iters, T seed, T* out) {
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; i++) a[i] = seed + (T)(threadIdx.x + i);
  const T m = (T)0.999999, c = (T)1e-7;
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) a[i] = a[i] * m + c;  // contracted to one FMA
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; i++) s += a[i];
  if (s == (T)-12345.0) out[threadIdx.x] = s;  // keeps the chains alive
}

// kind::f16 (BF16) with K = 16 or kind::tf32 with K = 8: 32 bytes of K per row
template <bool TF32>
__global__ void __launch_bounds__(128, 1) k_mma_peak(int iters, int* err) {
  __shared__ __align__(1024) unsigned char sA[128 * 32];
  __shared__ __align__(1024) unsigned char sB[256 * 32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int q = tid; q < 128 * 32 / 16; q += 128) ((uint4*)sA)[q] = make_uint4(0, 0, 0, 0);
  for (int q = tid; q < 256 * 32 / 16; q += 128) ((uint4*)sB)[q] = make_uint4(0, 0, 0, 0);
  if (tid == 0) {
    mbar_init(smem_u32(&bar), 1);
    mbar_init_fence();
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) tmem_alloc(smem_u32(&tmem_slot), 256);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  if (tid == 0) {
    const uint32_t id = TF32 ? ((1u << 4) | (2u << 7) | (2u << 10) | ((256u >> 3) << 17) | ((128u >> 4) << 24))
                             : idesc_bf16(128, 256);
    const uint64_t ad = sdesc(smem_u32(sA)), bd = sdesc(smem_u32(sB));
    for (int it = 0; it < iters; it++) {
      const uint32_t acc = it > 0 ? 1u : 0u;
      if (TF32)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
      else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc)
            : "memory");
    }
    mma_commit(smem_u32(&bar));
    if (!mbar_wait(smem_u32(&bar), 0u, nullptr)) {
      atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
      mbar_wait(smem_u32(&bar), 0u, nullptr);  // once more, bounded, for the MMAs in flight
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

}  // namespace

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_measure_peak(int kind, double* tflops) {
  try {
    if (!tflops || kind < 0 || kind > 3) fail(DEMAG_ERR_INVALID_ARG, "demag_measure_peak: kind in 0..3, non-NULL out");
    int dev = 0, nsm = 0;
    DM_CUDA(cudaGetDevice(&dev));
    DM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    cudaStream_t s = nullptr;
    DM_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    cudaEvent_t a = nullptr, b = nullptr;
    void* scratch = nullptr;
    double best = 0.0;
    try {
      DM_CUDA(cudaEventCreate(&a));
      DM_CUDA(cudaEventCreate(&b));
      DM_CUDA(cudaMalloc(&scratch, 4096));
      DM_CUDA(cudaMemsetAsync(scratch, 0, 4096, s));
      for (int rep = 0; rep < 4; rep++) {
        double flops = 0.0;
        DM_CUDA(cudaEventRecord(a, s));
        if (kind == 0) {
          const int iters = 1 << 14, blocks = nsm * 8;
          k_fma_peak<double><<<blocks, 256, 0, s>>>(iters, 1.0, (double*)scratch);
          flops = 2.0 * 8 * iters * 256.0 * blocks;
        } else if (kind == 1) {
          const int iters = 1 << 16, blocks = nsm * 8;
          k_fma_peak<float><<<blocks, 256, 0, s>>>(iters, 1.0f, (float*)scratch);
          flops = 2.0 * 8 * iters * 256.0 * blocks;
        } else {
          const int iters = 1 << 12;
          if (kind == 2)
            k_mma_peak<false><<<nsm, 128, 0, s>>>(iters, (int*)scratch);
          else
            k_mma_peak<true><<<nsm, 128, 0, s>>>(iters, (int*)scratch);
          flops = 2.0 * 128 * 256 * (kind == 2 ? 16 : 8) * (double)iters * nsm;
        }
        DM_LAUNCH("peak probe");
        DM_CUDA(cudaEventRecord(b, s));
        DM_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        DM_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (rep > 0) best = std::max(best, flops / (ms * 1e-3) / 1e12);  // rep 0 is the warm-up
      }
      int herr = 0;
      DM_CUDA(cudaMemcpyAsync(&herr, scratch, sizeof(int), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      if ((kind == 2 || kind == 3) && herr) fail(DEMAG_ERR_TIMEOUT, "tensor-core peak probe: a bounded wait expired");
    } catch (...) {
      if (a) cudaEventDestroy(a);
      if (b) cudaEventDestroy(b);
      if (scratch) cudaFree(scratch);
      cudaStreamDestroy(s);
      throw;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(scratch);
    cudaStreamDestroy(s);
    *tflops = best;
    return DEMAG_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (...) {
    set_last_error("unexpected internal error");
    return DEMAG_ERR_CUDA;
  }
}
