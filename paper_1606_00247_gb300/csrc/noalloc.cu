// noalloc.cu -- demag_eval_noalloc: the evaluation with all of its scratch in
// one fixed, file-scope device array instead of memory from cudaMalloc.
//
// Who needs it: a caller that must not allocate device memory while it runs --
// for example a host application whose own pool allocator has reserved the
// device memory up front and forbids other cudaMalloc/cudaFree calls, or a
// latency-critical loop that cannot afford the implicit device-wide
// synchronisation and the unbounded cost of cudaMalloc/cudaFree.  demag_eval
// allocates its workspace on the first call and whenever a larger batch needs a
// larger one; this entry point never does.
//
// The array below is part of the loaded module: the CUDA runtime reserves it
// on every device that loads libdemag.so, and keeps it until the process exits.
// Its host-side name is only a stand-in for the device symbol, so its device
// address is looked up once per device (cudaGetSymbolAddress, with that device
// current) on the first call of the entry point on that device -- and again if
// the device's context has changed since; that first call should therefore
// come before any stream capture.  A bounded device wait that expires is
// recorded in a flag inside the array; demag_eval_status reads it.
//
// Every call on a device uses the same array, and the array keeps the
// contents of the previous call: each scratch buffer that must start at zero
// is cleared on the stream by the call itself.  Calls that overlap on the GPU
// (different streams, or a concurrent demag_eval_noalloc on another plan of the
// same device) race on the array and must be serialised by the caller.
#include <cuda.h>  // the CUcontext type; the driver entry point itself is fetched through the runtime

#include <mutex>

#include "common.cuh"

namespace demag {

static __device__ __align__(256) unsigned char g_noalloc_scratch[DEMAG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
struct ScratchAddr {
  void* ctx = nullptr;         // the CUDA context the address belongs to
  unsigned char* ptr = nullptr;
};
ScratchAddr g_addr[MAX_DEVICES];  // device -> device address of g_noalloc_scratch

// the current CUDA context of the calling thread (nullptr if it cannot be told)
void* current_context() {
  using GetCurrent = CUresult (*)(CUcontext*);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return (GetCurrent)f;
  }();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return (void*)c;
}

// Device address of the fixed array for the current device and context: looked
// up once (cudaGetSymbolAddress with that device current) and kept; looked up
// again when the thread's context of the device has changed (for instance after
// cudaDeviceReset), or on every call if the context cannot be told.
unsigned char* scratch_address(int device) {
  if (device < 0 || device >= MAX_DEVICES) fail(DEMAG_ERR_UNSUPPORTED, "device ordinal beyond 63");
  void* ctx = current_context();
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_addr[device].ptr && ctx && g_addr[device].ctx == ctx) return g_addr[device].ptr;
  void* ptr = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || ptr == nullptr) {
    cudaGetLastError();
    fail(DEMAG_ERR_CUDA, std::string("cudaGetSymbolAddress of the fixed scratch area failed: ") +
                             cudaGetErrorString(e));
  }
  g_addr[device] = ScratchAddr{ctx, (unsigned char*)ptr};
  return g_addr[device].ptr;
}

// carve the buffers one evaluation of B states needs, 256-byte aligned
struct Carver {
  unsigned char* base;
  size_t used = 0;
  template <class T>
  T* take(size_t n) {
    used = (used + 255) & ~size_t(255);
    T* p = base ? (T*)(base + used) : nullptr;
    used += n * sizeof(T);
    return p;
  }
};

size_t carve(Plan& P, int B, unsigned char* base, Workspace* W) {
  Carver c{base};
  const size_t nn = P.nn, nt = P.nt, nc = P.nc, ncell = P.ncells;
  const bool mixed = P.opt.precision != DEMAG_FP64, otf = P.opt.near_mode == 0;
  Workspace w;
  w.B = B;
  if (!mixed || otf) w.Ms = c.take<double>(nn * 3 * B);
  if (!mixed) {
    w.Q = c.take<double>(ncell * nc * B);
    w.L = c.take<double>(ncell * nc * B);
  } else {
    w.Ms32 = c.take<float>(nn * 3 * B);
    w.Q32 = c.take<float>(ncell * nc * B + 16);  // tail pad for 16-byte bulk copies
    w.L32 = c.take<float>(ncell * nc * B);
    w.u32 = c.take<float>(nn * B);
    const size_t qp = m2l_tc_pack_bytes(P, B);
    if (qp) w.QP = c.take<unsigned char>(qp);
    const size_t mp = nf_mp_floats(P, B);
    if (mp) w.MP = c.take<float>(mp);
  }
  if (!mixed || otf) w.u_s = c.take<double>(nn * B);
  if (otf) w.state = c.take<double>(nt * TET_STATE * std::min(B, P2P_AT_MIN_B - 1));
  w.err = c.take<int>(1);
  if (W) {
    W->B = w.B;
    W->Ms = w.Ms;
    W->Q = w.Q;
    W->L = w.L;
    W->Ms32 = w.Ms32;
    W->Q32 = w.Q32;
    W->L32 = w.L32;
    W->u32 = w.u32;
    W->QP = w.QP;
    W->MP = w.MP;
    W->u_s = w.u_s;
    W->state = w.state;
    W->err = w.err;
  }
  return c.used;
}

}  // namespace

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_eval_noalloc(demag_plan plan, const double* M, int batch, double* u, double* H,
                                           void* cuda_stream) {
  try {
    if (!plan || !M || !u) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (batch < 1) fail(DEMAG_ERR_INVALID_ARG, "batch must be >= 1");
    if (!is_device_ptr(M) || !is_device_ptr(u) || (H && !is_device_ptr(H)))
      fail(DEMAG_ERR_INVALID_ARG, "demag_eval_noalloc takes device pointers only");
    const size_t need = carve(*plan, batch, nullptr, nullptr);
    if (need > (size_t)DEMAG_NOALLOC_SCRATCH_BYTES)
      fail(DEMAG_ERR_INVALID_ARG, "this plan and batch need " + std::to_string(need) +
                                      " bytes of scratch; the fixed area holds " +
                                      std::to_string((size_t)DEMAG_NOALLOC_SCRATCH_BYTES));
    int dev = 0;
    DM_CUDA(cudaGetDevice(&dev));
    Workspace W;
    carve(*plan, batch, scratch_address(dev), &W);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (plan->opt.precision == DEMAG_FP64)
      eval_fp64_ws(*plan, W, M, batch, u, H, s, false);
    else
      eval_mixed_ws(*plan, W, M, batch, u, H, s, false);
    return DEMAG_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (...) {
    set_last_error("unexpected internal error");
    return DEMAG_ERR_CUDA;
  }
}
