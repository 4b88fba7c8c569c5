// multi.cu -- demag_eval_multi: several plans (meshes, each with its own batch
// of states) evaluated through one submission.
//
// The first call with a given signature (plans, batches, pointers, workspaces)
// runs every plan's evaluation directly on the caller's stream -- which also
// performs the one-time setup of each plan (workspace, kernel attributes) --
// and then records the same work once more, without running it, as a CUDA
// graph: one branch per plan, forked from and joined back to a private
// capture stream, so the plans' kernels may overlap on the GPU.  Later calls
// with the same signature replay that graph with one launch on the caller's
// stream.  Graphs are cached per signature (a few at a time, least recently
// used dropped first) and dropped when one of their plans is destroyed or a
// plan's workspace is reallocated (the workspace address is part of the
// signature).
#include <algorithm>
#include <list>
#include <mutex>

#include "common.cuh"

namespace demag {

namespace {

struct GraphEntry {
  std::vector<const void*> key;
  int device = -1;
  cudaGraphExec_t exec = nullptr;
  std::vector<const Plan*> plans;
};

std::mutex g_mu;
std::list<GraphEntry> g_cache;  // most recently used first
constexpr size_t kMaxGraphs = 8;

void drop(GraphEntry& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  e.exec = nullptr;
}

void eval_one(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, cudaStream_t s) {
  if (P.opt.precision == DEMAG_FP64)
    eval_fp64_ws(P, W, M, B, u, H, s, false);
  else
    eval_mixed_ws(P, W, M, B, u, H, s, false);
}

}  // namespace

void multi_forget_plan(const Plan* P) {
  std::lock_guard<std::mutex> lock(g_mu);
  for (auto it = g_cache.begin(); it != g_cache.end();) {
    if (std::find(it->plans.begin(), it->plans.end(), P) != it->plans.end()) {
      drop(*it);
      it = g_cache.erase(it);
    } else {
      ++it;
    }
  }
}

void eval_multi(Plan* const* plans, int n, const double* const* M, const int* batch, double* const* u,
                double* const* H, cudaStream_t s) {
  int dev = 0;
  DM_CUDA(cudaGetDevice(&dev));
  std::vector<Workspace*> ws(n);
  std::vector<const void*> key;
  key.reserve(7 * n);
  for (int i = 0; i < n; i++) {
    ws[i] = &workspace(*plans[i], batch[i]);
    key.insert(key.end(), {(const void*)plans[i], (const void*)(intptr_t)batch[i], (const void*)M[i],
                           (const void*)u[i], (const void*)(H ? H[i] : nullptr), (const void*)ws[i],
                           (const void*)(intptr_t)ws[i]->B});
  }
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it)
      if (it->device == dev && it->key == key) {
        DM_CUDA(cudaGraphLaunch(it->exec, s));
        g_cache.splice(g_cache.begin(), g_cache, it);
        return;
      }
  }
  // first call with this signature: run it, then record it as a graph
  for (int i = 0; i < n; i++) eval_one(*plans[i], *ws[i], M[i], batch[i], u[i], H ? H[i] : nullptr, s);
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> br(n, nullptr);
  std::vector<cudaEvent_t> done(n, nullptr);
  cudaEvent_t fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&] {
    for (auto& e : done)
      if (e) cudaEventDestroy(e);
    for (auto& b : br)
      if (b) cudaStreamDestroy(b);
    if (fork) cudaEventDestroy(fork);
    if (cap) cudaStreamDestroy(cap);
    if (graph) cudaGraphDestroy(graph);
  };
  try {
    DM_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    DM_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int i = 0; i < n; i++) {
      DM_CUDA(cudaStreamCreateWithFlags(&br[i], cudaStreamNonBlocking));
      DM_CUDA(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
    }
    DM_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    try {
      DM_CUDA(cudaEventRecord(fork, cap));
      for (int i = 0; i < n; i++) {
        DM_CUDA(cudaStreamWaitEvent(br[i], fork, 0));
        eval_one(*plans[i], *ws[i], M[i], batch[i], u[i], H ? H[i] : nullptr, br[i]);
        DM_CUDA(cudaEventRecord(done[i], br[i]));
        DM_CUDA(cudaStreamWaitEvent(cap, done[i], 0));
      }
    } catch (...) {
      cudaGraph_t g = nullptr;
      cudaStreamEndCapture(cap, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    DM_CUDA(cudaStreamEndCapture(cap, &graph));
    DM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  } catch (...) {
    cleanup();
    throw;
  }
  cleanup();
  std::lock_guard<std::mutex> lock(g_mu);
  GraphEntry e;
  e.key = std::move(key);
  e.device = dev;
  e.exec = exec;
  for (int i = 0; i < n; i++) e.plans.push_back(plans[i]);
  g_cache.push_front(std::move(e));
  while (g_cache.size() > kMaxGraphs) {
    drop(g_cache.back());
    g_cache.pop_back();
  }
}

}  // namespace demag
