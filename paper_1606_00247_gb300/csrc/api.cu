// api.cu -- the extern "C" boundary of libdemag.so (include/demag.h).
// No exception crosses it: every entry point catches and returns a status.
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define DEMAG_NVTX 1
#else
#define DEMAG_NVTX 0
#endif

namespace demag {

static const char* const kStageName[DEMAG_N_STAGES] = {"demag:gather", "demag:p2m", "demag:m2m",
                                                       "demag:m2l",    "demag:l2l", "demag:l2p",
                                                       "demag:near_prep", "demag:p2p", "demag:h"};

static uint64_t range_start(const char* name) {
#if DEMAG_NVTX
  return (uint64_t)nvtxRangeStartA(name);
#else
  (void)name;
  return 0;
#endif
}

static void range_end(uint64_t id) {
#if DEMAG_NVTX
  if (id) nvtxRangeEnd((nvtxRangeId_t)id);
#else
  (void)id;
#endif
}

void smem_opt_in(const void* func, size_t bytes) {
  int dev = 0;
  DM_CUDA(cudaGetDevice(&dev));
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> opted;
  std::lock_guard<std::mutex> lock(mu);
  size_t& have = opted[{func, dev}];
  if (bytes <= have) return;
  DM_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  have = bytes;
}

// an NVTX range over one entry point
struct EntryRange {
  uint64_t id;
  explicit EntryRange(const char* name) : id(range_start(name)) {}
  ~EntryRange() { range_end(id); }
};

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(demag_status s, const std::string& msg) { throw Error{s, msg}; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  cudaGetLastError();
  demag_status s = (e == cudaErrorMemoryAllocation) ? DEMAG_ERR_OUT_OF_MEMORY : DEMAG_ERR_CUDA;
  throw Error{s, std::string(what) + " failed: " + cudaGetErrorString(e) + " (" + file + ":" + std::to_string(line) +
                     ")"};
}

StageClock::StageClock(Plan& P_, cudaStream_t s_, bool allow) : P(P_), s(s_), on(allow && P_.opt.profile != 0) {
  if (on)
    for (auto& e : ev) DM_CUDA(cudaEventCreate(&e));
}
StageClock::~StageClock() {
  range_end(range);
  if (on)
    for (auto& e : ev) cudaEventDestroy(e);
}
void StageClock::begin(int stage) {
  cur = stage;
  used[stage] = true;
  range_end(range);
  range = range_start(kStageName[stage]);
  if (on) DM_CUDA(cudaEventRecord(ev[2 * stage], s));
}
void StageClock::end() {
  range_end(range);
  range = 0;
  if (on) DM_CUDA(cudaEventRecord(ev[2 * cur + 1], s));
}
void StageClock::finish() {
  int64_t total = 0;
  for (int k = 0; k < DEMAG_N_STAGES; k++) total += launches[k];
  P.eval_launches = total;
  if (!on) return;
  DM_CUDA(cudaStreamSynchronize(s));
  for (int k = 0; k < DEMAG_N_STAGES; k++) {
    if (!used[k]) continue;
    float ms = 0;
    DM_CUDA(cudaEventElapsedTime(&ms, ev[2 * k], ev[2 * k + 1]));
    P.stage_ms[k] += ms;
    P.stage_launches[k] += launches[k];
  }
  P.n_evals_profiled++;
}

void dfree_all(Plan& P) {
  for (auto& b : P.bufs) cudaFree(b.ptr);
  P.bufs.clear();
}

void dfree(Plan& P, void* ptr) {
  for (size_t i = 0; i < P.bufs.size(); i++)
    if (P.bufs[i].ptr == ptr) {
      cudaFree(ptr);
      P.device_bytes -= (int64_t)P.bufs[i].bytes;
      P.bufs.erase(P.bufs.begin() + (long)i);
      return;
    }
  P.device_bytes = 0;
}

template <class F>
static demag_status guarded(F&& f) {
  try {
    f();
    return DEMAG_OK;
  } catch (const Error& e) {
    set_last_error(e.msg);
    return e.status;
  } catch (const std::bad_alloc&) {
    set_last_error("host allocation failed");
    return DEMAG_ERR_OUT_OF_MEMORY;
  } catch (...) {
    set_last_error("unexpected internal error");
    return DEMAG_ERR_CUDA;
  }
}

template <class Dst, class Src>
static void copy_convert(Dst* dst, const Src* src_dev, int64_t n, cudaStream_t s) {
  if (!dst || n <= 0) return;
  std::vector<Src> h(n);
  DM_CUDA(cudaMemcpyAsync(h.data(), src_dev, n * sizeof(Src), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  for (int64_t i = 0; i < n; i++) dst[i] = (Dst)h[i];
}

// leaf-size tuning: a fixed, smooth field of unit vectors (B x N_n x 3) to time evaluations with
__global__ void k_tune_m(int64_t n, double* M) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = 0.37 * (double)(i % 9973), b = 0.11 * (double)(i % 7919);
    M[3 * i] = sin(a) * cos(b);
    M[3 * i + 1] = sin(a) * sin(b);
    M[3 * i + 2] = cos(a);
  }
}

static void release_plan(demag_plan_s* P) {
  if (!P) return;
  multi_forget_plan(P);
  destroy_workspace(*P);
  dfree_all(*P);
  if (P->stream) cudaStreamDestroy(P->stream);
  delete P;
}

// choices of the tuners (autotune bits 0-2) for one mesh, options and device
struct TuneChoice {
  int p = 0, leaf = 0, nt = 0, kps = 0, budget = 0;  // order, leaf size, M2L targets per CTA, k-steps, ring bytes
};

static demag_plan_s* new_plan(const demag_options& o, int64_t n_nodes, int64_t n_tets, const double* nodes,
                              const int32_t* tets, const TuneChoice* preset = nullptr) {
  demag_plan_s* P = new demag_plan_s();
  try {
    P->opt = o;
    if (preset) {
      P->tc_preset_nt = preset->nt;
      P->tc_preset_kps = preset->kps;
      P->tc_preset_budget = preset->budget;
    }
    P->p = o.p;
    P->nc = ncoef_of(o.p);
    P->nn = n_nodes;
    P->nt = n_tets;
    DM_CUDA(cudaGetDevice(&P->device));
    DM_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
    build_plan(*P, nodes, tets);
  } catch (...) {
    release_plan(P);
    throw;
  }
  return P;
}

// device time of one evaluation of B states (after one untimed evaluation)
static float time_eval(demag_plan_s* P, int B, const double* M, double* u, double* H) {
  cudaEvent_t a = nullptr, b = nullptr;
  DM_CUDA(cudaEventCreate(&a));
  DM_CUDA(cudaEventCreate(&b));
  float ms = 0.f;
  for (int k = 0; k < 3; k++) {
    if (k == 1) DM_CUDA(cudaEventRecord(a, P->stream));
    if (P->opt.precision == DEMAG_FP64)
      eval_fp64(*P, M, B, u, H, P->stream);
    else
      eval_mixed(*P, M, B, u, H, P->stream);
  }
  DM_CUDA(cudaEventRecord(b, P->stream));
  DM_CUDA(cudaEventSynchronize(b));
  DM_CUDA(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / 2;
}

// autotune bit 1: build the plan for leaf sizes L/2, L, 2L, 4L (L = the
// requested one), time an evaluation of max_batch states on each and keep the
// fastest; the others are released as soon as they lose
static demag_plan_s* tune_leaf(const demag_options& o, int64_t n_nodes, int64_t n_tets, const double* nodes,
                               const int32_t* tets) {
  const auto t0 = std::chrono::steady_clock::now();
  const int64_t nm = (int64_t)o.max_batch * n_nodes;
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)(nm * 7)) != cudaSuccess) {
    cudaGetLastError();
    fail(DEMAG_ERR_OUT_OF_MEMORY, "leaf-size tuning buffers");
  }
  double *M = buf, *u = buf + 3 * nm, *H = buf + 4 * nm;
  demag_plan_s* best = nullptr;
  float best_ms = 0.f;
  try {
    k_tune_m<<<256, 256>>>(nm, M);
    DM_CUDA(cudaGetLastError());
    DM_CUDA(cudaDeviceSynchronize());
    const int L = o.leaf_size;
    for (int leaf : {std::max(1, L / 2), L, 2 * L, 4 * L}) {
      demag_options oc = o;
      oc.leaf_size = leaf;
      demag_plan_s* P = new_plan(oc, n_nodes, n_tets, nodes, tets);
      float ms = 0.f;
      try {
        ms = time_eval(P, o.max_batch, M, u, H);
        destroy_workspace(*P);
      } catch (...) {
        release_plan(P);
        throw;
      }
      if (!best || ms < best_ms) {
        release_plan(best);
        best = P;
        best_ms = ms;
      } else {
        release_plan(P);
      }
    }
  } catch (...) {
    release_plan(best);
    cudaFree(buf);
    throw;
  }
  cudaFree(buf);
  best->tuned_leaf_ms = best_ms;
  best->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return best;
}

// relative L2 distance of two device vectors of n doubles (host reduction, plan time only)
static double rel_l2_dev(const double* a, const double* b, int64_t n) {
  std::vector<double> ha(n), hb(n);
  DM_CUDA(cudaMemcpy(ha.data(), a, sizeof(double) * n, cudaMemcpyDeviceToHost));
  DM_CUDA(cudaMemcpy(hb.data(), b, sizeof(double) * n, cudaMemcpyDeviceToHost));
  double num = 0.0, den = 0.0;
  for (int64_t i = 0; i < n; i++) {
    num += (ha[i] - hb[i]) * (ha[i] - hb[i]);
    den += hb[i] * hb[i];
  }
  return den > 0.0 ? std::sqrt(num / den) : std::sqrt(num);
}

// autotune bit 2: the smallest p in {4, 6, 8, 10} whose u and H on one state are within
// DEMAG_TUNE_P_TARGET (rel-L2) of an FP64 evaluation at p = 10 with the same leaf and theta
// (the truncation error at p = 10 is ~1e-6 at theta = 0.5, two orders below the target)
constexpr double DEMAG_TUNE_P_TARGET = 5e-5;

static int tune_p(const demag_options& o, int64_t n_nodes, int64_t n_tets, const double* nodes,
                  const int32_t* tets) {
  double* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(double) * (size_t)(n_nodes * 11)) != cudaSuccess) {
    cudaGetLastError();
    fail(DEMAG_ERR_OUT_OF_MEMORY, "order tuning buffers");
  }
  double *M = buf, *u0 = buf + 3 * n_nodes, *H0 = buf + 4 * n_nodes, *u = buf + 7 * n_nodes, *H = buf + 8 * n_nodes;
  int chosen = 10;
  try {
    k_tune_m<<<256, 256>>>(n_nodes, M);
    DM_CUDA(cudaGetLastError());
    DM_CUDA(cudaDeviceSynchronize());  // the plans evaluate on their own non-blocking streams
    demag_options oc = o;
    oc.max_batch = 1;
    oc.autotune = 0;
    oc.precision = DEMAG_FP64;
    oc.p = 10;
    demag_plan_s* R = new_plan(oc, n_nodes, n_tets, nodes, tets);
    try {
      eval_fp64(*R, M, 1, u0, H0, R->stream);
      DM_CUDA(cudaStreamSynchronize(R->stream));
    } catch (...) {
      release_plan(R);
      throw;
    }
    release_plan(R);
    for (int p : {4, 6, 8}) {
      oc = o;
      oc.max_batch = 1;
      oc.autotune = 0;
      oc.p = p;
      demag_plan_s* P = new_plan(oc, n_nodes, n_tets, nodes, tets);
      double err = 0.0;
      try {
        if (oc.precision == DEMAG_FP64)
          eval_fp64(*P, M, 1, u, H, P->stream);
        else
          eval_mixed(*P, M, 1, u, H, P->stream);
        DM_CUDA(cudaStreamSynchronize(P->stream));
        err = std::max(rel_l2_dev(u, u0, n_nodes), rel_l2_dev(H, H0, 3 * n_nodes));
      } catch (...) {
        release_plan(P);
        throw;
      }
      release_plan(P);
      if (err <= DEMAG_TUNE_P_TARGET) {
        chosen = p;
        break;
      }
    }
  } catch (...) {
    cudaFree(buf);
    throw;
  }
  cudaFree(buf);
  return chosen;
}

// ---------------------------------------------------------------------------
// Tuner cache.  The tuners choose by timing, which costs up to ~50 s of plan
// time on a ball of half a million tets.  With the environment variable
// DEMAG_TUNE_CACHE naming a file, a tuned plan's choices are appended to it
// under a key that hashes the mesh, the options and the device, and a later
// demag_plan_create with the same key builds the plan from them without timing.
// Every candidate plan is built deterministically, so the plan built from the
// cached choices is the one the tuners kept.  Lines that do not parse, carry
// another format version or hold values out of range are skipped; the last
// valid line of a key wins.
constexpr int TUNE_CACHE_VERSION = 1;

static const char* tune_cache_path() {
  const char* p = std::getenv("DEMAG_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

// FNV-1a over 64-bit words (a byte tail is zero-padded, the length appended)
struct Fnv1a {
  uint64_t h = 1469598103934665603ull;
  void word(uint64_t w) { h = (h ^ w) * 1099511628211ull; }
  void bytes(const void* p, size_t n) {
    const unsigned char* c = (const unsigned char*)p;
    size_t i = 0;
    for (; i + 8 <= n; i += 8) {
      uint64_t w;
      std::memcpy(&w, c + i, 8);
      word(w);
    }
    if (i < n) {
      uint64_t w = 0;
      std::memcpy(&w, c + i, n - i);
      word(w);
    }
    word(n);
  }
};

template <class T>
static void hash_array(Fnv1a& f, const T* a, int64_t n) {
  if (is_device_ptr(a)) {
    std::vector<T> h(n);
    DM_CUDA(cudaMemcpy(h.data(), a, sizeof(T) * n, cudaMemcpyDeviceToHost));
    f.bytes(h.data(), sizeof(T) * n);
  } else {
    f.bytes(a, sizeof(T) * n);
  }
}

static uint64_t tune_key(const demag_options& o, int64_t n_nodes, int64_t n_tets, const double* nodes,
                         const int32_t* tets) {
  Fnv1a f;
  f.word(TUNE_CACHE_VERSION);
  int dev = 0;
  DM_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp prop{};
  DM_CUDA(cudaGetDeviceProperties(&prop, dev));
  f.bytes(prop.name, std::strlen(prop.name));
  f.word((uint64_t)prop.multiProcessorCount);
  f.word((uint64_t)(prop.major * 100 + prop.minor));
  // every option that changes what the tuners build or time (profile and graph do not)
  const int opts[] = {o.p, o.leaf_size, o.precision, o.near_mode, o.max_batch, o.autotune, o.m2l_targets_per_cta,
                      o.m2l_kps, o.m2l_promote, o.m2l_promote_rows, o.m2l_table_batch, o.sources, o.near_tc,
                      o.m2l_split_degree};
  for (int v : opts) f.word((uint64_t)(int64_t)v);
  uint64_t th;
  std::memcpy(&th, &o.theta, sizeof th);
  f.word(th);
  f.word((uint64_t)n_nodes);
  f.word((uint64_t)n_tets);
  hash_array(f, nodes, 3 * n_nodes);
  hash_array(f, tets, 4 * n_tets);
  return f.h;
}

static bool tune_cache_find(const char* path, uint64_t key, TuneChoice& c) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[256];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char tag[16];
    int ver = 0;
    unsigned long long k = 0;
    TuneChoice t;
    if (std::sscanf(line, "%15s %d %llx %d %d %d %d %d", tag, &ver, &k, &t.p, &t.leaf, &t.nt, &t.kps, &t.budget) != 8)
      continue;
    if (std::strcmp(tag, "demag-tune") != 0 || ver != TUNE_CACHE_VERSION || k != key) continue;
    if (t.p < 1 || t.p > MAX_P || t.leaf < 1 || t.nt < 0 || t.nt > 2 || t.kps < 0 || t.kps > 8 || t.budget < 0 ||
        t.budget > 227 * 1024)
      continue;
    c = t;
    found = true;
  }
  std::fclose(f);
  return found;
}

static void tune_cache_add(const char* path, uint64_t key, const TuneChoice& c) {
  FILE* f = std::fopen(path, "a");  // one short line in append mode: concurrent writers do not interleave
  if (!f) {
    set_last_error(std::string("warning: the tuner cache ") + path + " cannot be written");
    return;
  }
  std::fprintf(f, "demag-tune %d %016llx %d %d %d %d %d\n", TUNE_CACHE_VERSION, (unsigned long long)key, c.p, c.leaf,
               c.nt, c.kps, c.budget);
  std::fclose(f);
}

}  // namespace demag

using namespace demag;

extern "C" {

void demag_options_default(demag_options* o) {
  if (!o) return;
  o->p = 4;
  o->leaf_size = 32;
  o->theta = 0.5;
  o->precision = DEMAG_FP64;
  o->near_mode = 0;
  o->max_batch = 1;
  o->autotune = 0;
  o->m2l_targets_per_cta = 0;
  o->m2l_kps = 0;
  o->m2l_promote = 0;
  o->m2l_promote_rows = 0;
  o->m2l_table_batch = 0;
  o->sources = DEMAG_SOURCES_TETS;
  o->profile = 0;
  o->near_tc = 0;
  o->graph = 0;
  o->m2l_split_degree = 0;
}

demag_status demag_plan_create(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, int p,
                               int leaf_size, double theta, const demag_options* opt, demag_plan* out) {
  EntryRange range_("demag_plan_create");
  set_last_error("");
  if (out) *out = nullptr;
  demag_plan_s* P = nullptr;
  demag_status st = guarded([&] {
    if (!nodes || !tets || !out) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (n_nodes < 4 || n_tets < 1) fail(DEMAG_ERR_INVALID_ARG, "need n_nodes >= 4 and n_tets >= 1");
    if (n_nodes > INT32_MAX / 4 || n_tets > INT32_MAX / 4) fail(DEMAG_ERR_INVALID_ARG, "mesh too large");
    demag_options o;
    demag_options_default(&o);
    if (opt) o = *opt;
    o.p = p;
    o.leaf_size = leaf_size;
    o.theta = theta;
    if (o.p < 1 || o.p > MAX_P) fail(DEMAG_ERR_INVALID_ARG, "p must be in 1..12");
    if (o.leaf_size < 1) fail(DEMAG_ERR_INVALID_ARG, "leaf_size must be >= 1");
    if (!(o.theta > 0) || !std::isfinite(o.theta)) fail(DEMAG_ERR_INVALID_ARG, "theta must be finite and > 0");
    if (o.max_batch < 1) fail(DEMAG_ERR_INVALID_ARG, "max_batch must be >= 1");
    if (o.autotune < 0 || o.autotune > 7) fail(DEMAG_ERR_INVALID_ARG, "autotune must be in 0..7");
    if (o.m2l_targets_per_cta < 0 || o.m2l_targets_per_cta > 2)
      fail(DEMAG_ERR_INVALID_ARG, "m2l_targets_per_cta must be 0, 1 or 2");
    if (o.m2l_kps < 0 || o.m2l_kps > 8) fail(DEMAG_ERR_INVALID_ARG, "m2l_kps must be in 0..8");
    if (o.m2l_promote_rows < 0 || o.m2l_promote_rows > 64) fail(DEMAG_ERR_INVALID_ARG, "m2l_promote_rows must be in 0..64");
    if (o.m2l_split_degree > 0) fail(DEMAG_ERR_INVALID_ARG, "m2l_split_degree must be 0 (default) or < 0 (every term)");
    if (o.near_mode != 0 && o.near_mode != 1) fail(DEMAG_ERR_INVALID_ARG, "near_mode must be 0 or 1");
    if (o.sources != DEMAG_SOURCES_TETS && o.sources != DEMAG_SOURCES_DIPOLES && o.sources != DEMAG_SOURCES_PATCHES)
      fail(DEMAG_ERR_INVALID_ARG, "sources must be DEMAG_SOURCES_TETS, _DIPOLES or _PATCHES");
    if (o.sources != DEMAG_SOURCES_TETS && o.near_mode != 1)
      fail(DEMAG_ERR_UNSUPPORTED, "point-dipole and vertex-patch sources need near_mode = 1");
    if (o.precision < DEMAG_FP64 || o.precision > DEMAG_MIXED_BF16X6)
      fail(DEMAG_ERR_INVALID_ARG, "unknown precision");
    if (o.graph != 0 && o.graph != 1) fail(DEMAG_ERR_INVALID_ARG, "graph must be 0 or 1");
    const auto t0 = std::chrono::steady_clock::now();
    const bool tuning = (o.autotune & 7) != 0;
    const char* cache = tuning ? tune_cache_path() : nullptr;
    const uint64_t key = cache ? tune_key(o, n_nodes, n_tets, nodes, tets) : 0;
    TuneChoice hit;
    if (cache && tune_cache_find(cache, key, hit)) {
      demag_options oc = o;
      if (o.autotune & 4) oc.p = hit.p;
      if (o.autotune & 2) oc.leaf_size = hit.leaf;
      oc.autotune &= ~4;
      P = new_plan(oc, n_nodes, n_tets, nodes, tets, &hit);
      P->tune_source = 2;
    } else {
      if (o.autotune & 4) {
        o.p = tune_p(o, n_nodes, n_tets, nodes, tets);
        o.autotune &= ~4;
      }
      P = (o.autotune & 2) ? tune_leaf(o, n_nodes, n_tets, nodes, tets) : new_plan(o, n_nodes, n_tets, nodes, tets);
      if (tuning) {
        P->tune_source = 1;
        TuneChoice c;
        c.p = P->p;
        c.leaf = P->opt.leaf_size;
        c.nt = P->tc_nt;
        c.kps = P->tc_kps;
        c.budget = P->tc_budget;
        if (cache) tune_cache_add(cache, key, c);
      }
    }
    if (tuning) P->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (o.theta >= 1.0)
      set_last_error("warning: theta >= 1, multipole expansions may not converge for accepted pairs");
    *out = P;
  });
  if (st != DEMAG_OK && P) release_plan(P);
  return st;
}

demag_status demag_eval(demag_plan plan, const double* M, int batch, double* u, double* H, void* cuda_stream) {
  EntryRange range_("demag_eval");
  return guarded([&] {
    if (!plan || !M || !u) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (batch < 1 || batch > plan->opt.max_batch) fail(DEMAG_ERR_INVALID_ARG, "batch must be in 1..max_batch");
    if (plan->opt.graph && !plan->opt.profile && is_device_ptr(M) && is_device_ptr(u) && (!H || is_device_ptr(H))) {
      Plan* pp = plan;
      eval_multi(&pp, 1, &M, &batch, &u, H ? &H : nullptr, (cudaStream_t)cuda_stream);  // record once, replay
      return;
    }
    if (plan->opt.precision == DEMAG_FP64)
      eval_fp64(*plan, M, batch, u, H, (cudaStream_t)cuda_stream);
    else
      eval_mixed(*plan, M, batch, u, H, (cudaStream_t)cuda_stream);
  });
}

demag_status demag_eval_field(demag_plan plan, const double* M, int batch, double* u, double* H, void* cuda_stream) {
  EntryRange range_("demag_eval_field");
  return guarded([&] {
    if (!plan || !M || !u || !H) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (batch < 1 || batch > plan->opt.max_batch) fail(DEMAG_ERR_INVALID_ARG, "batch must be in 1..max_batch");
    eval_field(*plan, M, batch, u, H, (cudaStream_t)cuda_stream);
  });
}

demag_status demag_plan_debug(demag_plan plan, int flags) {
  if (!plan || (flags & ~3)) {
    set_last_error("demag_plan_debug: NULL plan or unknown flag bits");
    return DEMAG_ERR_INVALID_ARG;
  }
  plan->debug_flags = flags;
  return DEMAG_OK;
}

demag_status demag_plan_audit(demag_plan plan) {
  return guarded([&] {
    if (!plan) fail(DEMAG_ERR_INVALID_ARG, "NULL plan");
    audit_plan(*plan, (plan->debug_flags & 2) != 0);
  });
}

demag_status demag_eval_status(demag_plan plan, void* cuda_stream) {
  int herr = 0;
  demag_status st = guarded([&] {
    if (!plan) fail(DEMAG_ERR_INVALID_ARG, "NULL plan");
    if (!plan->last_err) return;  // never evaluated
    cudaStream_t s = (cudaStream_t)cuda_stream;
    DM_CUDA(cudaMemcpyAsync(&herr, plan->last_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
  });
  if (st != DEMAG_OK) return st;
  if (herr == DEMAG_ERR_TIMEOUT) {
    set_last_error("a bounded device wait expired in the last evaluation of this plan; its outputs are unspecified");
    return DEMAG_ERR_TIMEOUT;
  }
  return herr ? DEMAG_ERR_CUDA : DEMAG_OK;
}

demag_status demag_eval_multi(const demag_plan* plans, int n_plans, const double* const* M, const int* batch,
                              double* const* u, double* const* H, void* cuda_stream) {
  EntryRange range_("demag_eval_multi");
  return guarded([&] {
    if (!plans || !M || !batch || !u || n_plans < 1) fail(DEMAG_ERR_INVALID_ARG, "NULL array or n_plans < 1");
    std::vector<Plan*> ps(n_plans);
    for (int i = 0; i < n_plans; i++) {
      if (!plans[i] || !M[i] || !u[i]) fail(DEMAG_ERR_INVALID_ARG, "NULL plan or pointer in the arrays");
      if (batch[i] < 1 || batch[i] > plans[i]->opt.max_batch)
        fail(DEMAG_ERR_INVALID_ARG, "batch must be in 1..max_batch of its plan");
      if (!is_device_ptr(M[i]) || !is_device_ptr(u[i]) || (H && H[i] && !is_device_ptr(H[i])))
        fail(DEMAG_ERR_INVALID_ARG, "demag_eval_multi takes device pointers only");
      for (int j = 0; j < i; j++)
        if (plans[j] == plans[i]) fail(DEMAG_ERR_INVALID_ARG, "a plan appears twice (they share a workspace)");
      ps[i] = plans[i];
    }
    eval_multi(ps.data(), n_plans, M, batch, u, H, (cudaStream_t)cuda_stream);
  });
}

demag_status demag_energy(demag_plan plan, const double* M, const double* H, int batch, double* e,
                          void* cuda_stream) {
  return guarded([&] {
    if (!plan || !M || !H || !e) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (batch < 1) fail(DEMAG_ERR_INVALID_ARG, "batch must be >= 1");
    if (!is_device_ptr(M) || !is_device_ptr(H) || !is_device_ptr(e))
      fail(DEMAG_ERR_INVALID_ARG, "demag_energy takes device pointers");
    energy(*plan, M, H, batch, e, (cudaStream_t)cuda_stream);
  });
}

demag_status demag_llg_rk4(demag_plan plan, double* m, int batch, double Ms, double alpha, const double* h_ext,
                           double dt, int steps, void* cuda_stream) {
  EntryRange range_("demag_llg_rk4");
  return guarded([&] {
    if (!plan || !m) fail(DEMAG_ERR_INVALID_ARG, "NULL pointer argument");
    if (batch < 1 || batch > plan->opt.max_batch) fail(DEMAG_ERR_INVALID_ARG, "batch must be in 1..max_batch");
    if (!(Ms > 0) || !(alpha >= 0) || !(dt > 0) || steps < 0 || !std::isfinite(Ms * alpha * dt))
      fail(DEMAG_ERR_INVALID_ARG, "need Ms > 0, alpha >= 0, dt > 0, steps >= 0 (finite)");
    if (!is_device_ptr(m)) fail(DEMAG_ERR_INVALID_ARG, "demag_llg_rk4 takes a device pointer");
    const double zero[3] = {0.0, 0.0, 0.0};
    llg_rk4(*plan, m, batch, Ms, alpha, h_ext ? h_ext : zero, dt, steps, (cudaStream_t)cuda_stream);
  });
}

demag_status demag_plan_destroy(demag_plan plan) {
  if (!plan) return DEMAG_ERR_INVALID_ARG;
  return guarded([&] {
    multi_forget_plan(plan);
    cudaStreamSynchronize(plan->stream);
    destroy_workspace(*plan);
    dfree_all(*plan);
    cudaStreamDestroy(plan->stream);
    delete plan;
  });
}

demag_status demag_plan_stats(demag_plan plan, demag_stats* o) {
  if (!plan || !o) return DEMAG_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->n_nodes = plan->nn;
  o->n_tets = plan->nt;
  o->n_cells = plan->ncells;
  o->n_leaves = plan->nleaves;
  o->n_levels = plan->nlevels;
  o->n_m2l = plan->n_m2l;
  o->n_p2p = plan->n_p2p;
  o->n_p2p_pairs = plan->n_p2p_pairs;
  o->n_near_cols = plan->n_wentries / 3;
  o->device_bytes = plan->device_bytes;
  for (int a = 0; a < 3; a++) o->lo[a] = plan->lo[a];
  o->side = plan->side;
  o->scale = plan->scale;
  o->plan_ms = plan->plan_ms;
  o->p = plan->p;
  o->leaf_size = plan->opt.leaf_size;
  o->precision = plan->opt.precision;
  o->near_mode = plan->opt.near_mode;
  o->max_batch = plan->opt.max_batch;
  o->theta = plan->opt.theta;
  o->eval_launches = plan->eval_launches;
  o->n_evals_profiled = plan->n_evals_profiled;
  for (int k = 0; k < DEMAG_N_STAGES; k++) {
    o->stage_ms[k] = plan->stage_ms[k];
    o->stage_launches[k] = plan->stage_launches[k];
  }
  o->n_m2l_ops = plan->n_tc_ops;
  o->m2l_kps = plan->tc_kps;
  o->m2l_ring_bytes = plan->tc_budget;
  o->m2l_targets_per_cta = plan->tc_ops ? plan->tc_nt : 0;
  o->n_near_tiles = plan->nf_ntiles;
  o->near_tile_cols = plan->nf_ncols;
  o->tune_source = plan->tune_source;
  o->near_bytes = plan->nf_W ? plan->nf_wbytes
                             : (plan->W32 ? plan->n_wentries / 3 * 16
                                          : (plan->W64 ? plan->n_wentries * 8 : 0));
  return DEMAG_OK;
}

demag_status demag_plan_reset_timers(demag_plan plan) {
  if (!plan) return DEMAG_ERR_INVALID_ARG;
  for (int k = 0; k < DEMAG_N_STAGES; k++) {
    plan->stage_ms[k] = 0;
    plan->stage_launches[k] = 0;
  }
  plan->n_evals_profiled = 0;
  return DEMAG_OK;
}

demag_status demag_plan_export_tree(demag_plan plan, demag_tree_export* o) {
  if (!plan || !o) return DEMAG_ERR_INVALID_ARG;
  return guarded([&] {
    Plan& P = *plan;
    cudaStream_t s = P.stream;
    const int64_t nc = P.ncells;
    copy_convert(o->node_key, P.node_key, P.nn, s);
    copy_convert(o->tet_key, P.tet_key, P.nt, s);
    copy_convert(o->node_perm, P.node_perm, P.nn, s);
    copy_convert(o->tet_perm, P.tet_perm, P.nt, s);
    copy_convert(o->cell_level, P.cell_level, nc, s);
    copy_convert(o->cell_prefix, P.cell_prefix, nc, s);
    copy_convert(o->cell_parent, P.cell_parent, nc, s);
    copy_convert(o->cell_centre, P.cell_centre, 3 * nc, s);
    copy_convert(o->m2l_off, P.m2l_off, nc + 1, s);
    copy_convert(o->m2l_src, P.m2l_src, P.n_m2l, s);
    copy_convert(o->p2p_off, P.p2p_off, nc + 1, s);
    copy_convert(o->p2p_src, P.p2p_src, P.n_p2p, s);
    if (o->cell_ranges) {
      std::vector<int4> h(nc);
      DM_CUDA(cudaMemcpyAsync(h.data(), P.cell_range, nc * sizeof(int4), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      for (int64_t c = 0; c < nc; c++) {
        o->cell_ranges[4 * c] = h[c].x;
        o->cell_ranges[4 * c + 1] = h[c].y;
        o->cell_ranges[4 * c + 2] = h[c].z;
        o->cell_ranges[4 * c + 3] = h[c].w;
      }
    }
    if (o->cell_child) {
      std::vector<int32_t> c0(nc), cn(nc);
      DM_CUDA(cudaMemcpyAsync(c0.data(), P.cell_child0, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaMemcpyAsync(cn.data(), P.cell_nchild, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      for (int64_t c = 0; c < nc; c++) {
        o->cell_child[2 * c] = c0[c];
        o->cell_child[2 * c + 1] = cn[c];
      }
    }
    if (o->cell_radius) {
      std::vector<double> rs(nc), rt(nc);
      DM_CUDA(cudaMemcpyAsync(rs.data(), P.cell_rsrc, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaMemcpyAsync(rt.data(), P.cell_rtgt, nc * sizeof(double), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      for (int64_t c = 0; c < nc; c++) {
        o->cell_radius[2 * c] = rs[c];
        o->cell_radius[2 * c + 1] = rt[c];
      }
    }
  });
}

const char* demag_status_string(demag_status s) {
  switch (s) {
    case DEMAG_OK: return "ok";
    case DEMAG_ERR_INVALID_ARG: return "invalid argument";
    case DEMAG_ERR_DEGENERATE_TET: return "degenerate tetrahedron";
    case DEMAG_ERR_OUT_OF_MEMORY: return "out of device memory";
    case DEMAG_ERR_CUDA: return "CUDA error";
    case DEMAG_ERR_TIMEOUT: return "device wait timed out";
    case DEMAG_ERR_UNSUPPORTED: return "unsupported option";
    case DEMAG_ERR_INTERNAL: return "plan audit failed";
  }
  return "unknown status";
}

const char* demag_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
