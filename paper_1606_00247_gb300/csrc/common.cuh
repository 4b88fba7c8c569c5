// common.cuh -- internal declarations shared by the translation units of
// libdemag.so: the plan structure, error plumbing, multi-index helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/demag.h"

namespace demag {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
struct Error {
  demag_status status;
  std::string msg;
};
void set_last_error(const std::string& msg);
[[noreturn]] void fail(demag_status s, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define DM_CUDA(x) ::demag::check_cuda((x), #x, __FILE__, __LINE__)
#define DM_LAUNCH(what) ::demag::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__)

// Octree constants (Sec. 3.1 reading): 21 bits per axis, cells split up to level 20.
constexpr int KEY_BITS = 21;
constexpr int MAX_LEVEL = 20;
constexpr int MAX_P = 12;
constexpr int MAX_NCOEF = (MAX_P + 1) * (MAX_P + 2) * (MAX_P + 3) / 6;  // 455
constexpr int NF_ROWS = 128;  // target nodes per tile of the tensor-core near field (MMA N <= 128)

__host__ __device__ inline int ncoef_of(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// one coefficient of an FP32 octree translation: target coefficient += (bit
// `octant` of neg ? -c : c) * source coefficient k (octant of the child cell)
struct TEnt {
  uint16_t k;
  uint8_t neg;
  uint8_t pad;
  float c;
};

// Graded multi-index order: total degree t ascending; within t, n_x descending,
// then n_z ascending.  Index of (a,b,c):
//   t(t+1)(t+2)/6 + (b+c)(b+c+1)/2 + c,  t = a+b+c.
__host__ __device__ inline int mi_index(int a, int b, int c) {
  int t = a + b + c, j = b + c;
  return t * (t + 1) * (t + 2) / 6 + j * (j + 1) / 2 + c;
}
__host__ __device__ inline void mi_decode(int idx, int& a, int& b, int& c) {
  int t = 0;
  while ((t + 1) * (t + 2) * (t + 3) / 6 <= idx) t++;
  int r = idx - t * (t + 1) * (t + 2) / 6;
  int j = 0;
  while ((j + 1) * (j + 2) / 2 <= r) j++;
  c = r - j * (j + 1) / 2;
  b = j - c;
  a = t - j;
}

// ---------------------------------------------------------------------------
// per-tet record used by the near field (sorted tet order, 66 doubles):
//   [0..11]  vertices v0..v3
//   [12..23] unit outward face normals n_F (face F opposite vertex F)
//   [24..59] unit outward in-plane edge normals m_{F,e}, edge e of face F
//   [60..65] edge lengths of the 6 edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3)
// Tets are stored positively oriented (vertices 2,3 swapped when needed) so the
// faces have the fixed counter-clockwise vertex orders below.
// ---------------------------------------------------------------------------
constexpr int TET_GEO = 66;
// per-tet, per-state record for the on-the-fly near field of small batches
// (56 doubles):
//   [0..2] M(v0)  [3..11] J = dM/dx (row a = component)  [12..23] alpha_{F,e}
//   [24..35] beta_{F,e}  [36..47] mu_{F,e}  [48..51] gamma_F  [52..55] eps_F
constexpr int TET_STATE = 56;

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct Plan;
struct Workspace;

struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct Plan {
  int device = 0;
  cudaStream_t stream = nullptr;  // plan-build stream
  demag_options opt{};
  int p = 4, nc = 35, nc1 = 20;   // order, ncoef(p), ncoef(p-1)
  int64_t nn = 0, nt = 0;
  double lo[3] = {0, 0, 0}, side = 0, scale = 0;
  double plan_ms = 0;
  float tuned_leaf_ms = 0;  // leaf-size tuning: device time of one evaluation of max_batch states
  int tune_source = 0;      // 0: no tuning asked, 1: tuned by timing, 2: choices read from the tuner cache
  int tc_preset_nt = 0, tc_preset_kps = 0, tc_preset_budget = 0;  // M2L launch shape from the tuner cache

  // sorted geometry
  double* nodes_s = nullptr;      // nn x 3 (sorted node order)
  int32_t* tets_s = nullptr;      // nt x 4 sorted node ids, positively oriented
  int32_t* node_perm = nullptr;   // sorted -> original
  int32_t* tet_perm = nullptr;
  uint64_t* node_key = nullptr;   // original order
  uint64_t* tet_key = nullptr;
  double* tet_geo = nullptr;      // nt x TET_GEO
  double* tet_grad = nullptr;     // nt x 12 gradients of the barycentric coords
  double* tet_vol = nullptr;      // nt, |vol|
  double* node_vol = nullptr;     // nn, lumped nodal volume (original order), on first use
  double* node_vol_s = nullptr;   // nn, lumped nodal volume (sorted order), point-dipole sources

  // cells
  int64_t ncells = 0;
  int nlevels = 0;
  std::vector<int64_t> level_start;  // host, nlevels+1
  uint64_t* cell_prefix = nullptr;
  int32_t* cell_level = nullptr;
  int4* cell_range = nullptr;       // tet begin,end, node begin,end
  int32_t* cell_parent = nullptr;
  int32_t* cell_child0 = nullptr;
  int32_t* cell_nchild = nullptr;
  double* cell_centre = nullptr;    // ncells x 3
  double* cell_rsrc = nullptr;
  double* cell_rtgt = nullptr;
  int64_t nleaves = 0;

  // interaction lists (CSR by target cell)
  int64_t n_m2l = 0, n_p2p = 0, n_p2p_pairs = 0;
  int64_t* m2l_off = nullptr;
  int32_t* m2l_src = nullptr;
  int64_t* p2p_off = nullptr;
  int32_t* p2p_src = nullptr;
  // host copies used for launch shapes
  std::vector<int32_t> h_m2l_targets;  // cells with non-empty M2L lists
  std::vector<int32_t> h_p2p_targets;  // leaves with nodes and non-empty P2P lists
  int32_t* m2l_targets = nullptr;      // device copies of the two lists above
  int32_t* p2p_targets = nullptr;

  // targets
  int32_t* node_leaf = nullptr;     // sorted node -> leaf cell
  int32_t* node_leaves = nullptr;   // leaves holding nodes (their nodes are cell_range[c].z .. .w)
  int64_t n_node_leaves = 0;
  // source leaves: support nodes (unique nodes of the leaf's tets)
  int64_t n_sup = 0;
  int64_t* sup_off = nullptr;       // ncells + 1
  int32_t* sup_node = nullptr;      // n_sup sorted node ids
  int32_t* tet_col = nullptr;       // nt x 4: column of each vertex in its leaf's support
  std::vector<int32_t> h_src_leaves;// leaves holding tets
  int32_t* src_leaves = nullptr;
  double* Ghat = nullptr;           // n_sup x nc1 : int lambda_k y^m/m! over the leaf's tets at that node

  // node -> incident tets (for lumped H)
  int64_t* nt_off = nullptr;        // nn + 1
  int32_t* nt_tet = nullptr;        // 4 nt, sorted tet ids

  // host copies of the shapes (plan time)
  std::vector<int4> h_range;
  std::vector<int64_t> h_p2p_off;
  std::vector<int32_t> h_p2p_src;

  // precomputed near field (near_mode = 1), per P2P target leaf ti:
  //   columns = unique source nodes of the tets of its P2P source leaves,
  //   W[w_off[ti] + (col * n_T + i) * 3 + c] = sum over those tets t ni col of
  //   int_t lambda_col(r') (r_i - r')_c / |r_i - r'|^3 dV'
  int64_t n_wcols = 0, n_wentries = 0;
  int64_t* w_coloff = nullptr;      // nT + 1
  int32_t* w_cols = nullptr;        // sorted node ids
  int64_t* w_off = nullptr;         // nT + 1, in units of doubles
  double* W64 = nullptr;
  int64_t* w_off32 = nullptr;       // nT + 1, in floats; W32 is [col][node][4]
  float* W32 = nullptr;

  // the same coefficients for the tensor-core near field (split-BF16
  // precisions, near_mode = 1; near_tc.cu): tiles of at most NF_ROWS target
  // nodes of consecutive P2P target leaves (leaves ordered by first node), the
  // union of their columns in groups of 16, W in split BF16 per k-step
  // (group, component) in the tensor-core K-major layout
  int64_t nf_ntiles = 0, nf_ncols = 0, nf_wbytes = 0;
  int64_t* nf_woff = nullptr;       // ntiles: byte offset of the tile in nf_W
  int64_t* nf_coff = nullptr;       // ntiles: first column of the tile in nf_cols
  int32_t* nf_ng = nullptr;         // ntiles: column groups of 16
  int32_t* nf_npad = nullptr;       // ntiles: rows padded to 16
  int32_t* nf_rownode = nullptr;    // ntiles x NF_ROWS: sorted node of each row, -1 = none
  int32_t* nf_cols = nullptr;       // sorted node of each column (groups padded with the last column)
  int32_t* nf_order = nullptr;      // ntiles: launch order, by decreasing column groups
  unsigned char* nf_W = nullptr;
  float* nf_S = nullptr;            // nn x 3: row sums S_i = sum_j W_ij of the coefficients (FP64 sums)

  // tensor-core M2L (TF32 / split BF16): one operator tile set per distinct
  // (level difference, lattice offset) and the operator index of every pair
  int64_t n_tc_ops = 0;
  unsigned char* tc_ops = nullptr;
  int32_t* m2l_op = nullptr;        // n_m2l
  float* m2l_tab = nullptr;         // n_tc_ops x nc: FP32 b_k(v) per key (CUDA-core M2L)
  int32_t* m2l_tab_opdl = nullptr;  // n_m2l: key index | (level difference & 255) << 24
  uint32_t* m2l_rc_items = nullptr; // row-chunk items (m | c << 16), then per row a CSR of its items
  int m2l_rc_nitems = 0, m2l_rc_ch = 0;
  int tc_nt = 1, tc_kps = 0, tc_budget = 0;  // M2L launch shape: targets per CTA, k-steps per slot, ring bytes
  int tc_ls = 0;                    // split BF16 limb scheme of the tensor-core M2L (m2l_tc.cu)
  int tc_prom_group = 0, tc_prom_rows = 16;  // accumulator promotion: sources per group (0 = off), rows
  int64_t* tc_g1_off = nullptr;     // one-target groups: list offsets in target order
  int64_t tc_n_g2 = 0;              // two-target groups (consecutive targets), union lists:
  int32_t* tc_g2_tgt = nullptr;     //   2 per group, -1 = none
  int64_t* tc_g2_off = nullptr;
  int32_t* tc_g2_src = nullptr;
  int32_t* tc_g2_op = nullptr;      //   2 per entry: each target's operator, -1 = not in its list

  // FP32 octree translations as coefficient lists (mixed precision):
  //   M2M: Qt^P_n += sum over entries e of n: sign_e(octant) c_e Qt^C_{k_e}
  //   L2L: Lt^C_m += sum over entries e of m: sign_e(octant) c_e Lt^P_{k_e}
  int32_t* m2m_eoff = nullptr;      // nc + 1
  TEnt* m2m_ent = nullptr;
  int32_t* l2l_eoff = nullptr;      // nc + 1
  TEnt* l2l_ent = nullptr;
  int32_t* par_list = nullptr;      // cells with children, level by level
  std::vector<int64_t> par_start;   // host, nlevels + 1: parents of level l are par_list[par_start[l] ..]
  // FP32 mass-lumped gradient operator (mixed precision), rows by sorted node:
  //   H_i = sum_e w_e u_{col_e},  w_e = -(1/V_i) sum_{t ni i, col_e} vol_t grad lambda_{col_e}^t
  int64_t* hg_off = nullptr;        // nn + 1
  int32_t* hg_col = nullptr;
  float4* hg_w = nullptr;           // (x, y, z, 0)
  int32_t* node_iperm = nullptr;    // original -> sorted node

  // FP32 far-field operators (mixed precision, per-level scaled)
  float* Ghat32 = nullptr;          // n_sup x nc1: Ghat[e][m] / s_leaf^(|m|+1)

  std::vector<DevBuf> bufs;
  int64_t device_bytes = 0;
  Workspace* ws = nullptr;
  int* last_err = nullptr;          // device error flag of the most recent evaluation (demag_eval_status)
  uint8_t* bnd_flag = nullptr;      // pointwise field: sorted nodes on a boundary face (on first use)
  double* field_buf = nullptr;      // pointwise field: [sorted node][3][state]
  int field_states = 0;
  int debug_flags = 0;              // demag_plan_debug: test hooks (bit 0: near-field stall, bit 1: planted audit entry)

  // per-stage timers (opt.profile) and launch counts
  double stage_ms[DEMAG_N_STAGES] = {};
  int64_t stage_launches[DEMAG_N_STAGES] = {};
  int64_t n_evals_profiled = 0;
  int64_t eval_launches = 0;
};

// Records CUDA events around the stages of one demag_eval when profiling is on
// and counts kernel launches always; each stage is also an NVTX range (host
// side, seen by profilers that attach to NVTX, free otherwise).
struct StageClock {
  Plan& P;
  cudaStream_t s;
  bool on;
  cudaEvent_t ev[2 * DEMAG_N_STAGES];
  int launches[DEMAG_N_STAGES] = {};
  bool used[DEMAG_N_STAGES] = {};
  int cur = -1;
  uint64_t range = 0;  // open NVTX range of the current stage (0: none)
  StageClock(Plan& P_, cudaStream_t s_, bool allow = true);
  ~StageClock();
  void begin(int stage);
  void end();
  void launched(int n = 1) { launches[cur] += n; }
  void finish();  // synchronises on the last event and accumulates
};

template <class T>
T* dalloc(Plan& P, size_t n) {
  void* p = nullptr;
  size_t bytes = n * sizeof(T);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(DEMAG_ERR_OUT_OF_MEMORY, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  P.bufs.push_back({p, bytes});
  P.device_bytes += (int64_t)bytes;
  return (T*)p;
}
void dfree_all(Plan& P);
void dfree(Plan& P, void* ptr);  // one plan buffer, before the plan is destroyed

// stages (defined in plan.cu / fmm.cu / p2p.cu / eval.cu)
void build_plan(Plan& P, const double* nodes, const int32_t* tets);
// opt a kernel in to `bytes` of dynamic shared memory on the current device
// (set once per kernel, device and size; thread-safe)
void smem_opt_in(const void* func, size_t bytes);
// bounds audit of every index list of the plan (audit.cu); plant: also audit a
// copy of the M2L source list with one entry out of range (test hook)
void audit_plan(Plan& P, bool plant = false);
void eval_fp64(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s);
void destroy_workspace(Plan& P);
// pointwise field at the interior nodes (field.cu)
void eval_field(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s);

// evaluation workspace (one per plan, sized for max_batch states)
struct Workspace {
  int B = 0;
  double *Ms = nullptr, *Q = nullptr, *L = nullptr, *u_s = nullptr, *state = nullptr;
  float *Ms32 = nullptr, *Q32 = nullptr, *L32 = nullptr, *u32 = nullptr;
  unsigned char* QP = nullptr;  // moments in the tensor-core tile layout (TF32 / split BF16 M2L)
  float* MP = nullptr;          // tensor-core near field: M per 128-state block, [block][node][3][128]
  double *M_dev = nullptr, *u_dev = nullptr, *H_dev = nullptr;  // staging for host pointers
  int* err = nullptr;
  std::vector<void*> ptrs;
};
Workspace& workspace(Plan& P, int B);
// the two drivers on a given workspace (profile_ok = false: no CUDA events are created)
void eval_fp64_ws(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, cudaStream_t s,
                  bool profile_ok);
void eval_mixed_ws(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, cudaStream_t s,
                   bool profile_ok);
bool is_device_ptr(const void* p);
// shared FP64 stages (fmm.cu)
bool eval_io_begin(Plan& P, Workspace& W, const double* M, int B, double* u, double* H, const double** Md, double** ud,
                   double** Hd, cudaStream_t s);
void eval_io_end(Plan& P, Workspace& W, bool dev, int B, double* u, double* H, cudaStream_t s);
void near_field_fp64(Plan& P, Workspace& W, int B, StageClock& clk, cudaStream_t s);
void launch_gather_M(Plan& P, const double* M, int B, double* Ms, cudaStream_t s);
void launch_lumped_H_out(Plan& P, int B, const double* u_s, double* u, double* H, cudaStream_t s);

// precomputed near field (near.cu)
void build_near_field(Plan& P);
void launch_near_apply64(Plan& P, const double* Ms, int B, double* u_s, cudaStream_t s);
void launch_near_apply32(Plan& P, const float* Ms, int B, float* u_s, int* err, cudaStream_t s);
// tensor-core near field (near_tc.cu): used when the plan holds the tiles
bool near_tc_wanted(const Plan& P);
// MP: workspace of nf_mp_floats(P, B) floats for M in the layout of the kernel's bulk copies
size_t nf_mp_floats(const Plan& P, int B);
void launch_near_tc(Plan& P, const float* Ms, float* MP, int B, float* u_s, int* err, cudaStream_t s);
struct M2lKeys {  // distinct translation keys (dl, lattice offset) and the key of every M2L pair
  bool ok = false;
  std::vector<int4> keys;
  std::vector<int64_t> off;           // host copy of m2l_off
  std::vector<int32_t> src, op;       // host copies of m2l_src and of the key index per pair
};
// mixed-precision far field (fmm32.cu)
void build_mixed_operators(Plan& P);
void eval_mixed(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s);
bool launch_m2l32_fast(Plan& P, int B, const float* Q, float* L, int* err, cudaStream_t s);  // m2l32.cu
// FP32 table-driven M2L on CUDA cores (m2l32.cu): derivative table per key at
// plan time; launch returns false when the plan has no table
void build_m2l_tab(Plan& P, const M2lKeys& K);
bool launch_m2l32_tab(Plan& P, int B, const float* Q, float* L, cudaStream_t s);
// largest batch for which the tensor-core precisions run the table-driven FP32
// M2L instead of the tensor-core one (whose tiles hold 128 states)
inline int m2l_table_batch(const Plan& P) {
  return P.opt.m2l_table_batch < 0 ? 0 : (P.opt.m2l_table_batch == 0 ? 8 : P.opt.m2l_table_batch);
}
// several plans in one submission (multi.cu); cached graphs of a plan are
// dropped before the plan or its workspace goes away
void eval_multi(Plan* const* plans, int n, const double* const* M, const int* batch, double* const* u,
                double* const* H, cudaStream_t s);
void multi_forget_plan(const Plan* P);
// energy and LLG stepping (llg.cu); device pointers, user layout (B, N_n, 3)
const double* node_volumes(Plan& P);
void energy(Plan& P, const double* M, const double* H, int B, double* e, cudaStream_t s);
void llg_rk4(Plan& P, double* m, int B, double Ms, double alpha, const double* hext, double dt, int steps,
             cudaStream_t s);
// tensor-core M2L (m2l_tc.cu): operator table at plan time; bytes of the packed
// moments for B states (0 when the tensor-core M2L is off); packs Q into QP and
// runs the M2L (false: not available for this plan, use the CUDA-core M2L)
M2lKeys build_m2l_keys(Plan& P);      // also fills P.m2l_op
void build_m2l_tc(Plan& P, const M2lKeys& K);
size_t m2l_tc_pack_bytes(const Plan& P, int B);
bool launch_m2l_tc(Plan& P, int B, const float* Q, unsigned char* QP, float* L, int* err, cudaStream_t s);

// near field (p2p.cu)
void build_tet_geometry(Plan& P);
// FP64 on-the-fly near field.  Batches of P2P_AT_MIN_B states or more: the
// pair geometry once per (target, tet), contracted with every state (Ms);
// smaller batches: pair by pair and state by state on the per-tet records
// of launch_tet_state (state).
constexpr int P2P_AT_MIN_B = 2;
void launch_tet_state(Plan& P, const double* Ms, int B, double* state, cudaStream_t s);
void launch_p2p_fp64(Plan& P, const double* Ms, const double* state, int B, double* u_s, int* err_flag,
                     cudaStream_t s);

}  // namespace demag

// the opaque handle of the C ABI is the plan itself
struct demag_plan_s : demag::Plan {};
