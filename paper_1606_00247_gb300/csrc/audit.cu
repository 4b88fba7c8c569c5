// audit.cu -- bounds audit of the plan's index lists, on the device.
//
// Every list that an evaluation kernel follows into another array (node and
// tet permutations, cell links and ranges, the CSR interaction lists of
// Sec. 3.3, support nodes, near-field columns and tile rows, M2L operator
// indices and groups, gradient-operator columns) is written once, while the
// plan is built, and only read afterwards.  Checking each entry once here is
// therefore the same guarantee as a bounds check at every read, at no cost to
// an evaluation, and without a device assert (which would end the context).
// Each list's count is first checked against the size of the allocation it
// lives in (a list whose count runs past it is reported, not read).
// A failed check is a planner bug: the plan is not returned and
// demag_last_error() names the list, the first bad position and its value.
#include <climits>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace demag {

namespace {

struct AuditOut {
  unsigned long long bad;    // entries that failed
  unsigned long long first;  // first failing position (ULLONG_MAX: none)
};

__device__ __forceinline__ void audit_fail(AuditOut* o, int64_t i) {
  atomicAdd(&o->bad, 1ull);
  atomicMin(&o->first, (unsigned long long)i);
}

// lo <= (a[i] & mask) < hi for every i < n (mask = -1: the value itself)
template <class T>
__global__ void k_audit_values(const T* __restrict__ a, int64_t n, int64_t mask, int64_t lo, int64_t hi, AuditOut* o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = (int64_t)a[i] & mask;
    if (v < lo || v >= hi) audit_fail(o, i);
  }
}

// n + 1 non-decreasing offsets within [lo, hi]; first = off[0] and last = off[n] when >= 0
__global__ void k_audit_offsets(const int64_t* __restrict__ off, int64_t n, int64_t lo, int64_t hi, int64_t first,
                                int64_t last, AuditOut* o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = off[i];
    bool ok = v >= lo && v <= hi;
    if (i < n) ok = ok && v <= off[i + 1];
    if (i == 0 && first >= 0) ok = ok && v == first;
    if (i == n && last >= 0) ok = ok && v == last;
    if (!ok) audit_fail(o, i);
  }
}

// cell ranges: 0 <= tet begin <= tet end <= nt, 0 <= node begin <= node end <= nn
__global__ void k_audit_ranges(const int4* __restrict__ r, int64_t n, int64_t nt, int64_t nn, AuditOut* o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int4 v = r[i];
    if (!(0 <= v.x && v.x <= v.y && v.y <= nt && 0 <= v.z && v.z <= v.w && v.w <= nn)) audit_fail(o, i);
  }
}

// child links: 0 <= nchild <= 8; children of a parent lie after it and inside the cell array
__global__ void k_audit_children(const int32_t* __restrict__ child0, const int32_t* __restrict__ nchild, int64_t n,
                                 AuditOut* o) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int k = nchild[i];
    if (k < 0 || k > 8 || (k > 0 && (child0[i] <= i || (int64_t)child0[i] + k > n))) audit_fail(o, i);
  }
}

// a device scratch array freed on scope exit
struct Scratch32 {
  int32_t* p = nullptr;
  explicit Scratch32(int64_t n) {
    if (cudaMalloc(&p, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)) != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "plan audit scratch");
    }
  }
  ~Scratch32() {
    if (p) cudaFree(p);
  }
};

struct Check {
  std::string name;
  const void* ptr;
  int esize;  // bytes of one entry (its value is read back for the message), 0 = none
};

class Auditor {
 public:
  explicit Auditor(Plan& P) : P_(P), s_(P.stream) {}

  template <class T>
  void values(const char* name, const T* a, int64_t n, int64_t lo, int64_t hi, int64_t mask = -1) {
    if (!begin(name, a, n, sizeof(T), n * (int64_t)sizeof(T))) return;
    k_audit_values<T><<<grid(n), 256, 0, s_>>>(a, n, mask, lo, hi, out(name));
    DM_LAUNCH("k_audit_values");
  }
  void offsets(const char* name, const int64_t* off, int64_t n, int64_t lo, int64_t hi, int64_t first, int64_t last) {
    if (!begin(name, off, n + 1, sizeof(int64_t), (n + 1) * (int64_t)sizeof(int64_t))) return;
    k_audit_offsets<<<grid(n + 1), 256, 0, s_>>>(off, n, lo, hi, first, last, out(name));
    DM_LAUNCH("k_audit_offsets");
  }
  void ranges(const char* name, const int4* r, int64_t n) {
    if (!begin(name, r, n, 0, n * (int64_t)sizeof(int4))) return;
    k_audit_ranges<<<grid(n), 256, 0, s_>>>(r, n, P_.nt, P_.nn, out(name));
    DM_LAUNCH("k_audit_ranges");
  }
  void children(const char* name, const int32_t* child0, const int32_t* nchild, int64_t n) {
    if (!begin(name, child0, n, 0, n * (int64_t)sizeof(int32_t))) return;
    k_audit_children<<<grid(n), 256, 0, s_>>>(child0, nchild, n, out(name));
    DM_LAUNCH("k_audit_children");
  }
  // the last of n + 1 device offsets (the length of the list they index)
  int64_t last(const int64_t* off, int64_t n) {
    int64_t v = 0;
    if (!off) return 0;
    DM_CUDA(cudaMemcpyAsync(&v, off + n, sizeof v, cudaMemcpyDeviceToHost, s_));
    DM_CUDA(cudaStreamSynchronize(s_));
    return v;
  }

  void finish() {
    if (!checks_.empty()) {
      std::vector<AuditOut> h(checks_.size());
      DM_CUDA(cudaMemcpyAsync(h.data(), dout_, sizeof(AuditOut) * h.size(), cudaMemcpyDeviceToHost, s_));
      DM_CUDA(cudaStreamSynchronize(s_));
      for (size_t k = 0; k < h.size(); k++) {
        if (h[k].bad == 0) continue;
        const Check& c = checks_[k];
        std::string msg = "plan audit: " + c.name + "[" + std::to_string(h[k].first) + "]";
        if (c.esize == 4 || c.esize == 8) {
          int64_t v = 0;
          int32_t v32 = 0;
          const char* src = (const char*)c.ptr + h[k].first * (unsigned long long)c.esize;
          DM_CUDA(cudaMemcpy(c.esize == 4 ? (void*)&v32 : (void*)&v, src, c.esize, cudaMemcpyDeviceToHost));
          msg += " = " + std::to_string(c.esize == 4 ? (int64_t)v32 : v);
        }
        msg += " out of range (" + std::to_string(h[k].bad) + " entries)";
        release();
        fail(DEMAG_ERR_INTERNAL, msg);
      }
    }
    if (!error_.empty()) {
      release();
      fail(DEMAG_ERR_INTERNAL, error_);
    }
    release();
  }
  ~Auditor() { release(); }

 private:
  static unsigned grid(int64_t n) { return (unsigned)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 4096); }

  // size of the plan allocation that starts at p (0: not a plan allocation)
  size_t alloc_bytes(const void* p) const {
    for (const DevBuf& b : P_.bufs)
      if (b.ptr == p) return b.bytes;
    return 0;
  }

  bool begin(const char* name, const void* p, int64_t n, int esize, int64_t bytes) {
    if (n <= 0) return false;
    if (!p) {
      if (error_.empty()) error_ = std::string("plan audit: ") + name + " is missing (" + std::to_string(n) + " entries)";
      return false;
    }
    const size_t cap = alloc_bytes(p);
    if (cap && (size_t)bytes > cap) {  // the list's own count runs past its allocation: not read
      if (error_.empty())
        error_ = std::string("plan audit: ") + name + " counts " + std::to_string(n) + " entries, its allocation " +
                 std::to_string(cap) + " bytes";
      return false;
    }
    checks_.push_back(Check{name, p, esize});
    return true;
  }

  AuditOut* out(const char*) {
    const size_t k = checks_.size() - 1;
    if (k >= cap_) {  // grow the result array (results of earlier checks are still in flight)
      const size_t nc = std::max<size_t>(64, 2 * cap_);
      AuditOut* d = nullptr;
      if (cudaMalloc(&d, sizeof(AuditOut) * nc) != cudaSuccess) {
        cudaGetLastError();
        fail(DEMAG_ERR_OUT_OF_MEMORY, "plan audit buffers");
      }
      if (dout_) {
        DM_CUDA(cudaMemcpyAsync(d, dout_, sizeof(AuditOut) * cap_, cudaMemcpyDeviceToDevice, s_));
        DM_CUDA(cudaStreamSynchronize(s_));
        cudaFree(dout_);
      }
      dout_ = d;
      cap_ = nc;
    }
    const AuditOut init{0ull, ULLONG_MAX};
    DM_CUDA(cudaMemcpyAsync(dout_ + k, &init, sizeof init, cudaMemcpyHostToDevice, s_));
    DM_CUDA(cudaStreamSynchronize(s_));  // init is a host temporary
    return dout_ + k;
  }

  void release() {
    if (dout_) cudaFree(dout_);
    dout_ = nullptr;
    cap_ = 0;
  }

  Plan& P_;
  cudaStream_t s_;
  std::vector<Check> checks_;
  AuditOut* dout_ = nullptr;
  size_t cap_ = 0;
  std::string error_;
};

}  // namespace

void audit_plan(Plan& P, bool plant) {
  Auditor A(P);
  const int64_t nn = P.nn, nt = P.nt, nc = P.ncells;
  // sorted geometry and the octree (Sec. 3.1)
  A.values("node_perm", P.node_perm, nn, 0, nn);
  A.values("tet_perm", P.tet_perm, nt, 0, nt);
  A.values("tets_s", P.tets_s, 4 * nt, 0, nn);
  A.values("cell_level", P.cell_level, nc, 0, MAX_LEVEL + 1);
  A.values("cell_parent", P.cell_parent, nc, -1, nc);
  A.ranges("cell_range", P.cell_range, nc);
  A.children("cell_child0", P.cell_child0, P.cell_nchild, nc);
  A.values("node_leaf", P.node_leaf, nn, 0, nc);
  A.values("node_leaves", P.node_leaves, P.n_node_leaves, 0, nc);
  A.values("src_leaves", P.src_leaves, (int64_t)P.h_src_leaves.size(), 0, nc);
  A.offsets("nt_off", P.nt_off, nn, 0, 4 * nt, 0, 4 * nt);
  A.values("nt_tet", P.nt_tet, 4 * nt, 0, nt);
  // interaction lists (Sec. 3.3)
  A.offsets("m2l_off", P.m2l_off, nc, 0, P.n_m2l, 0, P.n_m2l);
  A.values("m2l_src", P.m2l_src, P.n_m2l, 0, nc);
  A.offsets("p2p_off", P.p2p_off, nc, 0, P.n_p2p, 0, P.n_p2p);
  A.values("p2p_src", P.p2p_src, P.n_p2p, 0, nc);
  A.values("m2l_targets", P.m2l_targets, (int64_t)P.h_m2l_targets.size(), 0, nc);
  A.values("p2p_targets", P.p2p_targets, (int64_t)P.h_p2p_targets.size(), 0, nc);
  // source-leaf supports (P2M)
  A.offsets("sup_off", P.sup_off, nc, 0, P.n_sup, 0, P.n_sup);
  A.values("sup_node", P.sup_node, P.n_sup, 0, nn);
  // stored near field
  if (P.opt.near_mode == 1) {
    const int64_t nT = (int64_t)P.h_p2p_targets.size();
    A.offsets("w_coloff", P.w_coloff, nT, 0, P.n_wcols, 0, P.n_wcols);
    A.offsets("w_off", P.w_off, nT, 0, P.n_wentries, 0, P.n_wentries);
    if (P.nf_ntiles > 0) {
      const int64_t nq = P.nf_ntiles;
      A.values("nf_cols", P.nf_cols, P.nf_ncols, 0, nn);
      A.values("nf_rownode", P.nf_rownode, nq * NF_ROWS, -1, nn);
      A.values("nf_order", P.nf_order, nq, 0, nq);
      A.values("nf_coff", P.nf_coff, nq, 0, P.nf_ncols + 1);
      A.values("nf_woff", P.nf_woff, nq, 0, P.nf_wbytes + 1);
      A.values("nf_ng", P.nf_ng, nq, 0, P.nf_ncols / 16 + 1);
      A.values("nf_npad", P.nf_npad, nq, 0, NF_ROWS + 1);
    } else {
      A.values("w_cols", P.w_cols, P.n_wcols, 0, nn);
      if (P.w_off32) A.offsets("w_off32", P.w_off32, nT, 0, P.n_wentries / 3 * 4, 0, P.n_wentries / 3 * 4);
    }
  }
  // mixed path: gradient operator, parent lists, M2L operator indices and groups
  if (P.opt.precision != DEMAG_FP64) {
    A.values("node_iperm", P.node_iperm, nn, 0, nn);
    const int64_t nh = A.last(P.hg_off, nn);
    A.offsets("hg_off", P.hg_off, nn, 0, nh, 0, nh);
    A.values("hg_col", P.hg_col, nh, 0, nn);
    A.values("par_list", P.par_list, P.par_start.empty() ? 0 : P.par_start.back(), 0, nc);
    if (P.m2l_op) A.values("m2l_op", P.m2l_op, P.n_m2l, 0, P.n_tc_ops);
    if (P.m2l_tab_opdl) A.values("m2l_tab_opdl", P.m2l_tab_opdl, P.n_m2l, 0, P.n_tc_ops, 0x00ffffff);
    if (P.tc_g1_off)
      A.offsets("tc_g1_off", P.tc_g1_off, (int64_t)P.h_m2l_targets.size(), 0, P.n_m2l, -1, -1);
    if (P.tc_n_g2 > 0) {
      const int64_t ne = A.last(P.tc_g2_off, P.tc_n_g2);
      A.values("tc_g2_tgt", P.tc_g2_tgt, 2 * P.tc_n_g2, -1, nc);
      A.offsets("tc_g2_off", P.tc_g2_off, P.tc_n_g2, 0, ne, 0, ne);
      A.values("tc_g2_src", P.tc_g2_src, ne, 0, nc);
      A.values("tc_g2_op", P.tc_g2_op, 2 * ne, -1, P.n_tc_ops);
    }
  }
  // test hook: a scratch copy of the M2L source list with its last entry set
  // to n_cells (read by this audit only; the plan's own list is untouched)
  if (plant && P.n_m2l > 0) {
    Scratch32 bad(P.n_m2l);
    DM_CUDA(cudaMemcpyAsync(bad.p, P.m2l_src, sizeof(int32_t) * P.n_m2l, cudaMemcpyDeviceToDevice, P.stream));
    const int32_t v = (int32_t)nc;
    DM_CUDA(cudaMemcpyAsync(bad.p + P.n_m2l - 1, &v, sizeof v, cudaMemcpyHostToDevice, P.stream));
    DM_CUDA(cudaStreamSynchronize(P.stream));
    A.values("m2l_src (planted copy)", bad.p, P.n_m2l, 0, nc);
    A.finish();  // before the copy is freed
    return;
  }
  A.finish();
}

}  // namespace demag
