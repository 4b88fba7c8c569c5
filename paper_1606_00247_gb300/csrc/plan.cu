// plan.cu -- plan construction on the GPU: validation, Morton keys, sort,
// octree, cell centres and radii, dual tree traversal into M2L / P2P lists,
// source-leaf supports and exact-moment operators.
//
// Octree and lists follow Sec. 3.1-3.3 of Palmesi et al. with these readings
// (the paper leaves them open):
//  * bounding cube: lo = min over nodes, side = (largest extent)*(1+2^-20),
//    scale = 2^21/side; q = min(2^21-1, trunc((x-lo)*scale)) per axis;
//  * 63-bit Morton key, bit b of q_x at 3b, q_y at 3b+1, q_z at 3b+2;
//  * nodes keyed by position, tets by centroid ((v0+v1)+(v2+v3))*0.25, both
//    sorted by (key, original index);
//  * split a cell iff it holds > leaf_size tets and level < 20; drop children
//    with neither tets nor nodes; number cells level by level, ascending prefix;
//  * centre = lo + (k+0.5) side/2^level; source radius = max distance to the
//    vertices of the cell's tets, target radius = max distance to its nodes
//    (the "most remote directly connected vertex" of Sec. 3.2 for tet clusters);
//  * MAC (Sec. 3.2): (r_T + r_S) < theta |c_T - c_S|;
//  * traversal of Listings 1-2, MAC tested first; split the target iff it is
//    the larger box and not a leaf, else the source if not a leaf, else the
//    target; drop pairs without target nodes or source tets.
// Every floating-point value that decides an integer is computed with
// explicitly rounded operations (__dadd_rn, __dmul_rn, __dsqrt_rn: no FMA
// contraction), so keys, cells and lists are reproducible bit for bit.
#include <cub/cub.cuh>

#include <algorithm>
#include <chrono>
#include <cmath>

#include "common.cuh"

namespace demag {

// ---------------------------------------------------------------------------
// small device-vector helper for temporaries of the build
// ---------------------------------------------------------------------------
template <class T>
struct Tmp {
  T* p = nullptr;
  size_t n = 0;
  Tmp() = default;
  explicit Tmp(size_t n_) { alloc(n_); }
  void alloc(size_t n_) {
    release();
    n = n_;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "temporary allocation failed");
    }
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  ~Tmp() { release(); }
  Tmp(const Tmp&) = delete;
  Tmp& operator=(const Tmp&) = delete;
};

struct CubTemp {
  void* p = nullptr;
  size_t bytes = 0;
  void need(size_t b) {
    if (b <= bytes) return;
    if (p) cudaFree(p);
    p = nullptr;
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "sort workspace allocation failed");
    }
    bytes = b;
  }
  ~CubTemp() {
    if (p) cudaFree(p);
  }
};

static inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------------------
// validation and bounding box
// ---------------------------------------------------------------------------
__global__ void k_validate(const double* __restrict__ nodes, int64_t nn, const int32_t* __restrict__ tets,
                           int64_t nt, int* flags) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  int32_t g[4];
  for (int k = 0; k < 4; k++) {
    g[k] = tets[4 * j + k];
    if (g[k] < 0 || g[k] >= nn) {
      atomicExch(&flags[0], 1);
      return;
    }
  }
  double v[4][3];
  for (int k = 0; k < 4; k++)
    for (int a = 0; a < 3; a++) v[k][a] = nodes[3 * (int64_t)g[k] + a];
  double e[3][3];
  for (int i = 0; i < 3; i++)
    for (int a = 0; a < 3; a++) e[i][a] = v[i + 1][a] - v[0][a];
  double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) - e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
               e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  double lmax = 0;
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      double dx = v[b][0] - v[a][0], dy = v[b][1] - v[a][1], dz = v[b][2] - v[a][2];
      lmax = fmax(lmax, sqrt(dx * dx + dy * dy + dz * dz));
    }
  if (!(fabs(det) / 6.0 >= 1e-14 * lmax * lmax * lmax)) atomicExch(&flags[1], 1);
}

__global__ void k_bbox_partial(const double* __restrict__ nodes, int64_t nn, double* out) {
  __shared__ double smin[3][256], smax[3][256];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
    for (int a = 0; a < 3; a++) {
      double x = nodes[3 * i + a];
      mn[a] = fmin(mn[a], x);
      mx[a] = fmax(mx[a], x);
    }
  for (int a = 0; a < 3; a++) {
    smin[a][threadIdx.x] = mn[a];
    smax[a][threadIdx.x] = mx[a];
  }
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int a = 0; a < 3; a++) {
        smin[a][threadIdx.x] = fmin(smin[a][threadIdx.x], smin[a][threadIdx.x + s]);
        smax[a][threadIdx.x] = fmax(smax[a][threadIdx.x], smax[a][threadIdx.x + s]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int a = 0; a < 3; a++) {
      out[6 * blockIdx.x + a] = smin[a][0];
      out[6 * blockIdx.x + 3 + a] = smax[a][0];
    }
}

// ---------------------------------------------------------------------------
// Morton keys
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread21(uint64_t x) {
  x &= 0x1fffffull;
  x = (x | (x << 32)) & 0x1f00000000ffffull;
  x = (x | (x << 16)) & 0x1f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}
__device__ __forceinline__ uint64_t quant(double x, double lo, double scale) {
  double s = __dmul_rn(__dsub_rn(x, lo), scale);
  uint64_t q = __double2ull_rz(s);
  return q > 0x1fffffull ? 0x1fffffull : q;
}
__device__ __forceinline__ uint64_t morton(double x, double y, double z, double3 lo, double scale) {
  return spread21(quant(x, lo.x, scale)) | (spread21(quant(y, lo.y, scale)) << 1) |
         (spread21(quant(z, lo.z, scale)) << 2);
}

__global__ void k_node_keys(const double* __restrict__ nodes, int64_t nn, double3 lo, double scale, uint64_t* key,
                            int32_t* idx) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  key[i] = morton(nodes[3 * i], nodes[3 * i + 1], nodes[3 * i + 2], lo, scale);
  idx[i] = (int32_t)i;
}

__global__ void k_tet_keys(const double* __restrict__ nodes, const int32_t* __restrict__ tets, int64_t nt, double3 lo,
                           double scale, uint64_t* key, int32_t* idx) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  double c[3];
  const int64_t g0 = tets[4 * j], g1 = tets[4 * j + 1], g2 = tets[4 * j + 2], g3 = tets[4 * j + 3];
  for (int a = 0; a < 3; a++)
    c[a] = __dmul_rn(__dadd_rn(__dadd_rn(nodes[3 * g0 + a], nodes[3 * g1 + a]),
                               __dadd_rn(nodes[3 * g2 + a], nodes[3 * g3 + a])),
                     0.25);
  key[j] = morton(c[0], c[1], c[2], lo, scale);
  idx[j] = (int32_t)j;
}

__global__ void k_apply_node_perm(const double* __restrict__ nodes, const int32_t* __restrict__ perm, int64_t nn,
                                  double* nodes_s, int32_t* rank) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  int32_t g = perm[i];
  for (int a = 0; a < 3; a++) nodes_s[3 * i + a] = nodes[3 * (int64_t)g + a];
  rank[g] = (int32_t)i;
}

__global__ void k_apply_tet_perm(const int32_t* __restrict__ tets, const int32_t* __restrict__ perm,
                                 const int32_t* __restrict__ rank, int64_t nt, int32_t* tets_s) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= nt) return;
  int64_t g = perm[j];
  for (int k = 0; k < 4; k++) tets_s[4 * j + k] = rank[tets[4 * g + k]];
}

// ---------------------------------------------------------------------------
// octree, one level per launch
// ---------------------------------------------------------------------------
// first index in [b, e) whose octant digit ((key >> shift) & 7) is >= o
__device__ __forceinline__ int32_t octant_lower(const uint64_t* key, int32_t b, int32_t e, int shift, int o) {
  while (b < e) {
    int32_t m = b + ((e - b) >> 1);
    if ((int)((key[m] >> shift) & 7ull) < o)
      b = m + 1;
    else
      e = m;
  }
  return b;
}

__global__ void k_count_children(const int4* __restrict__ range, int64_t lb, int64_t le, int level, int leaf,
                                  const uint64_t* __restrict__ tkey, const uint64_t* __restrict__ nkey, int32_t* nchild,
                                  int4* child_bounds /* (le-lb) x 8 : tet begin, node begin, -, - */) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= le - lb) return;
  int4 r = range[lb + i];
  int cnt = 0;
  if (r.y - r.x > leaf && level < MAX_LEVEL) {
    int shift = 3 * (KEY_BITS - 1 - level);
    for (int o = 0; o < 8; o++) {
      int32_t t0 = octant_lower(tkey, r.x, r.y, shift, o), t1 = octant_lower(tkey, r.x, r.y, shift, o + 1);
      int32_t n0 = octant_lower(nkey, r.z, r.w, shift, o), n1 = octant_lower(nkey, r.z, r.w, shift, o + 1);
      child_bounds[8 * i + o] = make_int4(t0, t1, n0, n1);
      cnt += (t1 > t0 || n1 > n0);
    }
  }
  nchild[lb + i] = cnt;
}

__global__ void k_write_children(int64_t lb, int64_t le, int level, const int32_t* __restrict__ nchild,
                                 const int32_t* __restrict__ excl, const int4* __restrict__ child_bounds,
                                 uint64_t* prefix, int32_t* clevel, int4* range, int32_t* parent, int32_t* child0) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= le - lb) return;
  int64_t c = lb + i;
  int32_t n = nchild[c];
  int32_t first = (int32_t)(le + excl[i]);
  child0[c] = n ? first : -1;
  if (!n) return;
  int k = 0;
  for (int o = 0; o < 8; o++) {
    int4 b = child_bounds[8 * i + o];
    if (b.y > b.x || b.w > b.z) {
      int64_t d = first + k++;
      prefix[d] = (prefix[c] << 3) | (uint64_t)o;
      clevel[d] = level + 1;
      range[d] = b;
      parent[d] = (int32_t)c;
    }
  }
}

// ---------------------------------------------------------------------------
// centres and radii
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t compact_axis(uint64_t prefix, int level, int axis) {
  uint32_t k = 0;
  for (int b = 0; b < level; b++) k |= (uint32_t)((prefix >> (3 * b + axis)) & 1ull) << b;
  return k;
}
__device__ __forceinline__ double dist_rn(double ax, double ay, double az, double bx, double by, double bz) {
  double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
  return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__global__ void k_centres(int64_t ncells, const uint64_t* __restrict__ prefix, const int32_t* __restrict__ level,
                          double3 lo, double side, double* centre) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int l = level[c];
  double cs = ldexp(side, -l);
  double lo3[3] = {lo.x, lo.y, lo.z};
  for (int a = 0; a < 3; a++) {
    double k = (double)compact_axis(prefix[c], l, a);
    centre[3 * c + a] = __dadd_rn(lo3[a], __dmul_rn(__dadd_rn(k, 0.5), cs));
  }
}

// one block per cell; radii are maxima of non-negative doubles, so their bit
// patterns order like unsigned integers and the block can combine them with
// an integer max
__global__ void k_radii(const int4* __restrict__ range, const double* __restrict__ centre,
                        const double* __restrict__ nodes_s, const int32_t* __restrict__ tets_s, double* rsrc,
                        double* rtgt) {
  __shared__ unsigned long long s_src, s_tgt;
  int64_t c = blockIdx.x;
  if (threadIdx.x == 0) s_src = s_tgt = 0ull;
  __syncthreads();
  int4 r = range[c];
  double cx = centre[3 * c], cy = centre[3 * c + 1], cz = centre[3 * c + 2];
  double ms = 0, mt = 0;
  for (int64_t q = r.x * 4ll + threadIdx.x; q < r.y * 4ll; q += blockDim.x) {
    int64_t g = tets_s[q];
    ms = fmax(ms, dist_rn(nodes_s[3 * g], nodes_s[3 * g + 1], nodes_s[3 * g + 2], cx, cy, cz));
  }
  for (int64_t i = r.z + threadIdx.x; i < r.w; i += blockDim.x)
    mt = fmax(mt, dist_rn(nodes_s[3 * i], nodes_s[3 * i + 1], nodes_s[3 * i + 2], cx, cy, cz));
  atomicMax(&s_src, (unsigned long long)__double_as_longlong(ms));
  atomicMax(&s_tgt, (unsigned long long)__double_as_longlong(mt));
  __syncthreads();
  if (threadIdx.x == 0) {
    rsrc[c] = __longlong_as_double((long long)s_src);
    rtgt[c] = __longlong_as_double((long long)s_tgt);
  }
}

// ---------------------------------------------------------------------------
// dual tree traversal, one frontier generation per launch
// ---------------------------------------------------------------------------
struct TravCells {
  const int4* range;
  const int32_t* level;
  const int32_t* child0;
  const int32_t* nchild;
  const double* centre;
  const double* rsrc;
  const double* rtgt;
  double theta;
  int dipoles;  // sources are the cells' nodes (point dipoles), not their tets
};

__device__ __forceinline__ void push(uint64_t* buf, unsigned long long* cnt, unsigned long long cap, int32_t a,
                                     int32_t b) {
  unsigned long long k = atomicAdd(cnt, 1ull);
  if (k < cap) buf[k] = ((uint64_t)(uint32_t)a << 32) | (uint32_t)b;
}

__device__ void interact(const TravCells& C, int32_t A, int32_t B, uint64_t* m2l, uint64_t* p2p, uint64_t* nxt,
                         unsigned long long* cnt, unsigned long long cap_m2l, unsigned long long cap_p2p,
                         unsigned long long cap_nxt) {
  int4 ra = C.range[A], rb = C.range[B];
  if (ra.w == ra.z || (C.dipoles ? rb.w == rb.z : rb.y == rb.x)) return;  // no targets / no sources
  double d = dist_rn(C.centre[3 * A], C.centre[3 * A + 1], C.centre[3 * A + 2], C.centre[3 * B], C.centre[3 * B + 1],
                     C.centre[3 * B + 2]);
  if (__dadd_rn(C.rtgt[A], C.rsrc[B]) < __dmul_rn(C.theta, d))
    push(m2l, &cnt[0], cap_m2l, A, B);
  else if (C.nchild[A] == 0 && C.nchild[B] == 0)
    push(p2p, &cnt[1], cap_p2p, A, B);
  else
    push(nxt, &cnt[2], cap_nxt, A, B);
}

__global__ void k_traverse(TravCells C, const uint64_t* __restrict__ cur, int64_t ncur, uint64_t* m2l, uint64_t* p2p,
                           uint64_t* nxt, unsigned long long* cnt, unsigned long long cap_m2l,
                           unsigned long long cap_p2p, unsigned long long cap_nxt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ncur) return;
  int32_t A = (int32_t)(cur[i] >> 32), B = (int32_t)(cur[i] & 0xffffffffu);
  bool leafA = C.nchild[A] == 0, leafB = C.nchild[B] == 0;
  bool split_target = (C.level[A] < C.level[B] && !leafA) || leafB;
  if (split_target) {
    for (int32_t a = C.child0[A]; a < C.child0[A] + C.nchild[A]; a++)
      interact(C, a, B, m2l, p2p, nxt, cnt, cap_m2l, cap_p2p, cap_nxt);
  } else {
    for (int32_t b = C.child0[B]; b < C.child0[B] + C.nchild[B]; b++)
      interact(C, A, b, m2l, p2p, nxt, cnt, cap_m2l, cap_p2p, cap_nxt);
  }
}

__global__ void k_interact_root(TravCells C, uint64_t* m2l, uint64_t* p2p, uint64_t* nxt, unsigned long long* cnt,
                                unsigned long long cap_m2l, unsigned long long cap_p2p, unsigned long long cap_nxt) {
  interact(C, 0, 0, m2l, p2p, nxt, cnt, cap_m2l, cap_p2p, cap_nxt);
}

// CSR offsets by target (high 32 bits of the sorted pair keys)
__global__ void k_csr_offsets(const uint64_t* __restrict__ keys, int64_t n, int64_t ncells, int64_t* off,
                              int32_t* src) {
  int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c <= ncells) {
    uint64_t k = (uint64_t)c << 32;
    int64_t b = 0, e = n;
    while (b < e) {
      int64_t m = (b + e) >> 1;
      if (keys[m] < k)
        b = m + 1;
      else
        e = m;
    }
    off[c] = b;
  }
  if (c < n) src[c] = (int32_t)(keys[c] & 0xffffffffu);
}

// ---------------------------------------------------------------------------
// target leaves, supports, node -> tets
// ---------------------------------------------------------------------------
__global__ void k_node_leaf(const int4* __restrict__ range, const int32_t* __restrict__ nchild, int64_t ncells,
                            int32_t* node_leaf) {
  int64_t c = blockIdx.x;
  if (nchild[c] != 0) return;
  int4 r = range[c];
  for (int32_t i = r.z + threadIdx.x; i < r.w; i += blockDim.x) node_leaf[i] = (int32_t)c;
}

__global__ void k_support_keys(const int4* __restrict__ range, const int32_t* __restrict__ leaves, int64_t nleaves,
                               const int32_t* __restrict__ tets_s, uint64_t* keys, const int64_t* __restrict__ key_off) {
  int64_t li = blockIdx.x;
  if (li >= nleaves) return;
  int32_t c = leaves[li];
  int4 r = range[c];
  int64_t o = key_off[li];
  for (int64_t q = threadIdx.x; q < 4ll * (r.y - r.x); q += blockDim.x)
    keys[o + q] = ((uint64_t)(uint32_t)c << 32) | (uint32_t)tets_s[4ll * r.x + q];
}

__global__ void k_tet_cols(const int4* __restrict__ range, const int32_t* __restrict__ leaves, int64_t nleaves,
                           const int32_t* __restrict__ tets_s, const int64_t* __restrict__ sup_off,
                           const int32_t* __restrict__ sup_node, int32_t* tet_col) {
  int64_t li = blockIdx.x;
  if (li >= nleaves) return;
  int32_t c = leaves[li];
  int4 r = range[c];
  int64_t b0 = sup_off[c], e0 = sup_off[c + 1];
  for (int64_t q = threadIdx.x; q < 4ll * (r.y - r.x); q += blockDim.x) {
    int32_t node = tets_s[4ll * r.x + q];
    int64_t b = b0, e = e0;
    while (b < e) {
      int64_t m = (b + e) >> 1;
      if (sup_node[m] < node)
        b = m + 1;
      else
        e = m;
    }
    tet_col[4ll * r.x + q] = (int32_t)(b - b0);
  }
}

// point-dipole sources: lumped nodal volume V_i = sum_{t ni i} |Omega_t| / 4 (sorted order)
__global__ void k_node_vol_sorted(int64_t nn, const int64_t* __restrict__ nt_off, const int32_t* __restrict__ nt_tet,
                                  const double* __restrict__ vol, double* V) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  double v = 0.0;
  for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) v += vol[nt_tet[e]];
  V[i] = 0.25 * v;
}

// point-dipole moment operator: Ghat[e][m] = V_i y^m / m!, y = r_i - c (one block per source
// leaf, one thread per multi-index m, |m| <= p - 1)
__global__ void k_ghat_dipole(const int32_t* __restrict__ leaves, int64_t nleaves, const double* __restrict__ centre,
                              const double* __restrict__ nodes_s, const double* __restrict__ V,
                              const int64_t* __restrict__ sup_off, const int32_t* __restrict__ sup_node, int pm1,
                              int nc1, double* Ghat) {
  const int64_t li = blockIdx.x;
  if (li >= nleaves || threadIdx.x >= nc1) return;
  const int32_t c = leaves[li];
  int ma, mb, mc;
  mi_decode(threadIdx.x, ma, mb, mc);
  for (int64_t e = sup_off[c]; e < sup_off[c + 1]; e++) {
    const int32_t i = sup_node[e];
    const double y0 = nodes_s[3 * i] - centre[3 * c], y1 = nodes_s[3 * i + 1] - centre[3 * c + 1],
                 y2 = nodes_s[3 * i + 2] - centre[3 * c + 2];
    double g = V[i];
    for (int k = 1; k <= ma; k++) g *= y0 / k;
    for (int k = 1; k <= mb; k++) g *= y1 / k;
    for (int k = 1; k <= mc; k++) g *= y2 / k;
    Ghat[e * nc1 + threadIdx.x] = g;
  }
  (void)pm1;
}

// Vertex-patch sources (the paper's clustering, Sec. 2.1 "vertex interaction"
// and Sec. 3.1-3.2): node i carries lambda_i M_i over every tet around it and
// is binned by its own key.  A cell's source radius reaches the farthest vertex
// of the tets around its nodes ("most remote directly connected vertex").
__global__ void k_radii_patch(const int4* __restrict__ range, const double* __restrict__ centre,
                              const double* __restrict__ nodes_s, const int32_t* __restrict__ tets_s,
                              const int64_t* __restrict__ nt_off, const int32_t* __restrict__ nt_tet, double* rsrc) {
  __shared__ unsigned long long s_src;
  const int64_t c = blockIdx.x;
  if (threadIdx.x == 0) s_src = 0ull;
  __syncthreads();
  const int4 r = range[c];
  const double cx = centre[3 * c], cy = centre[3 * c + 1], cz = centre[3 * c + 2];
  double ms = 0;
  for (int64_t i = r.z + threadIdx.x; i < r.w; i += blockDim.x)
    for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++)
      for (int k = 0; k < 4; k++) {
        const int64_t g = tets_s[4ll * nt_tet[e] + k];
        ms = fmax(ms, dist_rn(nodes_s[3 * g], nodes_s[3 * g + 1], nodes_s[3 * g + 2], cx, cy, cz));
      }
  atomicMax(&s_src, (unsigned long long)__double_as_longlong(ms));
  __syncthreads();
  if (threadIdx.x == 0) rsrc[c] = __longlong_as_double((long long)s_src);
}

// Exact moment operator of vertex patches: for every own node i of a source
// leaf and |m| <= p-1,
//   Ghat[i][m] = sum_{t ni i} int_t lambda_i(r') y^m/m! dV,  y = r' - c_leaf,
// with the Grundmann-Moeller rule of k_ghat.  One block per leaf, one thread
// per multi-index m; supports are the leaf's own nodes in order.
__global__ void k_ghat_patch(const int4* __restrict__ range, const int32_t* __restrict__ leaves, int64_t nleaves,
                             const double* __restrict__ centre, const double* __restrict__ nodes_s,
                             const int32_t* __restrict__ tets_s, const double* __restrict__ tet_vol,
                             const int64_t* __restrict__ nt_off, const int32_t* __restrict__ nt_tet,
                             const int64_t* __restrict__ sup_off, const double* __restrict__ gm, int ngm, int pm1,
                             int nc1, double* Ghat) {
  __shared__ double px[MAX_P + 1], py[MAX_P + 1], pz[MAX_P + 1];
  __shared__ double lam_w[5];
  const int64_t li = blockIdx.x;
  if (li >= nleaves) return;
  const int32_t c = leaves[li];
  const int4 r = range[c];
  const double cx = centre[3 * c], cy = centre[3 * c + 1], cz = centre[3 * c + 2];
  const bool active = threadIdx.x < nc1;
  int ma = 0, mb = 0, mc = 0;
  if (active) mi_decode(threadIdx.x, ma, mb, mc);
  for (int32_t i = r.z; i < r.w; i++) {
    double gsum = 0.0;
    for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) {
      const int32_t j = nt_tet[e];
      double v[4][3];
      int ki = 0;
      for (int k = 0; k < 4; k++) {
        const int64_t g = tets_s[4ll * j + k];
        if (g == i) ki = k;
        v[k][0] = nodes_s[3 * g];
        v[k][1] = nodes_s[3 * g + 1];
        v[k][2] = nodes_s[3 * g + 2];
      }
      double acc = 0.0;
      for (int q = 0; q < ngm; q++) {
        __syncthreads();
        if (threadIdx.x == 0) {
          const double l0 = gm[5 * q], l1 = gm[5 * q + 1], l2 = gm[5 * q + 2], l3 = gm[5 * q + 3];
          double y[3];
          for (int a = 0; a < 3; a++) y[a] = l0 * v[0][a] + l1 * v[1][a] + l2 * v[2][a] + l3 * v[3][a];
          y[0] -= cx;
          y[1] -= cy;
          y[2] -= cz;
          px[0] = py[0] = pz[0] = 1.0;
          for (int d = 1; d <= pm1; d++) {
            px[d] = px[d - 1] * y[0] / d;
            py[d] = py[d - 1] * y[1] / d;
            pz[d] = pz[d - 1] * y[2] / d;
          }
          for (int k = 0; k < 5; k++) lam_w[k] = gm[5 * q + k];
        }
        __syncthreads();
        if (active) acc += lam_w[ki] * lam_w[4] * px[ma] * py[mb] * pz[mc];
      }
      gsum += tet_vol[j] * acc;
    }
    if (active) Ghat[(sup_off[c] + (i - r.z)) * nc1 + threadIdx.x] = gsum;
  }
}

// Exact moment operator of a source leaf (Sec. 2.2, Eq. expCoeffs): for every
// support node j of the leaf and |m| <= p-1,
//   Ghat[j][m] = sum_{t in leaf, t ni j} int_t lambda_{k(t,j)}(r') y^m/m! dV,  y = r' - c_leaf,
// integrated with the Grundmann-Moeller rule of degree 2s+1 >= p, exact for
// these degree-(|m|+1) polynomials.  Then at every evaluation
//   Qhat_n = Q_n/n! = sum_j sum_c Ghat[j][n - e_c] M_c(j).
// One block per leaf, one thread per multi-index m.
__global__ void k_ghat(const int4* __restrict__ range, const int32_t* __restrict__ leaves, int64_t nleaves,
                       const double* __restrict__ centre, const double* __restrict__ nodes_s,
                       const int32_t* __restrict__ tets_s, const double* __restrict__ tet_vol,
                       const int64_t* __restrict__ sup_off, const int32_t* __restrict__ tet_col,
                       const double* __restrict__ gm, int ngm, int pm1, int nc1, double* Ghat) {
  __shared__ double px[MAX_P + 1], py[MAX_P + 1], pz[MAX_P + 1];
  __shared__ double lam_w[5];
  int64_t li = blockIdx.x;
  if (li >= nleaves) return;
  int32_t c = leaves[li];
  int4 r = range[c];
  double cx = centre[3 * c], cy = centre[3 * c + 1], cz = centre[3 * c + 2];
  int64_t so = sup_off[c];
  int ma = 0, mb = 0, mc = 0;
  bool active = threadIdx.x < nc1;
  if (active) mi_decode(threadIdx.x, ma, mb, mc);
  for (int32_t j = r.x; j < r.y; j++) {
    double v[4][3];
    for (int k = 0; k < 4; k++) {
      int64_t g = tets_s[4ll * j + k];
      v[k][0] = nodes_s[3 * g];
      v[k][1] = nodes_s[3 * g + 1];
      v[k][2] = nodes_s[3 * g + 2];
    }
    double vol = tet_vol[j];
    double acc[4] = {0, 0, 0, 0};
    for (int q = 0; q < ngm; q++) {
      __syncthreads();
      if (threadIdx.x == 0) {
        double l0 = gm[5 * q], l1 = gm[5 * q + 1], l2 = gm[5 * q + 2], l3 = gm[5 * q + 3];
        double y[3];
        for (int a = 0; a < 3; a++) y[a] = l0 * v[0][a] + l1 * v[1][a] + l2 * v[2][a] + l3 * v[3][a];
        y[0] -= cx;
        y[1] -= cy;
        y[2] -= cz;
        px[0] = py[0] = pz[0] = 1.0;
        for (int e = 1; e <= pm1; e++) {
          px[e] = px[e - 1] * y[0] / e;
          py[e] = py[e - 1] * y[1] / e;
          pz[e] = pz[e - 1] * y[2] / e;
        }
        for (int k = 0; k < 5; k++) lam_w[k] = gm[5 * q + k];
      }
      __syncthreads();
      if (active) {
        double s = lam_w[4] * px[ma] * py[mb] * pz[mc];
        for (int k = 0; k < 4; k++) acc[k] += lam_w[k] * s;
      }
    }
    if (active)
      for (int k = 0; k < 4; k++) {
        int64_t row = so + tet_col[4ll * j + k];
        Ghat[row * nc1 + threadIdx.x] += vol * acc[k];
      }
  }
}

// Grundmann-Moeller rule on the tetrahedron, degree d = 2s+1 (Grundmann &
// Moeller, SIAM J. Numer. Anal. 15, 1978).  Output rows (l0,l1,l2,l3,w) with
// barycentric points and weights normalised to sum 1 (fractions of the
// volume).  The rule is checked here against the closed form
//   avg over the tet of l^alpha = 3! alpha! / (|alpha|+3)!
// for every |alpha| <= d before it is used.
static std::vector<double> gm_rule(int s) {
  const int n = 3, d = 2 * s + 1;
  auto fact = [](int k) {
    double f = 1;
    for (int i = 2; i <= k; i++) f *= i;
    return f;
  };
  std::vector<double> out;
  for (int i = 0; i <= s; i++) {
    double w = ((i & 1) ? -1.0 : 1.0) * std::ldexp(1.0, -2 * s) * std::pow((double)(d + n - 2 * i), d) /
               (fact(i) * fact(d + n - i)) * 6.0;
    int m = s - i;
    for (int b0 = 0; b0 <= m; b0++)
      for (int b1 = 0; b0 + b1 <= m; b1++)
        for (int b2 = 0; b0 + b1 + b2 <= m; b2++) {
          int b3 = m - b0 - b1 - b2;
          double den = (double)(d + n - 2 * i);
          out.push_back((2 * b0 + 1) / den);
          out.push_back((2 * b1 + 1) / den);
          out.push_back((2 * b2 + 1) / den);
          out.push_back((2 * b3 + 1) / den);
          out.push_back(w);
        }
  }
  size_t np = out.size() / 5;
  double worst = 0;
  for (int a0 = 0; a0 <= d; a0++)
    for (int a1 = 0; a0 + a1 <= d; a1++)
      for (int a2 = 0; a0 + a1 + a2 <= d; a2++)
        for (int a3 = 0; a0 + a1 + a2 + a3 <= d; a3++) {
          double q = 0;
          for (size_t k = 0; k < np; k++)
            q += out[5 * k + 4] * std::pow(out[5 * k], a0) * std::pow(out[5 * k + 1], a1) *
                 std::pow(out[5 * k + 2], a2) * std::pow(out[5 * k + 3], a3);
          double ex = 6.0 * fact(a0) * fact(a1) * fact(a2) * fact(a3) / fact(a0 + a1 + a2 + a3 + 3);
          worst = std::max(worst, std::fabs(q - ex));
        }
  if (worst > 1e-12) fail(DEMAG_ERR_UNSUPPORTED, "Grundmann-Moeller rule failed its exactness check");
  return out;
}

// ---------------------------------------------------------------------------
// plan build driver
// ---------------------------------------------------------------------------
void build_plan(Plan& P, const double* nodes_in, const int32_t* tets_in) {
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = P.stream;
  const int64_t nn = P.nn, nt = P.nt;
  CubTemp ct;

  // inputs on the device (the caller may pass host or device pointers)
  Tmp<double> nodes(3 * nn);
  Tmp<int32_t> tets(4 * nt);
  DM_CUDA(cudaMemcpyAsync(nodes.p, nodes_in, sizeof(double) * 3 * nn, cudaMemcpyDefault, s));
  DM_CUDA(cudaMemcpyAsync(tets.p, tets_in, sizeof(int32_t) * 4 * nt, cudaMemcpyDefault, s));

  // validation
  {
    Tmp<int> flags(2);
    DM_CUDA(cudaMemsetAsync(flags.p, 0, 2 * sizeof(int), s));
    k_validate<<<nblk(nt, 256), 256, 0, s>>>(nodes.p, nn, tets.p, nt, flags.p);
    DM_LAUNCH("k_validate");
    int h[2];
    DM_CUDA(cudaMemcpyAsync(h, flags.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    if (h[0]) fail(DEMAG_ERR_INVALID_ARG, "tet node index out of range");
    if (h[1]) fail(DEMAG_ERR_DEGENERATE_TET, "degenerate tetrahedron (|vol| < 1e-14 * longest edge^3)");
  }

  // bounding cube (Sec. 3.1)
  {
    int nb = (int)std::min<int64_t>(256, (nn + 255) / 256);
    Tmp<double> part(6 * nb);
    k_bbox_partial<<<nb, 256, 0, s>>>(nodes.p, nn, part.p);
    DM_LAUNCH("k_bbox_partial");
    std::vector<double> h(6 * nb);
    DM_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * 6 * nb, cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; b++)
      for (int a = 0; a < 3; a++) {
        lo[a] = std::min(lo[a], h[6 * b + a]);
        hi[a] = std::max(hi[a], h[6 * b + 3 + a]);
      }
    double ext = 0;
    for (int a = 0; a < 3; a++) {
      volatile double e = hi[a] - lo[a];
      ext = std::max(ext, (double)e);
      P.lo[a] = lo[a];
    }
    if (!(ext > 0) || !std::isfinite(ext)) fail(DEMAG_ERR_INVALID_ARG, "mesh has zero or non-finite extent");
    volatile double side = ext * (1.0 + 1.0 / 1048576.0);
    P.side = side;
    volatile double scale = 2097152.0 / P.side;
    P.scale = scale;
  }
  double3 lo3 = make_double3(P.lo[0], P.lo[1], P.lo[2]);

  // keys and sort (stable radix sort: ties keep ascending original index)
  P.node_key = dalloc<uint64_t>(P, nn);
  P.tet_key = dalloc<uint64_t>(P, nt);
  P.node_perm = dalloc<int32_t>(P, nn);
  P.tet_perm = dalloc<int32_t>(P, nt);
  Tmp<uint64_t> nkey_s(nn), tkey_s(nt);
  {
    Tmp<int32_t> idx(std::max(nn, nt));
    k_node_keys<<<nblk(nn, 256), 256, 0, s>>>(nodes.p, nn, lo3, P.scale, P.node_key, idx.p);
    DM_LAUNCH("k_node_keys");
    size_t b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, b, P.node_key, nkey_s.p, idx.p, P.node_perm, (int)nn, 0, 63, s);
    ct.need(b);
    DM_CUDA(cub::DeviceRadixSort::SortPairs(ct.p, b, P.node_key, nkey_s.p, idx.p, P.node_perm, (int)nn, 0, 63, s));
    k_tet_keys<<<nblk(nt, 256), 256, 0, s>>>(nodes.p, tets.p, nt, lo3, P.scale, P.tet_key, idx.p);
    DM_LAUNCH("k_tet_keys");
    b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, b, P.tet_key, tkey_s.p, idx.p, P.tet_perm, (int)nt, 0, 63, s);
    ct.need(b);
    DM_CUDA(cub::DeviceRadixSort::SortPairs(ct.p, b, P.tet_key, tkey_s.p, idx.p, P.tet_perm, (int)nt, 0, 63, s));
  }
  P.nodes_s = dalloc<double>(P, 3 * nn);
  P.tets_s = dalloc<int32_t>(P, 4 * nt);
  {
    Tmp<int32_t> rank(nn);
    k_apply_node_perm<<<nblk(nn, 256), 256, 0, s>>>(nodes.p, P.node_perm, nn, P.nodes_s, rank.p);
    DM_LAUNCH("k_apply_node_perm");
    k_apply_tet_perm<<<nblk(nt, 256), 256, 0, s>>>(tets.p, P.tet_perm, rank.p, nt, P.tets_s);
    DM_LAUNCH("k_apply_tet_perm");
  }
  nodes.release();
  tets.release();

  // octree, level by level (Sec. 3.1)
  {
    size_t cap = 1024;
    Tmp<uint64_t> prefix(cap);
    Tmp<int32_t> clevel(cap), parent(cap), child0(cap), nchild(cap);
    Tmp<int4> range(cap);
    auto grow = [&](size_t need) {
      if (need <= cap) return;
      size_t nc = std::max(need, 2 * cap);
      auto regrow = [&](auto& t, size_t elem) {
        using T = std::remove_reference_t<decltype(*t.p)>;
        T* q = nullptr;
        if (cudaMalloc(&q, nc * sizeof(T)) != cudaSuccess) {
          cudaGetLastError();
          fail(DEMAG_ERR_OUT_OF_MEMORY, "octree allocation failed");
        }
        DM_CUDA(cudaMemcpyAsync(q, t.p, elem * sizeof(T), cudaMemcpyDeviceToDevice, s));
        DM_CUDA(cudaStreamSynchronize(s));
        cudaFree(t.p);
        t.p = q;
        t.n = nc;
      };
      regrow(prefix, cap);
      regrow(clevel, cap);
      regrow(parent, cap);
      regrow(child0, cap);
      regrow(nchild, cap);
      regrow(range, cap);
      cap = nc;
    };
    // root
    uint64_t z64 = 0;
    int32_t z32 = 0, m1 = -1;
    int4 r0 = make_int4(0, (int)nt, 0, (int)nn);
    DM_CUDA(cudaMemcpyAsync(prefix.p, &z64, sizeof(z64), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(clevel.p, &z32, sizeof(z32), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(parent.p, &m1, sizeof(m1), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaMemcpyAsync(range.p, &r0, sizeof(r0), cudaMemcpyHostToDevice, s));
    P.level_start.assign(1, 0);
    int64_t lb = 0, le = 1;
    int level = 0;
    while (lb < le) {
      int64_t n = le - lb;
      Tmp<int4> cb(8 * n);
      Tmp<int32_t> excl(n + 1);
      k_count_children<<<nblk(n, 128), 128, 0, s>>>(range.p, lb, le, level, P.opt.leaf_size, tkey_s.p, nkey_s.p,
                                                     nchild.p, cb.p);
      DM_LAUNCH("k_count_children");
      size_t b = 0;
      cub::DeviceScan::ExclusiveSum(nullptr, b, nchild.p + lb, excl.p, (int)n, s);
      ct.need(b);
      DM_CUDA(cub::DeviceScan::ExclusiveSum(ct.p, b, nchild.p + lb, excl.p, (int)n, s));
      int32_t last_ex = 0, last_n = 0;
      DM_CUDA(cudaMemcpyAsync(&last_ex, excl.p + (n - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaMemcpyAsync(&last_n, nchild.p + (le - 1), sizeof(int32_t), cudaMemcpyDeviceToHost, s));
      DM_CUDA(cudaStreamSynchronize(s));
      int64_t nnew = (int64_t)last_ex + last_n;
      grow(le + nnew);
      k_write_children<<<nblk(n, 128), 128, 0, s>>>(lb, le, level, nchild.p, excl.p, cb.p, prefix.p, clevel.p,
                                                     range.p, parent.p, child0.p);
      DM_LAUNCH("k_write_children");
      P.level_start.push_back(le);
      lb = le;
      le = le + nnew;
      level++;
    }
    P.nlevels = level;
    P.ncells = le;
    int64_t nc = le;
    P.cell_prefix = dalloc<uint64_t>(P, nc);
    P.cell_level = dalloc<int32_t>(P, nc);
    P.cell_range = dalloc<int4>(P, nc);
    P.cell_parent = dalloc<int32_t>(P, nc);
    P.cell_child0 = dalloc<int32_t>(P, nc);
    P.cell_nchild = dalloc<int32_t>(P, nc);
    DM_CUDA(cudaMemcpyAsync(P.cell_prefix, prefix.p, nc * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.cell_level, clevel.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.cell_range, range.p, nc * sizeof(int4), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.cell_parent, parent.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.cell_child0, child0.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaMemcpyAsync(P.cell_nchild, nchild.p, nc * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }
  const int64_t nc = P.ncells;

  // orientation, per-tet geometry for the near field and for H (p2p.cu)
  build_tet_geometry(P);

  // node -> incident tets (sorted by tet within a node): the lumped H, the vertex patches
  {
    Tmp<int32_t> key(4 * nt), val(4 * nt), key_s(4 * nt);
    P.nt_off = dalloc<int64_t>(P, nn + 1);
    P.nt_tet = dalloc<int32_t>(P, 4 * nt);
    // keys = node ids in tets_s order; values = tet ids
    DM_CUDA(cudaMemcpyAsync(key.p, P.tets_s, 4 * nt * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    std::vector<int32_t> hv(4 * nt);
    for (int64_t q = 0; q < 4 * nt; q++) hv[q] = (int32_t)(q / 4);
    DM_CUDA(cudaMemcpyAsync(val.p, hv.data(), 4 * nt * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    size_t b = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, b, key.p, key_s.p, val.p, P.nt_tet, (int)(4 * nt), 0, 32, s);
    ct.need(b);
    DM_CUDA(cub::DeviceRadixSort::SortPairs(ct.p, b, key.p, key_s.p, val.p, P.nt_tet, (int)(4 * nt), 0, 32, s));
    std::vector<int32_t> hk(4 * nt);
    DM_CUDA(cudaMemcpyAsync(hk.data(), key_s.p, 4 * nt * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> off(nn + 1, 0);
    for (int64_t q = 0; q < 4 * nt; q++) off[hk[q] + 1]++;
    for (int64_t i = 0; i < nn; i++) off[i + 1] += off[i];
    DM_CUDA(cudaMemcpyAsync(P.nt_off, off.data(), (nn + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }

  // centres and radii (Sec. 3.2)
  P.cell_centre = dalloc<double>(P, 3 * nc);
  P.cell_rsrc = dalloc<double>(P, nc);
  P.cell_rtgt = dalloc<double>(P, nc);
  k_centres<<<nblk(nc, 128), 128, 0, s>>>(nc, P.cell_prefix, P.cell_level, lo3, P.side, P.cell_centre);
  DM_LAUNCH("k_centres");
  k_radii<<<(int)nc, 256, 0, s>>>(P.cell_range, P.cell_centre, P.nodes_s, P.tets_s, P.cell_rsrc, P.cell_rtgt);
  DM_LAUNCH("k_radii");
  const bool dip = P.opt.sources == DEMAG_SOURCES_DIPOLES, patch = P.opt.sources == DEMAG_SOURCES_PATCHES;
  const bool nodesrc = dip || patch;  // sources bound to the cells' own nodes
  if (dip)  // point dipoles at the cell's own nodes: the source radius is the node radius
    DM_CUDA(cudaMemcpyAsync(P.cell_rsrc, P.cell_rtgt, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  if (patch) {
    k_radii_patch<<<(int)nc, 256, 0, s>>>(P.cell_range, P.cell_centre, P.nodes_s, P.tets_s, P.nt_off, P.nt_tet,
                                          P.cell_rsrc);
    DM_LAUNCH("k_radii_patch");
  }

  // dual tree traversal (Sec. 3.3, Listings 1-2), breadth first
  {
    TravCells C{P.cell_range, P.cell_level, P.cell_child0, P.cell_nchild,
                P.cell_centre, P.cell_rsrc, P.cell_rtgt, P.opt.theta, nodesrc ? 1 : 0};
    size_t cap_m = std::max<int64_t>(1024, 64 * nc), cap_p = std::max<int64_t>(1024, 32 * nc),
           cap_f = std::max<int64_t>(1024, 16 * nc);
    Tmp<uint64_t> m2l(cap_m), p2p(cap_p), cur(cap_f), nxt(cap_f);
    Tmp<unsigned long long> cnt(3);
    unsigned long long h[3] = {0, 0, 0};
    DM_CUDA(cudaMemcpyAsync(cnt.p, h, sizeof(h), cudaMemcpyHostToDevice, s));
    k_interact_root<<<1, 1, 0, s>>>(C, m2l.p, p2p.p, cur.p, cnt.p, cap_m, cap_p, cap_f);
    DM_LAUNCH("k_interact_root");
    DM_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    int64_t ncur = (int64_t)h[2];
    size_t cap_cur = cap_f, cap_nxt = cap_f;
    // grow t to hold `need` entries, keeping its first `keep` entries
    auto regrow = [&](Tmp<uint64_t>& t, size_t& cap, size_t need, size_t keep) {
      size_t ncap = std::max(need + need / 2, 2 * cap);
      uint64_t* q = nullptr;
      if (cudaMalloc(&q, ncap * sizeof(uint64_t)) != cudaSuccess) {
        cudaGetLastError();
        fail(DEMAG_ERR_OUT_OF_MEMORY, "interaction list allocation failed");
      }
      if (keep) DM_CUDA(cudaMemcpyAsync(q, t.p, keep * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
      DM_CUDA(cudaStreamSynchronize(s));
      cudaFree(t.p);
      t.p = q;
      t.n = ncap;
      cap = ncap;
    };
    for (int iter = 0; ncur > 0; iter++) {
      if (iter > 4 * (MAX_LEVEL + 2)) fail(DEMAG_ERR_UNSUPPORTED, "dual tree traversal did not terminate");
      unsigned long long before[3] = {h[0], h[1], 0};
      for (;;) {  // one generation; re-run with larger buffers if one overflowed
        DM_CUDA(cudaMemcpyAsync(cnt.p, before, sizeof(before), cudaMemcpyHostToDevice, s));
        k_traverse<<<nblk(ncur, 128), 128, 0, s>>>(C, cur.p, ncur, m2l.p, p2p.p, nxt.p, cnt.p, cap_m, cap_p,
                                                    cap_nxt);
        DM_LAUNCH("k_traverse");
        DM_CUDA(cudaMemcpyAsync(h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        DM_CUDA(cudaStreamSynchronize(s));
        bool again = false;
        if (h[0] > cap_m) { regrow(m2l, cap_m, h[0], before[0]); again = true; }
        if (h[1] > cap_p) { regrow(p2p, cap_p, h[1], before[1]); again = true; }
        if (h[2] > cap_nxt) { regrow(nxt, cap_nxt, h[2], 0); again = true; }
        if (!again) break;
      }
      std::swap(cur.p, nxt.p);
      std::swap(cur.n, nxt.n);
      std::swap(cap_cur, cap_nxt);
      ncur = (int64_t)h[2];
    }
    P.n_m2l = (int64_t)h[0];
    P.n_p2p = (int64_t)h[1];
    // canonical order: sort by (target, source)
    Tmp<uint64_t> sorted(std::max(P.n_m2l, P.n_p2p));
    P.m2l_off = dalloc<int64_t>(P, nc + 1);
    P.m2l_src = dalloc<int32_t>(P, std::max<int64_t>(P.n_m2l, 1));
    P.p2p_off = dalloc<int64_t>(P, nc + 1);
    P.p2p_src = dalloc<int32_t>(P, std::max<int64_t>(P.n_p2p, 1));
    for (int which = 0; which < 2; which++) {
      uint64_t* in = which == 0 ? m2l.p : p2p.p;
      int64_t n = which == 0 ? P.n_m2l : P.n_p2p;
      int64_t* off = which == 0 ? P.m2l_off : P.p2p_off;
      int32_t* src = which == 0 ? P.m2l_src : P.p2p_src;
      if (n > 0) {
        size_t b = 0;
        cub::DeviceRadixSort::SortKeys(nullptr, b, in, sorted.p, (int)n, 0, 64, s);
        ct.need(b);
        DM_CUDA(cub::DeviceRadixSort::SortKeys(ct.p, b, in, sorted.p, (int)n, 0, 64, s));
      }
      k_csr_offsets<<<nblk(std::max<int64_t>(nc + 1, n), 256), 256, 0, s>>>(sorted.p, n, nc, off, src);
      DM_LAUNCH("k_csr_offsets");
    }
  }

  // host copies of the shapes
  std::vector<int32_t> h_nchild(nc);
  std::vector<int4> h_range(nc);
  std::vector<int64_t> h_m2l_off(nc + 1), h_p2p_off(nc + 1);
  std::vector<int32_t> h_p2p_src(std::max<int64_t>(P.n_p2p, 1));
  DM_CUDA(cudaMemcpyAsync(h_nchild.data(), P.cell_nchild, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(h_range.data(), P.cell_range, nc * sizeof(int4), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(h_m2l_off.data(), P.m2l_off, (nc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaMemcpyAsync(h_p2p_off.data(), P.p2p_off, (nc + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  if (P.n_p2p)
    DM_CUDA(cudaMemcpyAsync(h_p2p_src.data(), P.p2p_src, P.n_p2p * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  DM_CUDA(cudaStreamSynchronize(s));
  P.nleaves = 0;
  P.h_m2l_targets.clear();
  P.h_p2p_targets.clear();
  P.h_src_leaves.clear();
  P.n_p2p_pairs = 0;
  for (int64_t c = 0; c < nc; c++) {
    bool leaf = h_nchild[c] == 0;
    P.nleaves += leaf;
    if (h_m2l_off[c + 1] > h_m2l_off[c]) P.h_m2l_targets.push_back((int32_t)c);
    if (h_p2p_off[c + 1] > h_p2p_off[c]) {
      P.h_p2p_targets.push_back((int32_t)c);
      int64_t ntg = h_range[c].w - h_range[c].z, nsrc = 0;
      for (int64_t e = h_p2p_off[c]; e < h_p2p_off[c + 1]; e++) {
        int4 r = h_range[h_p2p_src[e]];
        nsrc += nodesrc ? r.w - r.z : r.y - r.x;
      }
      P.n_p2p_pairs += ntg * nsrc;
    }
    if (leaf && (nodesrc ? h_range[c].w > h_range[c].z : h_range[c].y > h_range[c].x))
      P.h_src_leaves.push_back((int32_t)c);
  }
  // leaves holding nodes, for the leaf-wise L2P
  {
    std::vector<int32_t> nl;
    for (int64_t c = 0; c < nc; c++)
      if (h_nchild[c] == 0 && h_range[c].w > h_range[c].z) nl.push_back((int32_t)c);
    P.n_node_leaves = (int64_t)nl.size();
    P.node_leaves = dalloc<int32_t>(P, std::max<size_t>(nl.size(), 1));
    DM_CUDA(cudaMemcpyAsync(P.node_leaves, nl.data(), nl.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaStreamSynchronize(s));
  }

  P.m2l_targets = dalloc<int32_t>(P, std::max<size_t>(P.h_m2l_targets.size(), 1));
  P.p2p_targets = dalloc<int32_t>(P, std::max<size_t>(P.h_p2p_targets.size(), 1));
  DM_CUDA(cudaMemcpyAsync(P.m2l_targets, P.h_m2l_targets.data(), P.h_m2l_targets.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));
  DM_CUDA(cudaMemcpyAsync(P.p2p_targets, P.h_p2p_targets.data(), P.h_p2p_targets.size() * sizeof(int32_t),
                          cudaMemcpyHostToDevice, s));

  // node -> leaf
  P.node_leaf = dalloc<int32_t>(P, nn);
  k_node_leaf<<<(int)nc, 128, 0, s>>>(P.cell_range, P.cell_nchild, nc, P.node_leaf);
  DM_LAUNCH("k_node_leaf");

  // source-leaf supports: unique nodes of each leaf's tets
  int64_t nsl = (int64_t)P.h_src_leaves.size();
  P.src_leaves = dalloc<int32_t>(P, std::max<int64_t>(nsl, 1));
  DM_CUDA(cudaMemcpyAsync(P.src_leaves, P.h_src_leaves.data(), nsl * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  P.sup_off = dalloc<int64_t>(P, nc + 1);
  P.tet_col = dalloc<int32_t>(P, 4 * nt);
  if (nodesrc) {  // a dipole or patch leaf's support is its own nodes (sorted ids r.z .. r.w - 1)
    std::vector<int64_t> so(nc + 1, 0);
    std::vector<int32_t> sn;
    std::vector<char> is_src(nc, 0);
    for (int32_t c : P.h_src_leaves) is_src[c] = 1;
    for (int64_t c = 0; c < nc; c++) {
      if (is_src[c])
        for (int32_t i = h_range[c].z; i < h_range[c].w; i++) sn.push_back(i);
      so[c + 1] = (int64_t)sn.size();
    }
    P.n_sup = (int64_t)sn.size();
    P.sup_node = dalloc<int32_t>(P, std::max<int64_t>(P.n_sup, 1));
    DM_CUDA(cudaMemcpyAsync(P.sup_off, so.data(), (nc + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (P.n_sup)
      DM_CUDA(cudaMemcpyAsync(P.sup_node, sn.data(), sn.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    DM_CUDA(cudaStreamSynchronize(s));
  } else {
    std::vector<int64_t> koff(nsl + 1, 0);
    for (int64_t i = 0; i < nsl; i++) {
      int4 r = h_range[P.h_src_leaves[i]];
      koff[i + 1] = koff[i] + 4ll * (r.y - r.x);
    }
    int64_t nk = koff[nsl];
    Tmp<int64_t> dkoff(nsl + 1);
    DM_CUDA(cudaMemcpyAsync(dkoff.p, koff.data(), (nsl + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    Tmp<uint64_t> keys(nk), keys_s(nk), uniq(nk);
    Tmp<int> nuniq(1);
    k_support_keys<<<(int)std::max<int64_t>(nsl, 1), 128, 0, s>>>(P.cell_range, P.src_leaves, nsl, P.tets_s, keys.p,
                                                                    dkoff.p);
    DM_LAUNCH("k_support_keys");
    size_t b = 0;
    cub::DeviceRadixSort::SortKeys(nullptr, b, keys.p, keys_s.p, (int)nk, 0, 64, s);
    ct.need(b);
    DM_CUDA(cub::DeviceRadixSort::SortKeys(ct.p, b, keys.p, keys_s.p, (int)nk, 0, 64, s));
    b = 0;
    cub::DeviceSelect::Unique(nullptr, b, keys_s.p, uniq.p, nuniq.p, (int)nk, s);
    ct.need(b);
    DM_CUDA(cub::DeviceSelect::Unique(ct.p, b, keys_s.p, uniq.p, nuniq.p, (int)nk, s));
    int hn = 0;
    DM_CUDA(cudaMemcpyAsync(&hn, nuniq.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    DM_CUDA(cudaStreamSynchronize(s));
    P.n_sup = hn;
    P.sup_node = dalloc<int32_t>(P, std::max<int64_t>(hn, 1));
    k_csr_offsets<<<nblk(std::max<int64_t>(nc + 1, hn), 256), 256, 0, s>>>(uniq.p, hn, nc, P.sup_off, P.sup_node);
    DM_LAUNCH("k_csr_offsets(sup)");
    k_tet_cols<<<(int)std::max<int64_t>(nsl, 1), 128, 0, s>>>(P.cell_range, P.src_leaves, nsl, P.tets_s, P.sup_off,
                                                                P.sup_node, P.tet_col);
    DM_LAUNCH("k_tet_cols");
  }

  // exact-moment operators of the source leaves (Sec. 2.2); dipoles after the node volumes below
  if (!dip) {
    int pm1 = P.p - 1;
    P.nc1 = ncoef_of(pm1);
    int sgm = (P.p - 1 + 1) / 2;  // degree 2s+1 >= p
    std::vector<double> gm = gm_rule(sgm);
    int ngm = (int)(gm.size() / 5);
    Tmp<double> dgm(gm.size());
    DM_CUDA(cudaMemcpyAsync(dgm.p, gm.data(), gm.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    P.Ghat = dalloc<double>(P, std::max<int64_t>(P.n_sup, 1) * P.nc1);
    DM_CUDA(cudaMemsetAsync(P.Ghat, 0, std::max<int64_t>(P.n_sup, 1) * P.nc1 * sizeof(double), s));
    int threads = ((P.nc1 + 31) / 32) * 32;
    if (patch) {
      k_ghat_patch<<<(int)std::max<int64_t>(nsl, 1), threads, 0, s>>>(
          P.cell_range, P.src_leaves, nsl, P.cell_centre, P.nodes_s, P.tets_s, P.tet_vol, P.nt_off, P.nt_tet,
          P.sup_off, dgm.p, ngm, pm1, P.nc1, P.Ghat);
      DM_LAUNCH("k_ghat_patch");
    } else {
      k_ghat<<<(int)std::max<int64_t>(nsl, 1), threads, 0, s>>>(P.cell_range, P.src_leaves, nsl, P.cell_centre,
                                                                  P.nodes_s, P.tets_s, P.tet_vol, P.sup_off,
                                                                  P.tet_col, dgm.p, ngm, pm1, P.nc1, P.Ghat);
      DM_LAUNCH("k_ghat");
    }
    DM_CUDA(cudaStreamSynchronize(s));
  }

  // point dipoles: lumped nodal volumes (sorted order), then the moment operator
  // Ghat[e][m] = V_i y_i^m / m! at the support node i = sup_node[e], y_i = r_i - c_leaf
  if (dip) {
    P.node_vol_s = dalloc<double>(P, nn);
    k_node_vol_sorted<<<nblk(nn, 256), 256, 0, s>>>(nn, P.nt_off, P.nt_tet, P.tet_vol, P.node_vol_s);
    DM_LAUNCH("k_node_vol_sorted");
    P.nc1 = ncoef_of(P.p - 1);
    P.Ghat = dalloc<double>(P, std::max<int64_t>(P.n_sup, 1) * P.nc1);
    const int threads = ((P.nc1 + 31) / 32) * 32;
    k_ghat_dipole<<<(int)std::max<int64_t>(nsl, 1), threads, 0, s>>>(P.src_leaves, nsl, P.cell_centre, P.nodes_s,
                                                                      P.node_vol_s, P.sup_off, P.sup_node, P.p - 1,
                                                                      P.nc1, P.Ghat);
    DM_LAUNCH("k_ghat_dipole");
    DM_CUDA(cudaStreamSynchronize(s));
  }

  P.h_range = std::move(h_range);
  P.h_p2p_off = std::move(h_p2p_off);
  P.h_p2p_src = std::move(h_p2p_src);
  if (P.opt.near_mode == 1) build_near_field(P);
  if (P.opt.precision != DEMAG_FP64) build_mixed_operators(P);
  if (P.opt.precision != DEMAG_FP64 && P.opt.near_mode == 1) {
    // the mixed path with stored near-field coefficients evaluates from FP32
    // copies only: the FP64 per-tet geometry and P2M operator go
    DM_CUDA(cudaStreamSynchronize(P.stream));
    dfree(P, P.tet_geo);
    dfree(P, P.tet_grad);
    dfree(P, P.Ghat);
    P.tet_geo = P.tet_grad = P.Ghat = nullptr;
  }
  audit_plan(P);
  DM_CUDA(cudaStreamSynchronize(s));
  P.plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace demag
