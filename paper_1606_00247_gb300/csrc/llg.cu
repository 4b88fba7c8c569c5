// llg.cu -- magnetostatic energy and Landau-Lifshitz-Gilbert stepping on top of
// demag_eval: the states of successive integrator stages go straight into one
// batched evaluation per stage.
//
//   energy:  e_b = -(1/2) sum_i V_i M_{b,i} . H_{b,i}   (E = mu0 e; V_i the lumped nodal
//            volume sum_{t ni i} |Omega_t| / 4, the mass lumping of the H computation, Sec. 4.1)
//   LLG:     dm/dt = -1/(1 + alpha^2) [ m x h + alpha m x (m x h) ],
//            h = H_demag(Ms m) / Ms + h_ext, time in units of 1/(gamma mu0 Ms)
#include <algorithm>

#include "common.cuh"

namespace demag {

namespace {

inline int nblk(int64_t n, int t) { return (int)std::max<int64_t>(1, (n + t - 1) / t); }

// lumped nodal volume, original node order
__global__ void k_node_volume(int64_t nn, const int32_t* __restrict__ perm, const int64_t* __restrict__ nt_off,
                              const int32_t* __restrict__ nt_tet, const double* __restrict__ vol, double* V) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nn) return;
  double v = 0.0;
  for (int64_t e = nt_off[i]; e < nt_off[i + 1]; e++) v += vol[nt_tet[e]];
  V[perm[i]] = 0.25 * v;
}

// one block per state; per-thread partial sums over a fixed node stride, then a fixed tree
constexpr int EN_THREADS = 256;
__global__ void __launch_bounds__(EN_THREADS) k_energy(int64_t nn, const double* __restrict__ V,
                                                       const double* __restrict__ M, const double* __restrict__ H,
                                                       double* e) {
  __shared__ double red[EN_THREADS];
  const int64_t o = (int64_t)blockIdx.x * nn * 3;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < nn; i += EN_THREADS) {
    const double* m = M + o + 3 * i;
    const double* h = H + o + 3 * i;
    s += V[i] * (m[0] * h[0] + m[1] * h[1] + m[2] * h[2]);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = EN_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) e[blockIdx.x] = -0.5 * red[0];
}

// k = dm/dt at the state y (unit or not), field H of Ms y
__global__ void k_llg_rhs(int64_t n, const double* __restrict__ y, const double* __restrict__ H, double inv_ms,
                          double hx, double hy, double hz, double alpha, double* k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m0 = y[3 * i], m1 = y[3 * i + 1], m2 = y[3 * i + 2];
  const double h0 = H[3 * i] * inv_ms + hx, h1 = H[3 * i + 1] * inv_ms + hy, h2 = H[3 * i + 2] * inv_ms + hz;
  const double c0 = m1 * h2 - m2 * h1, c1 = m2 * h0 - m0 * h2, c2 = m0 * h1 - m1 * h0;  // m x h
  const double d0 = m1 * c2 - m2 * c1, d1 = m2 * c0 - m0 * c2, d2 = m0 * c1 - m1 * c0;  // m x (m x h)
  const double f = -1.0 / (1.0 + alpha * alpha);
  k[3 * i] = f * (c0 + alpha * d0);
  k[3 * i + 1] = f * (c1 + alpha * d1);
  k[3 * i + 2] = f * (c2 + alpha * d2);
}

// stage state y = m + c k and the magnetisation Ms y fed to the evaluation
__global__ void k_rk_stage(int64_t n3, const double* __restrict__ m, const double* __restrict__ k, double c, double Ms,
                           double* y, double* My) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n3) return;
  const double v = k ? m[i] + c * k[i] : m[i];
  y[i] = v;
  My[i] = Ms * v;
}

// m <- normalise(m + dt/6 (k1 + 2 k2 + 2 k3 + k4))
__global__ void k_rk4_final(int64_t n, double* m, const double* __restrict__ k1, const double* __restrict__ k2,
                            const double* __restrict__ k3, const double* __restrict__ k4, double dt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[3];
  for (int c = 0; c < 3; c++) {
    const int64_t j = 3 * i + c;
    v[c] = m[j] + dt / 6.0 * (k1[j] + 2.0 * k2[j] + 2.0 * k3[j] + k4[j]);
  }
  const double r = 1.0 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  for (int c = 0; c < 3; c++) m[3 * i + c] = v[c] * r;
}

struct Buf {
  double* p = nullptr;
  explicit Buf(size_t n) {
    if (cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      fail(DEMAG_ERR_OUT_OF_MEMORY, "LLG work buffer allocation failed");
    }
  }
  ~Buf() {
    if (p) cudaFree(p);
  }
};

void eval_any(Plan& P, const double* M, int B, double* u, double* H, cudaStream_t s) {
  if (P.opt.precision == DEMAG_FP64)
    eval_fp64(P, M, B, u, H, s);
  else
    eval_mixed(P, M, B, u, H, s);
}

}  // namespace

const double* node_volumes(Plan& P) {
  if (!P.node_vol) {
    P.node_vol = dalloc<double>(P, P.nn);
    k_node_volume<<<nblk(P.nn, 256), 256, 0, P.stream>>>(P.nn, P.node_perm, P.nt_off, P.nt_tet, P.tet_vol,
                                                         P.node_vol);
    DM_LAUNCH("k_node_volume");
    DM_CUDA(cudaStreamSynchronize(P.stream));
  }
  return P.node_vol;
}

void energy(Plan& P, const double* M, const double* H, int B, double* e, cudaStream_t s) {
  const double* V = node_volumes(P);
  k_energy<<<B, EN_THREADS, 0, s>>>(P.nn, V, M, H, e);
  DM_LAUNCH("k_energy");
}

void llg_rk4(Plan& P, double* m, int B, double Ms, double alpha, const double* hext, double dt, int steps,
             cudaStream_t s) {
  const int64_t n = (int64_t)B * P.nn, n3 = 3 * n;
  Buf k1(n3), k2(n3), k3(n3), k4(n3), y(n3), My(n3), H(n3), u(n);
  const double inv = 1.0 / Ms;
  double* ks[4] = {k1.p, k2.p, k3.p, k4.p};
  const double cs[4] = {0.0, 0.5 * dt, 0.5 * dt, dt};
  for (int step = 0; step < steps; step++) {
    for (int st = 0; st < 4; st++) {
      k_rk_stage<<<nblk(n3, 256), 256, 0, s>>>(n3, m, st ? ks[st - 1] : nullptr, cs[st], Ms, y.p, My.p);
      DM_LAUNCH("k_rk_stage");
      eval_any(P, My.p, B, u.p, H.p, s);
      k_llg_rhs<<<nblk(n, 256), 256, 0, s>>>(n, y.p, H.p, inv, hext[0], hext[1], hext[2], alpha, ks[st]);
      DM_LAUNCH("k_llg_rhs");
    }
    k_rk4_final<<<nblk(n, 256), 256, 0, s>>>(n, m, k1.p, k2.p, k3.p, k4.p, dt);
    DM_LAUNCH("k_rk4_final");
  }
  DM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace demag
