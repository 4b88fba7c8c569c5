// near_tc.cu -- the stored near field (Sec. 3.4: the direct-interaction
// coefficients are kept) applied on the tcgen05 tensor cores.
//
// Per tile of at most 128 target nodes (consecutive P2P target leaves in
// Morton order) and a block of 128 states the near field is the dense product
//     D[b][r] = sum_k A[b][k] W[r][k],   k = (column j, component c),
//     A[b][(j, c)] = M_c(node j, state b),   W[r][(j, c)] = W_c(target r, node j),
// over the union of the tile's columns (the distinct vertices of the source
// tets of its leaves' P2P lists; W is zero where a column is outside a row's
// own near set).  M = 128 states (tensor-memory lanes), N = rows padded to 16,
// K = columns in groups of 16, one k-step per (group, component).
//
// Split BF16: A = A_hi + A_lo and W = W_hi + W_lo (16 significant bits
// together); three MMAs per k-step (hi x hi, hi x lo, lo x hi) accumulate in
// FP32 in tensor memory.
//
// Offset of the states.  The product runs on M - Mbar, Mbar = M of the tile's
// first column (per state), and the epilogue adds S_i . Mbar with the row sums
// S_i = sum_j W_ij taken in FP64 at plan time:
//     u_i = sum_j W_ij . (M_j - Mbar) + S_i . Mbar.
// For smooth magnetisation the near-field terms of a node cancel to a small
// residual (a uniform M has no volume charge); M - Mbar is small over a tile,
// so the rounding of W and M to 16 bits and the tensor core's truncating
// accumulation act on small terms, and S_i . Mbar carries the large ones in
// FP32 (S_i itself is the cancelled sum).
//
// Data movement.  W is stored at plan time per tile in the order of use:
// per k-step the BF16 hi rows then the lo rows in the K-major no-swizzle
// core-matrix layout (8 rows x 16 bytes, the two 8-element halves of a k-step
// 128 bytes apart, 8-row groups 256 bytes apart), so one bulk copy per stage
// of three k-steps (one column group) fills a shared-memory ring slot; the M
// of the group's 16 columns (FP32, states innermost, 1.5 KB each) comes with
// it.  The A operand itself never touches shared memory: the warps that own
// the states read their M from the stage, split it into hi and lo and write it
// straight into a ring of tensor-memory slots (tcgen05.st), from which the MMA
// reads it.  One thread streams the stages (a ring of four in shared memory),
// one thread issues the MMAs and frees the slots with tcgen05.commit; the
// state warps move finished accumulators into FP32 totals (below) and at the
// end add the totals to u (rows are distinct nodes: no atomics).  Tensor
// memory holds two accumulators, the totals and an eight-slot A ring (512
// columns), so shared memory is left to the stages.
//
// Every wait is bounded: on expiry the kernel records DEMAG_ERR_TIMEOUT,
// stops issuing, waits (bounded) for its own copies and MMAs in flight, frees
// its tensor memory and returns.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace demag {

namespace {

using namespace tcx;

constexpr int NF_RING = 8;                       // A slots in tensor memory (k-steps in flight)
constexpr int NF_KSTEP_MAX = 64 * NF_ROWS;       // W bytes of one k-step: 2 limbs x 128 rows x 32 B
constexpr int NF_WPART = 3 * NF_KSTEP_MAX;       // W of one column group (x, y, z k-steps): 24 KB
constexpr int NF_MCOL = 3 * 128 * 4;             // M of one column for one state block: 1,536 B
constexpr int NF_STAGE = NF_WPART + 16 * NF_MCOL;  // ring slot: W and M of one column group, 48 KB
constexpr int NF_STAGES = 4;
constexpr int NF_CHUNK = 24;                     // k-steps per accumulator before it is promoted
constexpr int NF_PROMOTE_AT = 8;                 // ... promoted after this many k-steps of the next chunk
constexpr int NF_THREADS = 384;                  // 4 control warps + 2 x 4 state warps
constexpr int NF_TMEM_COLS = 512;  // accumulators D0, D1 (128 columns each), FP32 totals (128), A ring (8 x 16)
constexpr int NF_TOT0 = 256;
constexpr int NF_RING0 = 384;
constexpr int NF_NBARS = 2 * NF_STAGES + 2 * NF_RING + 4 + 1;
constexpr size_t NF_SMEM = (size_t)NF_STAGES * NF_STAGE + 8 * NF_NBARS + 16;
static_assert(NF_SMEM <= 227 * 1024, "shared memory of the near-field kernel");

// M per 128-state block in the layout of the kernel's copies: MP[sb][node][c][128]
// (zero for states beyond B), so the M of one column and one block is one
// contiguous 1,536-byte bulk copy
__global__ void k_nf_pack_m(int64_t nn, int B, const float* __restrict__ Ms, float* MP) {
  const int64_t node = blockIdx.x;
  const int sb = blockIdx.y;
  for (int q = threadIdx.x; q < 3 * 128; q += blockDim.x) {
    const int c = q >> 7, bl = q & 127, b = sb * 128 + bl;
    MP[(((int64_t)sb * nn + node) * 3 + c) * 128 + bl] = b < B ? Ms[(node * 3 + c) * (int64_t)B + b] : 0.f;
  }
}

// One CTA per (128-state block, tile); the state blocks of a tile are
// neighbours in launch order so the second reads the tile's W from L2.
//   warp 0       producer: per column group one stage = the group's W (one
//                bulk copy) and the M of its 16 columns (one bulk copy per
//                run of consecutive node ids, issued by the run's first lane)
//   warp 1       MMA issuer
//   warp 2       tensor-memory allocation
//   warps 4..11  state warps: warp 4 + 4 h + q owns tensor-memory lanes
//                32q .. 32q + 31 (states); half h converts the M of columns
//                8h .. 8h + 7 of every column group from shared memory into
//                the A ring of tensor memory (split BF16).
// A stage is free again when the MMAs of its three k-steps are done (one
// tcgen05.commit) and the eight state warps that read its M have arrived.
// Accumulation.  The tensor core adds each MMA's products into its FP32
// accumulator aligned to the larger operand, so its error grows with the
// number of MMAs an accumulator takes.  Every NF_CHUNK k-steps the issuer
// switches between two accumulators (D0, D1) and restarts the new one; the
// state warps add each finished chunk into FP32 totals in tensor memory
// (round to nearest) while the other accumulator fills.
__global__ void __launch_bounds__(NF_THREADS, 1)
    k_near_tc(const int32_t* __restrict__ order, const int64_t* __restrict__ woff, const int64_t* __restrict__ coff,
              const int32_t* __restrict__ ngrp,
              const int32_t* __restrict__ npad_t, const int32_t* __restrict__ rownode,
              const int32_t* __restrict__ cols, const unsigned char* __restrict__ W, const float* __restrict__ MP,
              const float* __restrict__ S, int64_t nn, int B, int nsb, float* u, int* err, int debug_no_copies) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t* bars = (uint64_t*)(sm + (size_t)NF_STAGES * NF_STAGE);
  uint32_t* tmem_slot = (uint32_t*)(bars + NF_NBARS);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* counts = (int*)(tmem_slot + 2);  // stages issued, stages consumed by the MMA issuer
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t slot_in_grid = blockIdx.x / nsb;  // the state blocks of a tile are neighbours in launch order
  const int sb = (int)(blockIdx.x - slot_in_grid * nsb);
  const int64_t tile = order ? order[slot_in_grid] : slot_in_grid;
  const int ng = ngrp[tile];
  if (ng == 0) return;  // uniform over the CTA
  const int npad = npad_t[tile];
  const int nk = 3 * ng, nch = (nk + NF_CHUNK - 1) / NF_CHUNK;
  const uint32_t kbytes = 64u * (uint32_t)npad;
  const uint32_t bar0 = smem_u32(bars);
  auto sfull = [&](int i) { return bar0 + 8u * i; };
  auto sempty = [&](int i) { return bar0 + 8u * (NF_STAGES + i); };
  auto afull = [&](int i) { return bar0 + 8u * (2 * NF_STAGES + i); };
  auto aempty = [&](int i) { return bar0 + 8u * (2 * NF_STAGES + NF_RING + i); };
  auto dfull = [&](int i) { return bar0 + 8u * (2 * NF_STAGES + 2 * NF_RING + i); };
  auto dfree = [&](int i) { return bar0 + 8u * (2 * NF_STAGES + 2 * NF_RING + 2 + i); };
  const uint32_t done = bar0 + 8u * (2 * NF_STAGES + 2 * NF_RING + 4);
  if (tid == 0) {
    for (int i = 0; i < NF_STAGES; i++) {
      mbar_init(sfull(i), 1);
      mbar_init(sempty(i), 1 + 8);  // the MMA commit and the four state warps that read its M
    }
    for (int i = 0; i < NF_RING; i++) {
      mbar_init(afull(i), 8);  // the four warps of the half that fills the slot
      mbar_init(aempty(i), 1);
    }
    for (int i = 0; i < 2; i++) {
      mbar_init(dfull(i), 1);
      mbar_init(dfree(i), 8);  // every state warp has read its rows of the chunk
    }
    mbar_init(done, 1);
    mbar_init_fence();
    *abort_flag = 0;
    counts[0] = counts[1] = 0;
  }
  if (warp == 2) tmem_alloc(smem_u32(tmem_slot), NF_TMEM_COLS);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t ring0 = smem_u32(sm);
  const int32_t* ct = cols + coff[tile];

  if (warp == 0) {
    // ---- producer (whole warp): one stage per column group
    const unsigned char* Wt = W + woff[tile];
    const float* MPb = MP + (int64_t)sb * nn * 384;
    int g = 0;
    int col_next = lane < 16 ? ct[lane] : 0;  // column ids one group ahead
    if (!debug_no_copies) {  // test hook: no stage is ever filled, so the waits for them expire
      for (; g < ng; g++) {
        const int col = col_next;
        if (g + 1 < ng && lane < 16) col_next = ct[16 * (g + 1) + lane];
        const int slot = g % NF_STAGES;
        int ok = 1;
        if (g >= NF_STAGES) {
          if (lane == 0) ok = mbar_wait(sempty(slot), (uint32_t)((g / NF_STAGES - 1) & 1), abort_flag) ? 1 : 0;
          ok = __shfl_sync(0xffffffffu, ok, 0);
        }
        if (!ok) {
          if (lane == 0) {
            if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
            *abort_flag = 1;
          }
          break;
        }
        if (*abort_flag) break;
        const uint32_t dst = ring0 + (uint32_t)slot * NF_STAGE;
        if (lane == 0) expect_tx(sfull(slot), 3u * kbytes + 16u * NF_MCOL);
        __syncwarp();
        if (lane == 0) bulk_load(dst, Wt + (int64_t)g * 3 * kbytes, 3u * kbytes, sfull(slot));
        // M of the 16 columns: one bulk copy per run of consecutive node ids
        // (M is node-major, so a run is contiguous; Morton-sorted columns give
        // ~2.6 runs per group)
        const int prev = __shfl_up_sync(0xffffffffu, col, 1);
        const bool start = lane < 16 && (lane == 0 || col != prev + 1);
        const uint32_t starts = __ballot_sync(0xffffffffu, start) & 0xffffu;
        if (start) {
          const uint32_t above = starts & ~((2u << lane) - 1u);  // run starts after this lane
          const int len = (above ? __ffs(above) - 1 : 16) - lane;
          bulk_load(dst + NF_WPART + (uint32_t)lane * NF_MCOL, MPb + (int64_t)col * 384, (uint32_t)len * NF_MCOL,
                    sfull(slot));
        }
        __syncwarp();
      }
    }
    if (lane == 0) counts[0] = g;
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {  // ---- MMA issuer: running ring positions, no divisions in the loop
      const uint32_t id = idesc_bf16(128, npad);
      const uint64_t dstep = (uint64_t)(kbytes >> 4);  // descriptor start-address step of one k-step
      const uint64_t dlimb = (uint64_t)((32u * (uint32_t)npad) >> 4);
      uint32_t sslot = 0, sphase = 0, aslot = 0, aphase = 0, db = 0;
      int kc = 0, c = 0, consumed = 0;
      bool bad = false;
      for (int g = 0; g < ng && !bad; g++) {
        if (!mbar_wait(sfull(sslot), sphase, abort_flag)) {
          bad = true;
          break;
        }
        consumed = g + 1;
        uint64_t bhi = sdesc(ring0 + sslot * NF_STAGE);
#pragma unroll
        for (int j = 0; j < 3; j++) {
          if (kc == 0 && c >= 2 && !mbar_wait(dfree(db), (uint32_t)((c / 2 - 1) & 1), abort_flag)) {
            bad = true;  // the state warps have not read the chunk that last used this accumulator
            break;
          }
          if (!mbar_wait(afull(aslot), aphase, abort_flag)) {
            bad = true;
            break;
          }
          fence_after();
          const uint32_t a = tmem + NF_RING0 + aslot * 16, d = tmem + 128 * db;
          mma_ts_bf16(d, a, bhi, id, kc > 0 ? 1u : 0u);
          mma_ts_bf16(d, a, bhi + dlimb, id, 1u);
          mma_ts_bf16(d, a + 8, bhi, id, 1u);
          mma_commit(aempty(aslot));  // the A slot is free once these are done
          bhi += dstep;
          if (++aslot == NF_RING) {
            aslot = 0;
            aphase ^= 1u;
          }
          if (++kc == NF_CHUNK) {  // the chunk is complete
            mma_commit(dfull(db));
            kc = 0;
            db ^= 1u;
            c++;
          }
        }
        if (bad) break;
        mma_commit(sempty(sslot));  // the stage's W after its last k-step
        if (++sslot == NF_STAGES) {
          sslot = 0;
          sphase ^= 1u;
        }
      }
      if (!bad && kc > 0) mma_commit(dfull(db));  // the last, partial chunk
      if (bad) {
        if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
        *abort_flag = 1;
      }
      counts[1] = consumed;
      mma_commit(done);  // arrives when every MMA issued above has completed
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---- state warps
    const int h = (warp - 4) >> 2, q = warp & 3;
    const int bl = 32 * q + lane, b = sb * 128 + bl;
    const bool live = b < B;
    float mbar[3];  // M of the tile's first column, this state
    {
      const float* m0 = MP + ((int64_t)sb * nn + ct[0]) * 384 + bl;
#pragma unroll
      for (int cc = 0; cc < 3; cc++) mbar[cc] = m0[cc * 128];
    }
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    int promoted = 0;
    bool bad = false;
    auto wait_warp = [&](uint32_t bar, uint32_t parity) {
      int ok = 1;
      if (lane == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
      return __shfl_sync(0xffffffffu, ok, 0) != 0;
    };
    // add this warp's rows (16-row chunks 2 i + h) of accumulator chunk c into
    // the FP32 totals (round to nearest), which live in tensor memory too
    // (columns NF_TOT0 + row; the first chunk initialises them)
    auto promote = [&](int c) {
      if (!wait_warp(dfull(c & 1), (uint32_t)((c / 2) & 1))) {
        bad = true;
        return;
      }
      fence_after();
      for (int c0 = 16 * h; c0 < npad; c0 += 32) {
        uint32_t r[16];
        tmem_ld16(tmem + lane_off + 128 * (c & 1) + c0, r);
        if (c > 0) {
          uint32_t t[16];
          tmem_ld16(tmem + lane_off + NF_TOT0 + c0, t);
#pragma unroll
          for (int i = 0; i < 16; i++) r[i] = __float_as_uint(__uint_as_float(t[i]) + __uint_as_float(r[i]));
        }
        tmem_st16(tmem + lane_off + NF_TOT0 + c0, r);
        tmem_wait_st();
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(dfree(c & 1));
      promoted = c + 1;
    };
    // one hand-off per column group: its three k-steps (x, y, z) fill three
    // consecutive A slots, half h the group's columns 8h .. 8h + 7 (tensor-
    // memory columns 4h .. 4h + 3 of each limb).  Every state warp takes part
    // in every group, so each waits for every use of a stage slot and of an A
    // slot in order: a phase parity can never alias an older phase.  The MMAs
    // complete in order, so the slot of the group's last k-step being free
    // means the other two are free as well.
    for (int g = 0; g < ng && !bad; g++) {
      const int slot = g % NF_STAGES, ks0 = 3 * g;
      if (!wait_warp(sfull(slot), (uint32_t)((g / NF_STAGES) & 1))) {
        bad = true;
        break;
      }
      const float* mst = (const float*)(sm + (size_t)slot * NF_STAGE + NF_WPART) + 8 * h * 384;  // [column][c][128]
      float v[3][8];
#pragma unroll
      for (int k = 0; k < 8; k++)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) v[cc][k] = mst[(k * 3 + cc) * 128 + bl] - mbar[cc];
      __syncwarp();
      if (lane == 0) mbar_arrive(sempty(slot));  // this warp has read the stage's M
      const int kl = ks0 + 2;
      if (kl >= NF_RING && !wait_warp(aempty(kl % NF_RING), (uint32_t)((kl / NF_RING - 1) & 1))) {
        bad = true;  // the MMAs of k-step kl - NF_RING have not read its slot
        break;
      }
      fence_after();
#pragma unroll
      for (int cc = 0; cc < 3; cc++) {
        uint32_t hi[4], lo[4];
        split_bf16<8>(v[cc], hi, lo);
        const uint32_t a = tmem + lane_off + NF_RING0 + ((ks0 + cc) % NF_RING) * 16 + 4 * h;
        tmem_st4(a, hi);
        tmem_st4(a + 8, lo);
      }
      tmem_wait_st();
      fence_before();
      __syncwarp();
      if (lane == 0)
#pragma unroll
        for (int cc = 0; cc < 3; cc++) mbar_arrive(afull((ks0 + cc) % NF_RING));
      // the earlier accumulator chunks, once this one is well under way
      const int c = kl / NF_CHUNK;
      if (kl - c * NF_CHUNK >= NF_PROMOTE_AT)
        while (!bad && promoted < c) promote(promoted);
    }
    while (!bad && promoted < nch) promote(promoted);
    if (bad && lane == 0) {
      if (!*abort_flag) atomicExch(err, (int)DEMAG_ERR_TIMEOUT);
      *abort_flag = 1;
    }
    // this warp's rows of the totals -> u (each row a distinct node; the
    // warp's lanes are consecutive states, so each row's update coalesces)
    if (!bad && !*abort_flag) {
      const int32_t* rn = rownode + tile * NF_ROWS;
      fence_after();
      for (int c0 = 16 * h; c0 < npad; c0 += 32) {
        uint32_t t[16];
        tmem_ld16(tmem + lane_off + NF_TOT0 + c0, t);
#pragma unroll
        for (int i = 0; i < 16; i++) {
          const int node = rn[c0 + i];
          if (node >= 0 && live) {
            const float* Si = S + 3ll * node;
            u[(int64_t)node * B + b] +=
                __uint_as_float(t[i]) + (Si[0] * mbar[0] + Si[1] * mbar[1] + Si[2] * mbar[2]);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid == 0) {
    // every MMA issued has completed before the tensor memory goes (bounded)
    mbar_wait(done, 0u, nullptr);
    // stages issued but never consumed still land in the ring: wait for them (bounded)
    if (*abort_flag)
      for (int st = counts[1]; st < counts[0]; st++)
        mbar_wait(sfull(st % NF_STAGES), (uint32_t)((st / NF_STAGES) & 1), nullptr);
  }
  fence_before();
  __syncthreads();
  if (warp == 2) tmem_dealloc(tmem, NF_TMEM_COLS);
}

}  // namespace

size_t nf_mp_floats(const Plan& P, int B) {
  return P.nf_W ? (size_t)((B + 127) / 128) * (size_t)P.nn * 384 : 0;
}

void launch_near_tc(Plan& P, const float* Ms, float* MP, int B, float* u_s, int* err, cudaStream_t s) {
  if (P.nf_ntiles == 0) return;
  smem_opt_in((const void*)k_near_tc, NF_SMEM);
  const unsigned nsb = (unsigned)((B + 127) / 128);
  k_nf_pack_m<<<dim3((unsigned)P.nn, nsb), 128, 0, s>>>(P.nn, B, Ms, MP);
  DM_LAUNCH("k_nf_pack_m");
  const dim3 grid((unsigned)(nsb * P.nf_ntiles));
  // launch order: a grid of a few waves starts its largest tiles first (a short
  // tail); a long one runs in Morton order, so that the CTAs in flight gather
  // the M of neighbouring columns from L2 (on GB300 the first is faster on the
  // 224k-tet ball at 128 states, ~2 waves; the second on the 559k-tet ball at
  // 256 states, ~10 waves)
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P.device);
  const int32_t* order = (int64_t)grid.x < 4ll * nsm ? P.nf_order : nullptr;
  k_near_tc<<<grid, NF_THREADS, NF_SMEM, s>>>(order, P.nf_woff, P.nf_coff, P.nf_ng, P.nf_npad, P.nf_rownode, P.nf_cols,
                                              P.nf_W, MP, P.nf_S, P.nn, B, (int)nsb, u_s, err, P.debug_flags & 1);
  DM_LAUNCH("k_near_tc");
}

}  // namespace demag
