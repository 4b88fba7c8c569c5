/*
 * demag.h -- C ABI of the GB300 tetrahedral-FMM demagnetisation library
 * (libdemag.so).
 *
 * Operation (Palmesi et al., Sec. 1, Eq. (1)-(2)): for a tetrahedral mesh whose
 * tets carry an affine (P1, nodal) magnetisation M, compute at every node
 *     u(r_i) = 1/(4 pi) sum_j int_{Omega_j} M(r') . grad'(1/|r_i - r'|) dr'
 * by the fast multipole method of Sec. 2-3: analytic near field over source
 * tets (P2P, Sec. 2.1), exact tet moments (P2M, Sec. 2.2 Eq. expCoeffs),
 * M2M / M2L / L2L on an octree (Sec. 2 steps 2-4, Sec. 2.3) and L2P (step 5),
 * with the octree, multipole acceptance criterion and dual tree traversal of
 * Sec. 3.1-3.3.  H is the mass-lumped field -grad u (Sec. 4.1, "mass lumping
 * was used for the computation of the B-field").
 *
 * Units: lengths in mesh units, M in A/m, u in A, H in A/m; no mu0.
 * Sign: H = -grad u, so H = -M/3 inside a uniformly magnetised ball.
 *
 * Error behaviour: no call throws across the ABI; every call returns a
 * demag_status.  demag_last_error() gives a thread-local message for the last
 * failing call.  On error, outputs are unspecified; a plan stays valid unless
 * the status is DEMAG_ERR_CUDA or DEMAG_ERR_OUT_OF_MEMORY.
 *
 * Threads: a plan is read-only during demag_eval except for its internal
 * workspace, so concurrent demag_eval calls on ONE plan must be serialised by
 * the caller (they share the workspace); different plans are independent.
 */
#ifndef DEMAG_H
#define DEMAG_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct demag_plan_s* demag_plan;

typedef enum {
  DEMAG_OK = 0,
  DEMAG_ERR_INVALID_ARG = 1,    /* bad pointer, size, index, p, leaf or theta     */
  DEMAG_ERR_DEGENERATE_TET = 2, /* |vol| < 1e-14 * (longest edge)^3               */
  DEMAG_ERR_OUT_OF_MEMORY = 3,  /* device allocation failed                        */
  DEMAG_ERR_CUDA = 4,           /* a CUDA runtime call failed                      */
  DEMAG_ERR_TIMEOUT = 5,        /* a bounded device wait expired                   */
  DEMAG_ERR_UNSUPPORTED = 6,    /* option combination not built                    */
  DEMAG_ERR_INTERNAL = 7        /* a plan's index lists failed their bounds audit
                                   (a planner bug; demag_last_error() names the list) */
} demag_status;

/* Arithmetic of the evaluation.  DEMAG_FP64: every stage in FP64 (the
 * reference path).  Mixed modes keep the near-field integrals in FP64 (they are
 * computed once, at plan time, when near_mode = 1) and run moments, M2M, M2L,
 * L2L, L2P and the near-field application in FP32 arithmetic (FP32 CUDA
 * cores, TF32 tensor cores, or split-BF16 x3 tensor cores for M2L), with the
 * expansion coefficients scaled per octree level. */
typedef enum {
  DEMAG_FP64 = 0,
  DEMAG_MIXED_FP32 = 1,
  DEMAG_MIXED_TF32 = 2,
  DEMAG_MIXED_BF16X3 = 3, /* M2L operands in two BF16 limbs (16 bits), 3 MMAs per k-step */
  DEMAG_MIXED_BF16X6 = 4  /* M2L operands in three BF16 limbs (24 bits = FP32), 6 MMAs per k-step */
} demag_precision;

typedef struct {
  int p;               /* Taylor order, |n| <= p (Sec. 2.2); 1..12        */
  int leaf_size;       /* split a cell holding more tets than this        */
  double theta;        /* MAC: accept iff (r_T + r_S) < theta |c_T - c_S| */
  int precision;       /* demag_precision                                  */
  int near_mode;       /* 0: near field integrated at every eval (FP64);
                          1: near-field coefficients W precomputed in FP64
                             at plan time and applied at eval (Sec. 3.4 stores
                             the direct-interaction coefficients)            */
  int max_batch;       /* largest batch B a demag_eval will be given       */
  int autotune;        /* bit 0 (1): at plan time, time the launch shapes of
                             the tensor-core M2L (TF32 / split BF16) on this
                             plan's own interaction lists and keep the
                             fastest (adds up to ~1 s to demag_plan_create);
                             otherwise a fixed default shape.
                          bit 1 (2): leaf size -- build the plan for
                             leaf_size / 2, leaf_size, 2 leaf_size and
                             4 leaf_size, time one evaluation of max_batch
                             states on each and keep the fastest (up to four
                             plan builds; demag_plan_stats reports the leaf
                             kept).
                          bit 2 (4): expansion order -- the smallest p in
                             {4, 6, 8, 10} whose u and H on one synthetic
                             state are within 5e-5 (rel-L2) of an FP64
                             evaluation at p = 10 with the same leaf and
                             theta; the p argument is then ignored and
                             demag_plan_stats reports the p kept.  Applied
                             before the leaf tuning.  0..7
                          Tuner cache: when the environment variable
                             DEMAG_TUNE_CACHE names a file, the choices of a
                             tuned plan (p, leaf size, M2L launch shape) are
                             appended to it as one text line keyed by a 64-bit
                             hash of the mesh (node coordinates and tets), of
                             every option except profile and graph, and of
                             the device (name, SM count, compute capability);
                             a later plan with the same key is built from the
                             cached choices without timing (the same plan the
                             tuners keep).  Unparsable or out-of-range lines
                             are skipped; a file that cannot be written only
                             sets a warning in demag_last_error().          */
  int profile;         /* 1: time every stage of demag_eval with CUDA events
                          on the eval stream (adds one synchronisation per
                          call); read with demag_plan_stats                  */
  int m2l_targets_per_cta; /* tensor-core M2L launch shape (TF32 / split BF16,
                          p in {4, 6, 8, 10}): target cells sharing each
                          source's moments in one CTA, 1 or 2; 0 = default
                          (1) or the autotuner's choice                     */
  int m2l_kps;         /* tensor-core M2L: k-steps per shared-memory slot,
                          1..8; 0 = default (2) or the autotuner's choice.
                          Every launch shape gives bit-identical results.   */
  int m2l_promote;     /* tensor-core M2L, one target per CTA: every this
                          many sources the leading accumulator rows are
                          moved into FP32 registers (round to nearest) and
                          restarted at zero; 0 = default (8), < 0 = never.
                          The tensor core adds products into its FP32
                          accumulator with alignment to the larger operand,
                          so without this the error follows the running
                          value, which for smooth M is far above the result */
  int m2l_promote_rows; /* rows moved (rounded up to 16, at most 64); 0 = 16 */
  int m2l_table_batch; /* TF32 / split BF16: batches B <= this run the M2L in
                          FP32 on CUDA cores, from a per-plan table of the
                          translation derivatives (p in {4, 6, 8}); larger
                          batches use the tensor cores, whose tiles hold 128
                          states.  0 = default (8), < 0 = never.  The FP32
                          precision always uses the table M2L when there is
                          one.                                              */
  int sources;         /* DEMAG_SOURCES_TETS (0): P1 magnetisation on the
                          tetrahedra, exact moments and analytic near field
                          (the paper's method); DEMAG_SOURCES_DIPOLES (1):
                          every node a point dipole V_i M_i (V_i its lumped
                          volume) with the Laplace kernel and the same tree,
                          lists and translations -- the node-dipole
                          comparison the paper makes (Sec. 4); needs
                          near_mode = 1.  DEMAG_SOURCES_PATCHES (2): the
                          paper's own clustering (Sec. 2.1, 3.1-3.2): node i
                          carries lambda_i M over every tet around it, is
                          binned by its own key, and a cell's source radius
                          reaches the farthest vertex of the tets around its
                          nodes; exact patch moments and analytic patch near
                          field; the same u as the tets up to the FMM
                          truncation; needs near_mode = 1                  */
  int near_tc;         /* DEMAG_MIXED_BF16X3 with near_mode = 1: 0
                          (default) applies the stored near-field
                          coefficients (Sec. 3.4) on the tensor cores --
                          tiles of up to 128 target nodes over the union of
                          their source columns, coefficients and M in two
                          BF16 limbs (16 significant bits; up to ~1e-5
                          relative error per product), three MMAs per
                          k-step, FP32 accumulation; < 0: FP32 CUDA cores,
                          as in the other mixed precisions (BF16X6 always) */
  int graph;           /* 1: demag_eval with device pointers (and profile =
                          0) runs the first call with a given (M, u, H,
                          batch, workspace) directly, records it as a CUDA
                          graph and replays that graph with one launch on
                          later calls with the same pointers (as
                          demag_eval_multi does for several plans; launch
                          arguments, including demag_plan_debug flags, are
                          those of the recorded call); 0 (default): every
                          call launches its kernels                         */
  int m2l_split_degree; /* DEMAG_MIXED_BF16X3, tensor-core M2L: 0 (default)
                          forms the products with the second BF16 limb
                          (hi x lo, lo x hi) only for the terms of degree
                          |m| + |n| <= p - 4 of the translation (Sec. 2.3;
                          p - 3 for p < 8); the highest degrees, whose share of the
                          expansion falls off like a power of the cell
                          size over the distance, take hi x hi alone
                          (about half the MMAs); < 0: both products for
                          every term; > 0 is invalid                      */
} demag_options;

enum { DEMAG_SOURCES_TETS = 0, DEMAG_SOURCES_DIPOLES = 1, DEMAG_SOURCES_PATCHES = 2 };

/* Defaults: p=4, leaf_size=32, theta=0.5, DEMAG_FP64, near_mode=0, max_batch=1,
 * autotune=0, profile=0, m2l_targets_per_cta=0, m2l_kps=0, m2l_promote=0, m2l_promote_rows=0,
 * m2l_table_batch=0, sources=0, near_tc=0, graph=0, m2l_split_degree=0. */
void demag_options_default(demag_options* opt);

/* Build a plan (Sec. 3.1-3.3): octree over the bounding cube, radii, MAC and
 * dual tree traversal into M2L and P2P lists, tet geometry, exact-moment
 * operators and, for near_mode=1, the near-field coefficients.
 *   nodes : n_nodes x 3 doubles, row-major (x,y,z).  Host or device pointer.
 *   tets  : n_tets x 4 int32, 0-based node indices, either orientation.
 *           Host or device pointer.
 *   p, leaf_size, theta override the corresponding fields of *opt.
 *   opt   : may be NULL (defaults).
 *   out   : receives the plan.  The plan copies nodes and tets; the caller
 *           keeps ownership of its arrays.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL pointers, n_nodes<4, n_tets<1, index out
 * of range, p outside 1..12, leaf_size<1, theta<=0 or non-finite, max_batch<1),
 * DEMAG_ERR_DEGENERATE_TET, DEMAG_ERR_OUT_OF_MEMORY, DEMAG_ERR_CUDA,
 * DEMAG_ERR_INTERNAL (the finished plan failed its bounds audit, see
 * demag_plan_audit; no plan is returned).
 * theta >= 1 is accepted; demag_last_error() then warns that expansions may
 * not converge.  Runs on the current CUDA device, on its own stream, and
 * synchronises before returning. */
demag_status demag_plan_create(const double* nodes, int64_t n_nodes, const int32_t* tets, int64_t n_tets, int p,
                               int leaf_size, double theta, const demag_options* opt, demag_plan* out);

/* Evaluate u (and H) for `batch` magnetisation states (Sec. 2 steps 1-5 + P2P,
 * Sec. 4.1 mass lumping).
 *   M : batch x n_nodes x 3 doubles (state-major), nodal magnetisation.
 *   u : batch x n_nodes doubles, output.
 *   H : batch x n_nodes x 3 doubles, output; may be NULL.
 *   M, u, H must be all device pointers or all host pointers.  With device
 *   pointers the call is asynchronous on `cuda_stream` (a cudaStream_t; NULL =
 *   the legacy default stream).  With host pointers the inputs are copied to
 *   the device, and the call returns after the outputs are back in host
 *   memory.  batch must be in 1..max_batch.
 * Nodes that belong to no tet get their potential, and H = 0. */
demag_status demag_eval(demag_plan plan, const double* M, int batch, double* u, double* H, void* cuda_stream);

/* Pointwise field H = -grad u at the interior nodes (Sec. 4.1-4.2: computing H
 * directly, instead of from the potential by mass lumping, gives lower
 * errors): the gradient of the local expansions (L2P of -grad u) plus the field
 * of the near tets' charges in closed form -- the affine surface charges n.M of
 * their faces and the constant volume charges -div M.  At an interior node the
 * face charges of the faces through the node cancel pairwise between the two
 * tets of each face (M is continuous) and are left out.  At boundary nodes
 * (nodes on a face of exactly one tet) the pointwise field is singular; there
 * H holds the mass-lumped field of demag_eval.
 *   M : batch x n_nodes x 3, u : batch x n_nodes, H : batch x n_nodes x 3; DEVICE
 *       pointers; u as demag_eval returns it.
 * FP64 plans (DEMAG_FP64) with tet sources; either near_mode.  The first call
 * finds the boundary nodes (on the host) and allocates a device buffer of
 * 3 x n_nodes x batch doubles kept by the plan.  Asynchronous on cuda_stream.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL or host pointers, batch out of range),
 * DEMAG_ERR_UNSUPPORTED (other precisions or sources), DEMAG_ERR_OUT_OF_MEMORY,
 * DEMAG_ERR_CUDA. */
demag_status demag_eval_field(demag_plan plan, const double* M, int batch, double* u, double* H, void* cuda_stream);

/* Device-side status of the most recent evaluation of `plan` (demag_eval,
 * demag_eval_noalloc, or this plan's part of a demag_eval_multi submission).
 * Calls with device pointers are asynchronous, so a bounded device wait that
 * expires in one of their kernels cannot be reported by the call itself; the
 * kernel records it in a device flag instead.  This synchronises cuda_stream
 * (the stream the evaluation was issued on) and returns DEMAG_ERR_TIMEOUT if
 * that flag is set -- the outputs of that evaluation are then unspecified and
 * the plan stays valid -- else DEMAG_OK (also for a plan never evaluated).
 * Host-pointer calls of demag_eval check the flag themselves.  The flag of
 * demag_eval_noalloc lives in the shared fixed scratch area and is cleared by
 * the next demag_eval_noalloc call on the same device, so query it before that
 * call.  Errors: DEMAG_ERR_INVALID_ARG (NULL plan), DEMAG_ERR_CUDA. */
demag_status demag_eval_status(demag_plan plan, void* cuda_stream);

/* Size of the fixed scratch area used by demag_eval_noalloc (64 MiB). */
#define DEMAG_NOALLOC_SCRATCH_BYTES (64ull * 1024ull * 1024ull)

/* demag_eval without any device allocation.  (The paper has no counterpart:
 * this is a service of the library.)  For callers that must not allocate
 * device memory while they run -- e.g. an application whose own pool allocator
 * has reserved the device memory and forbids further cudaMalloc/cudaFree, or a
 * latency-critical loop that cannot pay the implicit synchronisation of
 * cudaMalloc/cudaFree.  demag_eval allocates its workspace on its first call;
 * this entry point instead takes all of its scratch from one file-scope device
 * array of DEMAG_NOALLOC_SCRATCH_BYTES that the CUDA runtime reserves on every
 * device that loads the library, for the lifetime of the process.
 *   plan, batch : as for demag_eval (batch is not limited by max_batch).
 *   M, u, H     : DEVICE pointers only (H may be NULL); same layouts and results
 *                 as demag_eval.  The call is asynchronous on cuda_stream.
 * Errors: DEMAG_ERR_INVALID_ARG for NULL or host pointers, batch < 1, or a plan
 * and batch whose scratch exceeds DEMAG_NOALLOC_SCRATCH_BYTES (the message gives
 * both sizes); DEMAG_ERR_CUDA if the scratch address cannot be resolved.  A
 * bounded device wait that expires in the kernels is not seen by this
 * asynchronous call: check demag_eval_status before the next call.
 * The first call on a device resolves the array's device address with that
 * device current (one cudaGetSymbolAddress), so make that first call before any
 * stream capture.  The address is kept per device and CUDA context: a call
 * under a different context of the device (for instance after
 * cudaDeviceReset) resolves it again.  All calls on a device share the array and it keeps the last
 * call's contents (each call clears what must start at zero); calls that
 * overlap on the GPU race on it and must be serialised by the caller.
 * With opt.profile = 1 the stage timers are not updated by this entry point. */
demag_status demag_eval_noalloc(demag_plan plan, const double* M, int batch, double* u, double* H,
                                void* cuda_stream);

/* Evaluate several plans (meshes of any sizes, each with its own batch of
 * states) through one submission (Sec. 4 runs one mesh at a time; batching
 * meshes is a service of the library).
 *   plans   : n_plans plans, distinct.
 *   M, u, H : n_plans DEVICE pointers each, layouts as for demag_eval; H may be
 *             NULL (no H for any plan) or hold NULL entries.
 *   batch   : n_plans batch sizes, each in 1..max_batch of its plan.
 * Results are bit-identical to n_plans separate demag_eval calls.  The first
 * call with a given (plans, batches, pointers) signature runs the work directly
 * on cuda_stream and then records it as a CUDA graph (one branch per plan, so
 * the meshes' kernels may overlap); later calls with the same signature replay
 * the graph with a single launch, asynchronously on cuda_stream.  A few graphs
 * are cached (least recently used dropped first); destroying a plan or
 * enlarging its workspace drops the graphs that used it.  The first call must
 * not itself be issued while cuda_stream is being captured.  Stage timers
 * (opt.profile) are not updated by this entry point.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL arrays or pointers, n_plans < 1, a
 * repeated plan, host pointers, batch out of range), DEMAG_ERR_CUDA. */
demag_status demag_eval_multi(const demag_plan* plans, int n_plans, const double* const* M, const int* batch,
                              double* const* u, double* const* H, void* cuda_stream);

/* Magnetostatic self-energy of B states (the use of H the paper makes next to
 * the potential, Sec. 4.1-4.2):
 *   e[b] = -(1/2) sum_i V_i M_{b,i} . H_{b,i},   E = mu0 e,
 * V_i the lumped volume of node i (sum over its tets of |Omega_t| / 4; the
 * mass lumping of H).  M and H as returned by / given to demag_eval: DEVICE
 * pointers, (B, N_n, 3); e: B doubles, DEVICE.  Deterministic (fixed-order
 * reduction).  Asynchronous on cuda_stream.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL, batch < 1, host pointers). */
demag_status demag_energy(demag_plan plan, const double* M, const double* H, int batch, double* e,
                          void* cuda_stream);

/* Landau-Lifshitz-Gilbert stepping of B independent magnetisation states on
 * the plan's mesh with the demagnetising field as the effective field (plus a
 * uniform applied field), in reduced units:
 *   dm/dt = -1/(1 + alpha^2) [ m x h + alpha m x (m x h) ],
 *   h = H_demag(Ms m) / Ms + h_ext,  t in units of 1/(gamma mu0 Ms).
 * `steps` classical fourth-order Runge-Kutta steps of size dt; each stage's
 * field is one demag_eval of all B stage states (batch <= max_batch); m is
 * renormalised to unit length after each step.
 *   m      : DEVICE, (B, N_n, 3) unit vectors, advanced in place.
 *   h_ext  : 3 doubles (HOST) or NULL (zero).
 * Synchronous (returns when the steps are done).
 * Errors: DEMAG_ERR_INVALID_ARG (NULL m, batch out of range, Ms <= 0,
 * alpha < 0, dt <= 0, steps < 0, host m), DEMAG_ERR_OUT_OF_MEMORY, DEMAG_ERR_CUDA. */
demag_status demag_llg_rk4(demag_plan plan, double* m, int batch, double Ms, double alpha, const double* h_ext,
                           double dt, int steps, void* cuda_stream);

demag_status demag_plan_destroy(demag_plan plan);

/* Test hooks (the paper has no counterpart).
 * flags bit 0, the error path of the bounded device waits: the tensor-core near field (DEMAG_MIXED_BF16X3,
 * near_mode = 1) issues none of its coefficient copies, so its MMA issuer's
 * bounded wait for them expires (after about a second) with no copy and no MMA
 * in flight; the kernel records DEMAG_ERR_TIMEOUT, frees its tensor memory and
 * returns.  demag_eval then returns DEMAG_ERR_TIMEOUT for host pointers, and
 * demag_eval_status reports it for device pointers; the plan and the CUDA
 * context stay usable.
 * flags bit 1, the error path of the plan audit: demag_plan_audit also audits
 * a scratch copy of the M2L source list whose last entry is set to n_cells
 * (only the audit reads the copy; the plan's own lists are untouched), so it
 * returns DEMAG_ERR_INTERNAL naming that entry.
 * flags = 0 restores normal behaviour.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL plan, unknown flag bits). */
demag_status demag_plan_debug(demag_plan plan, int flags);

/* Bounds audit of the plan's index lists (every list an evaluation follows
 * into another array: node and tet permutations, cell links and ranges, the
 * M2L and P2P lists of Sec. 3.3, support nodes, near-field columns and tile
 * rows, M2L operator indices and groups, gradient-operator columns): each
 * list's count against its allocation, then every entry against the range of
 * the array it indexes, by device kernels that only read the lists.
 * demag_plan_create runs it on every plan before returning it; this call runs
 * it again (a plan's lists are never modified after planning).  Synchronous.
 * Errors: DEMAG_ERR_INVALID_ARG (NULL plan), DEMAG_ERR_INTERNAL (a list failed:
 * demag_last_error() gives the list, the first bad position and its value),
 * DEMAG_ERR_OUT_OF_MEMORY, DEMAG_ERR_CUDA. */
demag_status demag_plan_audit(demag_plan plan);

/* Stages of demag_eval, for the per-stage timers. */
enum {
  DEMAG_STAGE_GATHER = 0, /* M to the sorted, state-innermost layout          */
  DEMAG_STAGE_P2M = 1,    /* exact tet moments of the source leaves           */
  DEMAG_STAGE_M2M = 2,
  DEMAG_STAGE_M2L = 3,
  DEMAG_STAGE_L2L = 4,
  DEMAG_STAGE_L2P = 5,
  DEMAG_STAGE_NEAR_PREP = 6, /* per-tet records of the FP64 on-the-fly near field, one state */
  DEMAG_STAGE_P2P = 7,
  DEMAG_STAGE_H = 8,         /* mass-lumped H and the output layout           */
  DEMAG_N_STAGES = 9
};

typedef struct {
  int64_t n_nodes, n_tets;
  int64_t n_cells, n_leaves, n_levels;
  int64_t n_m2l;         /* M2L cell pairs                                   */
  int64_t n_p2p;         /* P2P leaf pairs                                   */
  int64_t n_p2p_pairs;   /* (target node, source tet) pairs in the near field */
  int64_t n_near_cols;   /* stored (target node, source node) coefficients   */
  int64_t device_bytes;  /* device memory held by the plan                   */
  double lo[3], side, scale; /* bounding cube and Morton scale              */
  double plan_ms;        /* wall time of demag_plan_create (with the order and
                            leaf tuning when autotune asks for them)        */
  int p, leaf_size, precision, near_mode, max_batch;
  double theta;
  int64_t eval_launches;           /* kernels launched by the last demag_eval */
  int64_t n_evals_profiled;        /* evals accumulated in stage_ms          */
  double stage_ms[DEMAG_N_STAGES]; /* summed per-stage device time (profile=1) */
  int64_t stage_launches[DEMAG_N_STAGES];
  int64_t n_m2l_ops;     /* distinct M2L translation keys (level difference,
                            lattice offset) tabulated for the tensor-core and
                            table-driven M2L of the mixed path (0: none)    */
  int m2l_kps;           /* tensor-core M2L ring: k-steps per slot          */
  int m2l_ring_bytes;    /* tensor-core M2L ring: shared memory per CTA     */
  int m2l_targets_per_cta; /* tensor-core M2L: target cells sharing each
                            source's moments in one CTA (1 or 2)            */
  int64_t n_near_tiles;  /* tiles of the tensor-core near field (0: none)   */
  int64_t near_tile_cols; /* columns of those tiles, summed (groups of 16)  */
  int64_t near_bytes;    /* bytes of stored near-field coefficients read by
                            one evaluation of up to 256 states (FP64, FP32
                            or split-BF16 layout, whichever the plan holds) */
  int tune_source;       /* 0: autotune = 0; 1: the tuners timed their
                            candidates; 2: their choices were read from the
                            DEMAG_TUNE_CACHE file                           */
} demag_stats;

demag_status demag_plan_stats(demag_plan plan, demag_stats* out);
/* Zero the per-stage timers. */
demag_status demag_plan_reset_timers(demag_plan plan);

/* Host copies of the tree and lists, for bit-exact checks.  Every pointer may
 * be NULL; sizes from demag_plan_stats.  Keys and permutations follow the
 * readings of Sec. 3.1 documented with the oracle: 63-bit Morton keys (x in
 * bit 3b, y in 3b+1, z in 3b+2) of the nodes and of the tet centroids
 * ((v0+v1)+(v2+v3))*0.25 over the cube [lo, lo+side), sorted by
 * (key, original index); cells level by level in ascending key prefix. */
typedef struct {
  uint64_t* node_key;    /* n_nodes, original node order            */
  uint64_t* tet_key;     /* n_tets, original tet order              */
  int64_t* node_perm;    /* n_nodes, sorted position -> node         */
  int64_t* tet_perm;     /* n_tets, sorted position -> tet           */
  int32_t* cell_level;   /* n_cells                                  */
  uint64_t* cell_prefix; /* n_cells, key >> 3*(21-level)             */
  int64_t* cell_ranges;  /* n_cells x 4: tet begin,end, node begin,end (sorted positions) */
  int64_t* cell_parent;  /* n_cells, -1 for the root                 */
  int64_t* cell_child;   /* n_cells x 2: first child, child count    */
  double* cell_centre;   /* n_cells x 3                              */
  double* cell_radius;   /* n_cells x 2: source radius, target radius */
  int64_t* m2l_off;      /* n_cells + 1, CSR by target cell          */
  int64_t* m2l_src;      /* n_m2l, ascending within a target         */
  int64_t* p2p_off;      /* n_cells + 1                              */
  int64_t* p2p_src;      /* n_p2p                                    */
} demag_tree_export;

demag_status demag_plan_export_tree(demag_plan plan, demag_tree_export* out);

/* Measured arithmetic peak of the current device, for stating roofline
 * fractions against a reproducible denominator (the paper has no counterpart):
 *   kind 0: FP64 FMA on the CUDA cores, 1: FP32 FMA on the CUDA cores,
 *   2: BF16 tcgen05.mma (M = 128, N = 256, K = 16, FP32 accumulation),
 *   3: TF32 tcgen05.mma (M = 128, N = 256, K = 8).
 * Register-resident FMA chains on every SM, or one CTA per SM issuing MMAs on
 * shared-memory operands; 2 flops per multiply-add; best of three timed runs
 * after a warm-up (CUDA events, a private stream).  *tflops receives TFLOP/s.
 * Synchronous; takes up to a second.
 * Errors: DEMAG_ERR_INVALID_ARG, DEMAG_ERR_CUDA, DEMAG_ERR_TIMEOUT. */
demag_status demag_measure_peak(int kind, double* tflops);

const char* demag_status_string(demag_status s);
/* Message of the last failing call on this thread ("" if none). */
const char* demag_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
