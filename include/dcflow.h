/*
 * dcflow: batched DC loadflow over many grid topologies on one NVIDIA B300.
 *
 * Method: "Accelerated DC loadflow solver for topology optimization"
 * (arXiv 2501.17529).  The reduced susceptance matrix of the base grid is
 * factored once (Sec. II, Def. 2, Eq. (1)); every topology (bus splits, the
 * busbar assignment t_b of Sec. III-A, and branch outages t_d) is then a
 * rank-r correction of the base branch-to-branch factors, solved with one
 * r x r FP64 system (the simultaneous form of the BSDF of Def. 5-6 / Eq. (7)
 * and of the MODF of Def. 4).  N-0 flows follow Eq. (2), the full N-1 follows
 * the LODF of Def. 3 / Eq. (5) evaluated on the updated factors, and every
 * N-1 case is reduced on the fly to the maximum relative loading (agg_m of
 * Sec. III-A), its arg-max and the overload sum, so the monitored x
 * contingency matrix is never stored.  Optional injection candidates T_i are
 * brute-forced per topology and timestep (Eq. (8), metric-first mode of
 * Sec. III-C).
 *
 * Conventions for every entry point:
 *  - returns DCFLOW_OK (0) or a negative DCFLOW_ERR_* code; no C++ exception
 *    crosses this interface; dcflow_last_error() gives a message for the
 *    calling thread's last failure;
 *  - "host" pointers are read during the call and may be freed afterwards;
 *    "device" pointers are CUDA device memory owned by the caller, read or
 *    written asynchronously on the given stream;
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *  - one context must not be used from two host threads at the same time.
 */
#ifndef DCFLOW_H
#define DCFLOW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dcflow_ctx dcflow_ctx;

enum {
  DCFLOW_OK = 0,
  DCFLOW_ERR_INVALID_ARG = -1,      /* bad size, index, pointer or option */
  DCFLOW_ERR_GRID_DISCONNECTED = -2,/* base grid not connected (setup) */
  DCFLOW_ERR_OOM = -3,              /* device allocation failed */
  DCFLOW_ERR_CUDA = -4,             /* a CUDA call failed */
  DCFLOW_ERR_TIMEOUT = -5,          /* a bounded device wait expired */
  DCFLOW_ERR_NO_STUDY = -6,         /* dcflow_solve_batch before dcflow_set_study */
  DCFLOW_ERR_SINGULAR = -7          /* base factorisation lost positive definiteness */
};

/* Arithmetic form of the per-topology contractions and the N-1 reduction.
 * The base factorisation, the r x r update systems and the N-1 denominators
 * 1 - Phi_f[c,c] are FP64 in every form. */
enum {
  DCFLOW_FP64 = 0,  /* everything FP64 */
  DCFLOW_FP32 = 1,  /* N-0 / N-1 contractions and reductions in FP32 */
  DCFLOW_BF16X3 = 2 /* as FP32, with the rank-r LODF update of every N-1 tile,
                       Phi_f = Phi - Z Vt (Def. 3 / Eq. (5) on the topology of
                       Eq. (7)), on the tensor cores: each operand split into
                       BF16 hi + lo, three products hi.hi + hi.lo + lo.hi
                       accumulated in FP32 (about 2^-16 relative per product).
                       Passes with one timestep keep the FP32 build. */
};

typedef struct {
  int32_t precision;     /* DCFLOW_FP64, DCFLOW_FP32 or DCFLOW_BF16X3 */
  int32_t device;        /* CUDA device ordinal; -1 = the current device */
  int32_t chunk_topo;    /* topologies per internal chunk; 0 = automatic */
  double island_tol;     /* pivot / denominator threshold for islanding; 0 = 1e-9 */
  int32_t compact_n1;    /* FP32 form: 0 = the N-1 kernel runs over every contingency column
                            and discards the invalid ones; 1 = over each topology's valid
                            contingencies only (compacted per topology, columns gathered from
                            the transposed factors): pays when a topology's splits island many
                            contingencies, costs about a tenth per block otherwise */
  int32_t autotune;      /* 1 = the first dcflow_solve_batch of every batch shape (timesteps,
                            candidates, extra outputs) first tunes the schedule on a prefix of
                            that batch (dcflow_autotune) and keeps the pick for the shape */
  int32_t autotune_sample; /* topologies of that prefix; 0 = 2048 */
  double tie_band;       /* worst_cont, worst_mon and best_var report the lowest position whose
                            value lies within tie_band * max(|best|, 1) of the best value (an
                            arg-max / arg-min up to the form's rounding); 0 = the form's
                            tolerance (1e-10 FP64, 1e-4 FP32 and BF16x3), < 0 = none (exact
                            ties only).  The screened solve reports the plain arg-max. */
  int32_t output_first;  /* injection candidates with top_k > 0 (Sec. III-A's injection module):
                            0 = metric-first (default): the candidates are screened on agg_m
                            alone and the top-k cases (agg_i) computed for the chosen one only;
                            1 = output-first: agg_i of every (timestep, candidate) is computed
                            inside the candidate loop and the chosen candidate's kept (needs
                            n_topo * n_time * candidates * n_cont floats of device scratch;
                            DCFLOW_ERR_OOM beyond what the device holds).  Every output is the
                            same in both modes; they differ in time. */
} dcflow_options;

/* Fill `opt` with the defaults (FP32 form, current device, automatic chunk, 1e-9,
 * every contingency column, no autotuning). */
void dcflow_default_options(dcflow_options* opt);

/*
 * Build a context for one grid and factor its reduced susceptance matrix.
 * Sec. II, Def. 1 (C_w, B = C^T diag(b) C, parallel branches add up) and
 * Def. 2 / Eq. (1) (slack removed, slack column of the PTDF zero).
 *
 * n_bus >= 2, n_branch >= 1; from/to: host int32[n_branch] bus indices
 * (from != to); b: host double[n_branch] susceptances (> 0); slack in
 * [0, n_bus).  `opt` may be NULL (defaults).  The base grid must be
 * connected (DCFLOW_ERR_GRID_DISCONNECTED otherwise).  On success *out owns
 * all device state; release it with dcflow_destroy.  Synchronous.
 */
int dcflow_setup(dcflow_ctx** out, int32_t n_bus, int32_t n_branch,
                 const int32_t* from, const int32_t* to, const double* b,
                 int32_t slack, const dcflow_options* opt);

/*
 * Rows of the base PTDF, Def. 2 / Eq. (1): out[i * n_bus + n] = PTDF[rows[i], n].
 * rows: host int32[n_rows] branch indices; out: device double[n_rows * n_bus],
 * row-major, caller-owned.  The slack column is 0.  Runs on `stream` and
 * returns after enqueueing.
 */
int dcflow_base_ptdf(dcflow_ctx* ctx, const int32_t* rows, int32_t n_rows,
                     double* out, void* stream);

/*
 * Same rows as dcflow_base_ptdf, for callers that cannot allocate device
 * memory (code running inside an arena or memory pool it does not own,
 * real-time loops that must not enter the driver allocator, hosts whose
 * allocator belongs to another framework).  The paper has no counterpart.
 *
 * It allocates nothing: its solve workspace and its device copy of `rows`
 * live in one fixed 8 MiB device array inside the library, which every GPU
 * that loads the library holds until the process exits.  A call needs
 * round_up(4 * n_rows, 256) + round_up(n_bus - 1, 64) * round_up(n_rows, 64) * 8
 * bytes of it; a larger request fails with DCFLOW_ERR_INVALID_ARG (use fewer
 * rows per call, or dcflow_base_ptdf).  Arguments, layout and ownership as for
 * dcflow_base_ptdf: rows host int32[n_rows], out device double[n_rows * n_bus]
 * row-major, caller-owned; enqueued on `stream`.
 *
 * The first call on each device looks up the array's device address (once
 * per device, with that device current); make that first call before any
 * stream capture.  Every call shares the array and it keeps the previous
 * call's contents (the workspace is cleared on each call), so calls that
 * overlap on the GPU (other streams or host threads) race: serialise them.
 */
int dcflow_base_ptdf_noalloc(dcflow_ctx* ctx, const int32_t* rows, int32_t n_rows,
                             double* out, void* stream);

/*
 * Bind the study sets that every later batch uses (PTDF row restriction of
 * Sec. II: only monitored, contingency and switching branches are needed).
 *
 * mon: host int32[n_mon] monitored branches (distinct); cont: host
 * int32[n_cont] N-1 contingency branches (distinct); limit: host
 * double[n_branch] thermal limits (> 0 on monitored branches), loading
 * rho = |flow| / limit.  split_bus: host int32[n_split_bus] substations that
 * batches may split (NULL = every bus); outage_cand: host
 * int32[n_outage_cand] branches batches may outage (NULL = every branch).
 * Only the PTDF rows of monitored, contingency, split-bus and outage-candidate
 * branches are built; a topology of a later batch that splits a bus outside
 * split_bus or takes out a branch outside outage_cand is invalid
 * (island_flag 2).
 * multi_ptr / multi_branch (optional, host): n_multi N-1 cases that take out
 * several branches at once (Def. 4, MODF; e.g. the windings of a
 * three-winding transformer), set m = multi_branch[multi_ptr[m] ..
 * multi_ptr[m + 1]), 1 to 4 distinct branches each, at most 262,140 sets.
 * Synchronous; may be called again to change the study.
 */
typedef struct {
  const int32_t* mon;  int32_t n_mon;
  const int32_t* cont; int32_t n_cont;
  const double* limit;
  const int32_t* split_bus;   int32_t n_split_bus;
  const int32_t* outage_cand; int32_t n_outage_cand;
  int32_t n_multi;
  const int32_t* multi_ptr;
  const int32_t* multi_branch;
} dcflow_study;

int dcflow_set_study(dcflow_ctx* ctx, const dcflow_study* study);

/*
 * One batch of topologies (t_b, t_d of Sec. III-A) evaluated for every
 * timestep, and optionally for every injection candidate (T_i, Eq. (8)).
 * All arrays are device memory, caller-owned, read on `stream`.
 *
 *  split_ptr  int32[n_topo+1]   CSR offsets into split_sub / split_mask
 *  split_sub  int32[]           substation (bus) split by each entry; at most
 *                               once per topology; must be a split bus of the study
 *  split_mask uint64[]          bit j = 1 moves the j-th incident branch of the
 *                               substation (ascending branch id) to the new
 *                               busbar B; a mask with an empty side is a no-op
 *  out_ptr    int32[n_topo+1]   CSR offsets into out_branch
 *  out_branch int32[]           outaged branches (t_d), distinct per topology;
 *                               each must be an outage candidate of the study
 *  inj        double[n_time * n_bus]  nodal injections per timestep; the slack
 *                               balances them (its PTDF column is zero)
 *  var_*      optional (n_var = 0 disables): candidate u adds
 *             var_delta[k] at bus var_bus[k] for k in [var_ptr[u], var_ptr[u+1])
 *
 * Per topology, effective splits + outages <= 16 and moved + outaged branches
 * <= 256.  A topology that breaks a rule is flagged 2 (invalid) in
 * island_flag, never faulted.
 */
typedef struct {
  int32_t n_topo;
  const int32_t* split_ptr;
  const int32_t* split_sub;
  const uint64_t* split_mask;
  const int32_t* out_ptr;
  const int32_t* out_branch;
  int32_t n_time;
  const double* inj;
  int32_t n_var;
  const int32_t* var_ptr;
  const int32_t* var_bus;
  const double* var_delta;
  /* generator-failure N-1 (the "N-1 generator" case of Sec. III-A), optional:
   * generator g sits at bus gen_bus[g] (int32[n_gen]) with output gen_p[t * n_gen + g]
   * (double[n_time * n_gen]); its failure removes that injection and the slack
   * takes it up.  n_gen = 0 skips them; not with candidates or the screener. */
  int32_t n_gen;
  const int32_t* gen_bus;
  const double* gen_p;
  /* injection topologies t_i (Sec. III-A: the busbar of every injection of a
   * split substation), optional (ti_ptr = NULL disables; not with var_*,
   * generator failures, multi-outage outputs or the screener).
   *  n_inj    injections whose busbar can be chosen
   *  inj_bus  int32[n_inj]  bus of each (its power is already part of inj)
   *  inj_p    double[n_time * n_inj]  their power per timestep
   *  ti_ptr   int32[n_topo + 1]  topology tau evaluates the candidates
   *           ti_mask[ti_ptr[tau] .. ti_ptr[tau + 1]) (its set T_i)
   *  ti_mask  uint64[]  bit j moves the topology's j-th eligible injection
   *           from busbar A onto busbar B
   * A topology's eligible injections are those at the bus of one of its splits
   * with both busbars non-empty, in ascending injection index, at most 64.
   * Per (topology, timestep) the candidate with the lowest n1_max_loading wins
   * (ties: lowest index; Eq. (8) over T_i) and best_var reports its index in
   * the topology's list; every other output is that candidate's.  A topology
   * without candidates, or with a mask bit at or beyond its number of eligible
   * injections, is invalid (island_flag 2).  n_time * max_tau |T_i| <= 2^20. */
  int32_t n_inj;
  const int32_t* inj_bus;
  const double* inj_p;
  const int32_t* ti_ptr;
  const uint64_t* ti_mask;
} dcflow_batch;

/*
 * Caller-owned device outputs ([n_topo * n_time] arrays are topology-major).
 *  n0_flow        double[n_topo * n_time * n_mon] N-0 flows (Eq. (2)), or NULL
 *  n0_max_loading double[n_topo * n_time] max_l |p_n0| / limit, or NULL
 *  n1_max_loading double[n_topo * n_time] max over monitored l and valid
 *                 contingencies c of |p_n1[c][l]| / limit (agg_m)
 *  overload_sum   double[n_topo * n_time] sum of max(0, rho - 1) over the same cases
 *  worst_cont     int32[n_topo * n_time]  position in `cont` of the arg-max (ties:
 *                 lowest position), -1 if no valid contingency
 *  worst_mon      int32[n_topo * n_time]  position in `mon` of the arg-max (ties:
 *                 lowest), -1 if none, or NULL
 *  best_var       int32[n_topo * n_time]  chosen candidate (argmin of n1_max_loading,
 *                 ties to the lowest index; for injection topologies the index in
 *                 the topology's own list), or NULL; -1 without candidates
 *  island_flag    uint8[n_topo]  0 ok, 1 the topology islands (outputs zero / -1),
 *                 2 invalid topology input
 *  n_island_cont  int32[n_topo]  contingencies skipped because they island
 *  n1_cont_max    float[n_topo * n_time * n_cont] max over monitored l of |p_n1[c][l]| /
 *                 limit for every contingency c (-1 where c is skipped or the topology
 *                 islands), or NULL: the per-contingency summary that labels the
 *                 learned screener
 *  top_k, top_cont, top_mon, top_loading   sparse worst results (agg_i of
 *                 Sec. III-A): per (topology, timestep) the top_k N-1 cases with the
 *                 highest maximum loading, each with its most loaded monitored
 *                 branch (the top 1 inside every case, then the top k over the cases;
 *                 ties to the lower contingency / monitored position), in
 *                 descending order: int32 positions in `cont` and `mon` and float
 *                 loadings [n_topo * n_time * top_k]; -1 / -1 / 0 beyond the valid
 *                 cases.  top_k = 0 (or NULL arrays) skips them; 1 <= top_k <= 64;
 *                 not available with the screened solve.
 * Outaged monitored branches load 0; outaged contingencies are skipped.
 */
typedef struct {
  double* n0_flow;
  double* n0_max_loading;
  double* n1_max_loading;
  double* overload_sum;
  int32_t* worst_cont;
  int32_t* worst_mon;
  int32_t* best_var;
  uint8_t* island_flag;
  int32_t* n_island_cont;
  float* n1_cont_max;
  int32_t top_k;
  int32_t* top_cont;
  int32_t* top_mon;
  float* top_loading;
  double* gen_max_loading;   /* [n_topo * n_time] max over generators g and monitored l of
                                |p_f[l] - P_g PTDF_f[l, bus_g]| / limit (with n_gen > 0) */
  int32_t* worst_gen;        /* [n_topo * n_time] the generator reaching it (lowest on ties), -1 if none */
  double* gen_overload_sum;  /* [n_topo * n_time] sum of max(0, rho - 1) over the same cases */
  /* multi-outage N-1 cases of the study (Def. 4), optional (all four or none): the maximum
   * over the sets and monitored branches of |p_n1| / limit, the set reaching it (lowest
   * on ties, -1 if none), the overload sum, and per topology the sets skipped because
   * they island it (a set with a branch the topology already lost is skipped, not counted) */
  double* multi_max_loading;   /* [n_topo * n_time] */
  int32_t* worst_multi;        /* [n_topo * n_time] */
  double* multi_overload_sum;  /* [n_topo * n_time] */
  int32_t* n_island_multi;     /* [n_topo] */
} dcflow_results;

/*
 * Evaluate a batch.  Enqueues all work on `stream`; blocks the host only for
 * one small device-to-host read of the per-rank topology histogram used to
 * group topologies by rank (Sec. III-C batching without dummy padding).
 * Scratch memory is allocated on first use and kept in the context.
 */
int dcflow_solve_batch(dcflow_ctx* ctx, const dcflow_batch* batch,
                       const dcflow_results* res, void* stream);

/* Number of kernel launches issued by the last dcflow_solve_batch call. */
int64_t dcflow_last_launch_count(const dcflow_ctx* ctx);

/*
 * Schedules.  The paper batches topologies of uneven depth by padding every
 * topology to the deepest one (Sec. III-C); here the topologies of a batch are
 * grouped by rank class (modifications per topology, padded to the class
 * bound) and processed in chunks that alternate between two scratch sets, and
 * the schedule below fixes how.  No choice changes the results beyond the
 * rounding of the reduction order (the remainder choice) or the set of
 * columns computed and then discarded (compact_n1).
 */
typedef struct {
  int32_t budget_mb;      /* scratch per buffer set in MiB (default 8192); sets the topologies
                             per chunk (at most 8192; dcflow_options.chunk_topo > 0 overrides) */
  int32_t rank_bounds[3]; /* rank classes: ascending upper bounds ending with 16, unused 0,
                             e.g. {4, 8, 16}, {8, 16, 0} */
  int32_t compact_n1;     /* FP32 / BF16x3 forms: as dcflow_options.compact_n1 */
  int32_t remainder;      /* 1 = at most 4 contingencies beyond the last block of 64 are
                             evaluated by the final pass instead of a block of their own */
  float ms;               /* dcflow_autotune: measured time of one solve of the sample */
} dcflow_schedule;

/*
 * Autotuner: time candidate schedules on `sample` (a batch the caller deems
 * representative, e.g. a prefix of the real one) with CUDA events on `stream`
 * (a warm-up and the best of two solves each, coordinate descent over the
 * chunk budget, the rank classes, compact_n1 and the remainder), keep the
 * fastest for batches of the sample's shape (timesteps, candidates, extra
 * outputs), and report it in *pick (optional) and every schedule tried in
 * tried[0 .. min(*n_tried, max_tried)) (optional).  `res` receives the
 * sample's results (device buffers as for dcflow_solve_batch).  Synchronous.
 */
int dcflow_autotune(dcflow_ctx* ctx, const dcflow_batch* sample, const dcflow_results* res, void* stream,
                    dcflow_schedule* tried, int32_t max_tried, int32_t* n_tried, dcflow_schedule* pick);
/* Fix the schedule of every later solve (NULL: back to tuned / default schedules). */
int dcflow_set_schedule(dcflow_ctx* ctx, const dcflow_schedule* s);
/* The schedule the last dcflow_solve_batch used. */
int dcflow_last_schedule(const dcflow_ctx* ctx, dcflow_schedule* out);

/*
 * Kernel timing.  dcflow_profile(ctx, 1) resets the counters and makes every
 * later dcflow_solve_batch bracket each launch of the timed kernels with CUDA
 * events recorded on the stream the kernel runs on; dcflow_profile(ctx, 0)
 * stops.  dcflow_profile_read_kind synchronises on the recorded events and
 * returns the summed time in milliseconds and the number of launches of one
 * kind; dcflow_profile_read is the fused N-1 kernel's (kind DCFLOW_PROF_N1:
 * the candidate screening passes included).
 */
enum {
  DCFLOW_PROF_N1 = 0,          /* fused N-1 (full, screening and screened passes) */
  DCFLOW_PROF_MULTI = 1,       /* multi-outage rows */
  DCFLOW_PROF_MULTI_PREP = 2,  /* multi-outage per-set systems (preparation stream) */
  DCFLOW_PROF_GEN = 3,         /* generator-failure N-1 */
  DCFLOW_PROF_TOPCASES = 4,    /* the k worst N-1 cases */
  DCFLOW_PROF_EXPAND = 5       /* operands of every (timestep, candidate) */
};
int dcflow_profile(dcflow_ctx* ctx, int32_t enable);
int dcflow_profile_read(dcflow_ctx* ctx, double* n1_ms, int64_t* n1_launches);
int dcflow_profile_read_kind(dcflow_ctx* ctx, int32_t kind, double* ms, int64_t* launches);

/*
 * Tensor-core BF16 GEMM used by the learned contingency screener (the paper
 * has no learned part; this is the dense contraction of its MLP):
 * D[M x N] = A[M x K] * B[N x K]^T (+ bias[N]) (ReLU if relu != 0).
 * A, B: device bf16 (uint16 bit patterns), row-major, K-major, row pitch lda /
 * ldb elements (multiples of 8), 16-byte aligned; D: device row-major FP32
 * (out_bf16 = 0) or bf16, pitch ldd; bias: device float[N] or NULL.
 * M and N multiples of 128, K a multiple of 64.  Accumulation is FP32 in
 * tensor memory (tcgen05).  Synchronous: returns after the product is
 * complete; DCFLOW_ERR_TIMEOUT if a bounded device wait expired.
 */
int dcflow_gemm_bf16(int32_t M, int32_t N, int32_t K, const void* A, int32_t lda, const void* B, int32_t ldb,
                     const float* bias, int32_t relu, void* D, int32_t ldd, int32_t out_bf16, void* stream);

/* ------------------------------------------------------------------------
 * Learned contingency screener.  The paper has no learned part: this is a
 * filter in front of the exact N-1 of Def. 3 / Eq. (5).  A 3-layer perceptron
 * (F -> 256 -> 256 -> C, ReLU, BF16 operands on the tensor cores, FP32
 * accumulation, FP32 master weights) scores every contingency of the bound
 * study for one (topology, timestep); the screened solve evaluates, per
 * topology, only the union over its timesteps of the top_k scored
 * contingencies.
 *
 * Features of one (topology, timestep), F = M + sum of the degrees of the
 * split-capable buses: the M signed N-0 loadings p_f[l] / limit_l of the
 * monitored branches (Eq. (2) on the modified topology), then one bit per
 * incident branch of every split-capable bus (ascending bus id, then the
 * incident branches in ascending branch id, the bit order of split_mask),
 * 1 if the branch is on busbar B.  Rows are BF16 (uint16 bit patterns) with a
 * row pitch ldx >= F_pad = round_up(F, 128), ldx % 8 == 0; columns F..F_pad
 * are zero.  A topology that islands or is invalid has an all-zero row.
 *
 * Labels (dcflow_screen_labels): y[c] = 1 iff the per-contingency maximum
 * loading (n1_cont_max of the exact solve) exceeds 1 and c is among the k
 * largest of the row (ties to the lower contingency position).
 *
 * Tensors (dcflow_screen_get / _set, row-major FP32, logical shapes):
 *   0 W1 [256 x F], 1 b1 [256], 2 W2 [256 x 256], 3 b2 [256],
 *   4 W3 [C x 256], 5 b3 [C];  kind 0 parameters, 1 gradients (of the last
 *   backward pass), 2 Adam first moments, 3 Adam second moments.
 *
 * Every call returns 0 or a negative error code; the screener belongs to the
 * context (and study) it was created on and must be destroyed before it.
 * Calls on one screener must not overlap (they share its work buffers).
 * ------------------------------------------------------------------------ */
typedef struct dcflow_screen dcflow_screen;

/* New screener for ctx's current study: He-normal weights from a
 * counter-based generator seeded by `seed`, b3 at the log-odds of 64/C.
 * max_rows (multiple of 128): the largest training batch. */
int dcflow_screen_create(dcflow_ctx* ctx, int32_t max_rows, uint64_t seed, dcflow_screen** out);
void dcflow_screen_destroy(dcflow_screen* s);
/* Feature count F and its padding, hidden width, contingencies C and padding. */
int dcflow_screen_dims(const dcflow_screen* s, int32_t* F, int32_t* F_pad, int32_t* H, int32_t* C, int32_t* C_pad);
/* Feature rows of a batch: row tau * n_time + t of X (device, caller-owned,
 * n_topo * n_time rows of pitch ldx); status (device uint8[n_topo], optional):
 * 0 ok, 1 islanded, 2 invalid.  The batch must carry no injection candidates. */
int dcflow_screen_features(dcflow_ctx* ctx, const dcflow_screen* s, const dcflow_batch* batch, void* X, int64_t ldx,
                           uint8_t* status, void* stream);
/* Labels from n1_cont_max rows (device float[n_rows * C]) into Y (device
 * uint8[n_rows * ldy], ldy >= C_pad for training; padding columns zero). */
int dcflow_screen_labels(dcflow_screen* s, const float* cont_max, int64_t n_rows, int32_t k, uint8_t* Y, int64_t ldy,
                         void* stream);
/* Forward and backward pass over rows[0..n) of X / Y (device int32 indices;
 * NULL: rows 0..n-1), n <= max_rows: the gradients of the mean binary
 * cross-entropy with logits over the n rows and C contingencies replace the
 * stored ones, and the loss is added to *loss (device float).  Synchronous. */
int dcflow_screen_backward(dcflow_screen* s, const void* X, int64_t ldx, const uint8_t* Y, int64_t ldy,
                           const int32_t* rows, int32_t n, float* loss, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8, bias-corrected) with the stored gradients. */
int dcflow_screen_adam(dcflow_screen* s, float lr, void* stream);
/* backward + adam without the synchronisation of dcflow_screen_backward;
 * dcflow_screen_check reports a bounded wait that expired since the last check. */
int dcflow_screen_train_step(dcflow_screen* s, const void* X, int64_t ldx, const uint8_t* Y, int64_t ldy,
                             const int32_t* rows, int32_t n, float lr, float* loss, void* stream);
int dcflow_screen_check(dcflow_screen* s, void* stream);
/* Scores (logits) of n_rows feature rows into Z (device float, pitch ldz >= C). */
int dcflow_screen_logits(dcflow_screen* s, const void* X, int64_t ldx, int64_t n_rows, float* Z, int64_t ldz,
                         void* stream);
int dcflow_screen_get(const dcflow_screen* s, int32_t tensor, int32_t kind, float* host);
int dcflow_screen_set(dcflow_screen* s, int32_t tensor, int32_t kind, const float* host);
/* Adam step counter: read (set = 0) or write (set != 0), for checkpoints. */
int dcflow_screen_adam_step(dcflow_screen* s, int64_t* t, int32_t set);

typedef struct dcflow_screen_options {
  int32_t top_k;         /* contingencies kept per (topology, timestep) */
  float fallback_logit;  /* the full N-1 of a topology runs when a k-th score exceeds this (INFINITY: never) */
  float min_prob;        /* every contingency whose predicted probability sigmoid(score) exceeds this
                            is evaluated as well, beyond the top_k (0: none): the rows the network is
                            unsure about get more */
} dcflow_screen_options;

typedef struct dcflow_screen_report {  /* device buffers, each optional */
  int32_t* n_eval;   /* [n_topo] contingencies evaluated exactly (bridges of the base grid, which
                        island every topology, are never evaluated) */
  uint8_t* fallback; /* [n_topo] 1 if the full N-1 ran */
  int32_t* pred;     /* [n_topo * n_time * top_k] the top_k per row, ascending; -1 padding (the
                        min_prob additions are not listed) */
  uint32_t* evaluated; /* [n_topo * ceil(n_cont / 32)] the evaluated set: bit c % 32 of word c / 32
                          for the contingency at position c */
} dcflow_screen_report;

/* dcflow_solve_batch with the N-1 restricted, per topology, to the union over
 * its timesteps of the top_k scored contingencies (all of them after a
 * fallback).  Results as dcflow_solve_batch, over the evaluated contingencies:
 * n1_max_loading / worst_cont / worst_mon are exact whenever the worst
 * contingency is evaluated, overload_sum counts evaluated contingencies only,
 * n1_cont_max (optional) is written for evaluated contingencies only.  No
 * injection candidates. */
int dcflow_solve_batch_screened(dcflow_ctx* ctx, const dcflow_batch* batch, const dcflow_results* results,
                                dcflow_screen* s, const dcflow_screen_options* opt, const dcflow_screen_report* report,
                                void* stream);

/* Failure-path self-test (no counterpart in the paper): one block waits on an
 * mbarrier that is never completed, with the same bounded wait (about 2 s at
 * 2 GHz) as the N-1 kernels; when the budget runs out the kernel records the
 * expiry in an error word and returns without faulting.  Returns
 * DCFLOW_ERR_TIMEOUT (the expected outcome); the context stays usable. */
int dcflow_selftest_bounded_wait(dcflow_ctx* ctx, void* stream);

void dcflow_destroy(dcflow_ctx* ctx);
const char* dcflow_strerror(int code);
const char* dcflow_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DCFLOW_H */
