/*
 * mcpd.h - C ABI of the GB300 library for coupled score-weighted Markov chain pool decoding.
 *
 * Problem (paper, Section "Knill's Method"): a pooling matrix A (m pools x n clones), observed
 * pool outcomes y, false-positive rate fp, false-negative rate fn and prior q define the posterior
 * pi(z | y) ∝ prod_i q^{z_i} (1-q)^{1-z_i} prod_j Pr{y_j | xi_j(z)}.  The library estimates
 * p_i = E_pi[Z_i] for every retained clone with the fixed-budget, completion-time-corrected
 * aggregate theta_CT of lag-1 coupled score-weighted random-scan Gibbs pairs (Algorithms 3 and 4;
 * Theorems 1 and 2) and returns a standard error per clone.
 *
 * Conventions for every call:
 *   - Return value 0 (MCPD_OK) on success, a negative MCPD_E* code otherwise; the message of the
 *     last failure on a context is available from mcpd_last_error().
 *   - Host inputs are borrowed for the duration of the call only (copied before return).
 *   - Host outputs are caller-owned arrays of the stated length.  Device outputs are caller-owned
 *     device allocations on the context's device, written on the context's stream.
 *   - Sizes are element counts unless a name says bytes.
 *   - All calls on one context are serialised on that context's stream; a context must not be
 *     used from two host threads at once.
 *   - Identical inputs and seed give bit-identical outputs whatever the GPU schedule: every random
 *     number is keyed by (seed, instance, global slot, replication, time) and every reduction is an
 *     integer sum.
 */
#ifndef MCPD_H
#define MCPD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Error codes. */
#define MCPD_OK 0
#define MCPD_EINVAL (-1)       /* an argument is out of range or inconsistent                     */
#define MCPD_ETOO_LARGE (-2)   /* a size exceeds what the kernels support (see mcpd_params)       */
#define MCPD_ENOMEM (-3)       /* a host or device allocation failed                              */
#define MCPD_ECUDA (-4)        /* a CUDA runtime call failed                                      */
#define MCPD_ESTEP_LIMIT (-5)  /* a pair reached params.step_limit without meeting; the outputs
                                  are written but must not be used                               */
#define MCPD_EOVERFLOW (-6)    /* an integer accumulator bound would be exceeded                  */

/* Site-selection schemes (Preliminaries; Section "Score-Weighted Update Gibbs Sampler"). */
#define MCPD_SCAN_SCORE 0      /* w_i = 0.5 softmax(tau_w s)_i + 0.5/n_a, the paper's weights    */
#define MCPD_SCAN_UNIFORM 1    /* w_i = 1/n_a (random update)                                    */
#define MCPD_SCAN_SYSTEMATIC 2 /* I_t = t mod n_a (Knill's systematic scan; uncoupled only)      */
#define MCPD_SCAN_CUSTOM 3     /* caller weights, each >= 0.25/n_a after normalisation           */

/* Pooling design as a clone -> pool CSR (the nonzeros of A by column).
 * clone_pools[clone_ptr[i] .. clone_ptr[i+1]) lists the pools holding clone i, strictly
 * increasing, each in [0, n_pools).  Limits of this build: n_clones <= 65535, n_pools <= 1022,
 * at most 8 pools per clone, at most 255 clones per pool; one chain's state (ceil(n_active / 32)
 * bit words and ceil((n_pools + 1) / 4) count words) at most 256 words, so that 15-bit offsets
 * address it; and, for a single instance, its tables (24 bytes per active clone) and one warp's
 * pair state within the device's shared memory per block.  MCPD_ETOO_LARGE otherwise. */
typedef struct mcpd_design {
    int32_t n_clones;          /* n */
    int32_t n_pools;           /* m */
    const int32_t *clone_ptr;  /* [n + 1], host */
    const int32_t *clone_pools;/* [clone_ptr[n]], host */
} mcpd_design;

/* Run parameters.  Zero-initialise and set what you need; -1 / 0 select the defaults noted. */
typedef struct mcpd_params {
    double fp, fn, prior_q;    /* 0 < fp, fn, q < 1 (Assumption 1)                                 */
    int32_t n_active;          /* 0: keep all clones; else keep the top n_active by the naive
                                  log score eta_i (ties to the lower index), others fixed to 0    */
    int32_t scan;              /* MCPD_SCAN_*                                                     */
    int32_t coupled;           /* 1: Algorithms 3-4 (coupled pairs, unbiased); 0: Algorithms 1-2
                                  (one chain per replication, burn-in average)                    */
    int32_t lanes_per_pair;    /* 0: automatic; 1: one thread per pair (the only layout of this
                                  build)                                                          */
    const double *scan_weights;   /* MCPD_SCAN_CUSTOM: [n_active] positive weights, host          */
    const double *init_marginals; /* NULL: Z_0 = 0 (all negative); else [n_active] in [0,1], host:
                                  Z_0 ~ prod_i Bernoulli(nu_i)                                    */
    int64_t k, ell;            /* coupled averaging window k:l, 0 <= k <= l; -1: one sweep,
                                  l = n_a, k = round_half_even(0.1 n_a) + 1                        */
    int64_t burn, length;      /* uncoupled: average X_b .. X_{b+T-1}; -1: b = round(0.1 n_a),
                                  T = n_a - b                                                    */
    int64_t slots;             /* P logical slots (>= 1)                                          */
    int64_t horizon;           /* B, progress units per slot (one progress unit = one shared draw
                                  (I_t, U_t)); used when budget_site_updates <= 0                 */
    double budget_site_updates;/* > 0: B = floor(budget / (2 P)) coupled, floor(budget / P)
                                  uncoupled                                                       */
    int64_t step_limit;        /* safety limit on one replication's length; 0: 10^4 n_a           */
    uint64_t seed;
    uint32_t instance_id;      /* < 2^24, enters every random-number counter                      */
    int32_t record_slots;      /* 1: keep per-slot N*_p, retained cost and replication counts     */
    int64_t slot_offset;       /* global id of slot 0 (partitioning slots across calls or GPUs)   */
    int64_t trace_stride;      /* > 0: keep the G vector of every slot p with p % stride == 0     */
    int64_t tau_audit;         /* > 0 (coupled): count completed replications whose meeting time
                                  tau exceeds this many progress units, the pairs a finite meeting
                                  cap at that length would have stopped (the run stays uncapped)  */
    int64_t meeting_cap;       /* > 0 (coupled, >= max(l, 1)): the finite meeting cap of the
                                  paper's runs.  A pair that has not met when its clock t reaches
                                  the cap stops there and is kept as completed at C = cap, every
                                  inner sum of its H_{k:l} cut at C (terms X_{r+s} - Y_{r+s-1}
                                  with r + s <= C).  The cap replaces step_limit; tau_audit
                                  defaults to the cap, so tau_over_audit counts the capped pairs
                                  (tau_audit, if set, must not exceed the cap).  0: uncapped      */
    int64_t lag;               /* coupled lag L (0 or 1: the paper's one-lag pair).  L > 1: the
                                  lag-L pair of Jacob, O'Leary and Atchade (2020): L pre-lag
                                  updates of X alone, then (I_t, U_t) moves X_{t+1} and Y_{t+1-L};
                                  tau = inf{t >= L : X_t = Y_{t-L}} and
                                  H_r = X_r + sum_{j>=1} (X_{r+jL} - Y_{r+(j-1)L}).  Every
                                  replication costs max(l, tau) >= max(l, L).  At most 2^20      */
    int64_t trace_steps;       /* > 0 (trace_stride > 0): also record, for the first
                                  trace_reps replications of every traced slot, the meeting time,
                                  the completion time and, for the first trace_steps draws, the
                                  site and which chains flipped (MCPD_FETCH_TRACE_REC).  Runs that
                                  set it launch a recording variant of the sampler; at most 2^20   */
    int64_t trace_reps;        /* replications recorded per traced slot (0: 8); at most 1024      */
} mcpd_params;

/* Counters of one run.  site_updates, reps_started, reps_retained and tau_over_audit are -1 if a
 * pair ran 2^32 or more progress units in one launch (this build keeps them in 32-bit halves). */
typedef struct mcpd_stats {
    int64_t progress_units;    /* shared draws executed, aborted replications included            */
    int64_t site_updates;      /* single-site updates executed (2 per coupled draw but the L
                                  pre-lag ones of each replication, 1 per uncoupled draw)         */
    int64_t reps_started, reps_retained, reps_aborted;
    int64_t zero_completion_slots;  /* slots with N_p(B) = 0 (first replication kept)             */
    int64_t step_limit_hits;
    int64_t max_tau, sum_tau;  /* meeting times of completed replications                         */
    int64_t n_buckets;         /* number of N*_p values the integer sums are kept for             */
    int64_t n_active;
    double kernel_ms;          /* device time of the sampling kernel (CUDA events)                */
    int64_t tau_over_audit;    /* completed replications with tau > params.tau_audit             */
    int64_t resident_pairs;    /* pairs the sampling kernel held at once (grid x block; the widest
                                  size class of a batch)                                         */
    int64_t h2d_bytes, d2h_bytes; /* single instance: bytes the library copied host -> device and
                                  device -> host for this plan so far (tables at creation; counters
                                  at each collect; fetches; mcpd_decode adds its est/se copies);
                                  0 for batches and mcpd_decode_noalloc                          */
} mcpd_stats;

typedef struct mcpd_ctx mcpd_ctx;
typedef struct mcpd_plan mcpd_plan;

/* Create a context on CUDA device `device` that issues all work on `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream).  The context owns the device scratch memory of its plans. */
int mcpd_ctx_create(int device, void *cuda_stream, mcpd_ctx **out);
/* Free the context.  Plans and batches made with it may be destroyed before or after it; any other
 * call on them needs a live context. */
void mcpd_ctx_destroy(mcpd_ctx *ctx);
/* Message of the last failing call made with ctx; owned by ctx, valid until its next call. */
const char *mcpd_last_error(const mcpd_ctx *ctx);

/* Build a plan: validate the inputs, compute the naive scores and pruning (Section "Knill's
 * Method"), the score weights and their integer alias table (Section "Score-Weighted Update Gibbs
 * Sampler"), the acceptance thresholds of the full conditional, and upload them with the device
 * scratch (per-pair accumulators, N*_p buckets).  y: [n_pools] 0/1 bytes, host. */
int mcpd_plan_create(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                     const mcpd_params *params, mcpd_plan **out);
void mcpd_plan_destroy(mcpd_plan *plan);

/* Plan facts: info[0] n_active, [1] n_buckets, [2] horizon B, [3] k (burn b uncoupled),
 * [4] l (b + T - 1 uncoupled), [5] L (window length), [6] slots P, [7] warps per block,
 * [8] resident pairs, [9] shared-memory bytes per block, [10] lanes per pair. */
int mcpd_plan_info(const mcpd_plan *plan, int64_t info[16]);
/* active[a] = original index of the a-th retained clone (ascending). */
int mcpd_plan_active(const mcpd_plan *plan, int32_t *active);

/* Run the sampler (Algorithms 3/4, or 1/2 when uncoupled) and finalize on the device.
 * est_dev, se_dev: device arrays [n_active] (active order) receiving theta_CT and its standard
 * error.  Asynchronous: returns after enqueueing on the context stream. */
int mcpd_run_async(mcpd_ctx *ctx, mcpd_plan *plan, double *est_dev, double *se_dev);
/* Run the sampler over `slots` slots (Algorithm 4 per slot) and finalize, like mcpd_run_async but
 * with a slot count of the caller's choosing, so that a fixed-budget estimate can be extended
 * until it reaches a precision.  accumulate = 0: the N*_p buckets are cleared and the slots are
 * global ids slot_offset .. slot_offset + slots - 1.  accumulate = 1: the slots continue those
 * already in the buckets since the last accumulate = 0 run (S of them: global ids
 * slot_offset + S .. slot_offset + S + slots - 1) and their sums are added.  est_dev / se_dev
 * receive theta_CT and its standard error over all S + slots slots (Theorem 2: the slot means are
 * i.i.d., so the estimator over more slots is the same estimator with a larger P).  Every slot
 * keeps the plan's horizon B, so the result is bit-identical to one mcpd_run_async of a plan with
 * P = S + slots and horizon B.  The launch keeps the plan's grid with its warps per block trimmed
 * to whole rounds of these slots.  S + slots <= 2^31 and slot_offset + S + slots <= 2^32;
 * per-slot records and traces (record_slots, trace_stride) allow only accumulate = 0 with
 * slots <= the plan's P.  Asynchronous; mcpd_collect reads this run's counters and kernel time. */
int mcpd_run_slots_async(mcpd_ctx *ctx, mcpd_plan *plan, int64_t slots, int32_t accumulate,
                         double *est_dev, double *se_dev);
/* Wait for the last run of `plan`, read its counters and its error flag.  Returns
 * MCPD_ESTEP_LIMIT if any pair hit the safety limit. stats may be NULL. */
int mcpd_collect(mcpd_ctx *ctx, mcpd_plan *plan, mcpd_stats *stats);

/* Fetch results of the last run to host memory: what = MCPD_FETCH_*; bytes must equal the size
 * the plan reports for it (mcpd_fetch_bytes). */
#define MCPD_FETCH_S1 0        /* int64  [n_buckets][n_active]: sum of G_pj over slots with N*_p = n */
#define MCPD_FETCH_S2_LO 1     /* uint64 [n_buckets][n_active]: low words of sum of G_pj^2          */
#define MCPD_FETCH_S2_HI 2     /* uint64 [n_buckets][n_active]: high words                         */
#define MCPD_FETCH_COUNT 3     /* int64  [n_buckets]: slots per N*_p value                          */
#define MCPD_FETCH_SLOT_NSTAR 4/* int32  [slots] (record_slots = 1)                                 */
#define MCPD_FETCH_SLOT_S 5    /* int64  [slots] retained progress units (record_slots = 1)         */
#define MCPD_FETCH_SLOT_REPS 6 /* int32  [slots] replications started (record_slots = 1)            */
#define MCPD_FETCH_TRACE_G 7   /* int64  [ceil(slots/stride)][n_active] (trace_stride > 0)          */
#define MCPD_FETCH_TRACE_REC 8 /* int32  [ceil(slots/stride)][trace_reps][4 + trace_steps]
                                  (trace_steps > 0): per replication r of traced slot p: [0] its
                                  meeting time tau (0: stopped unmet at the meeting cap, or an
                                  uncoupled chain), [1] its
                                  completion time C (or the clock when it was stopped), [2] 1
                                  completed, 2 stopped as doomed (Algorithm 4: it could not finish
                                  within the horizon), 3 step limit, 0 not started; [3] r; then for
                                  draw t < min(C, trace_steps): the site I_t | X flipped << 16 |
                                  Y flipped << 17 (the chain that draw t moves: X_{t+1} and, from
                                  t = L on, Y_{t+1-L}; an uncoupled run has X only)              */
size_t mcpd_fetch_bytes(const mcpd_plan *plan, int what);
int mcpd_fetch(mcpd_ctx *ctx, const mcpd_plan *plan, int what, void *host_dst, size_t bytes);

/* One call from host arrays to host arrays: plan, run, copy back, destroy the plan.
 * est, se: [n_clones] in the original clone order (pruned clones get 0 and 0);
 * active: [n_clones] 1 for retained clones, or NULL.  stats may be NULL.  Synchronous. */
int mcpd_decode(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                const mcpd_params *params, double *est, double *se, int32_t *active,
                mcpd_stats *stats);

/* Host only (no GPU needed): validate the inputs and build the plan's tables without uploading
 * them, for inspection and tests.  info as mcpd_plan_info (launch-shape entries 7-11 are 0);
 * active [n_active] original clone ids; w [n_active] scan weights; alias [n_active] words
 * (prob | alias << 32); T [81] acceptance thresholds indexed 9 n+ + n-.  Any output may be NULL;
 * the caller sizes them from a first call with all outputs NULL but info. */
int mcpd_inspect(const mcpd_design *design, const uint8_t *y, const mcpd_params *params,
                 int64_t info[16], int32_t *active, double *w, uint64_t *alias, uint64_t *T);

/* ---- Batched decoding: many instances of uneven size in one persistent launch ----------------
 * Each instance i is its own problem (design, y, params[i]: rates, prior, window, slots P_i,
 * horizon B_i, seed, instance_id) with its own theta_CT and standard errors; the instances share
 * one launch of the sampling kernel, which hands out (instance, slot) work items instance-major
 * from one device counter and reads each instance's tables through the read-only cache.  All
 * instances must agree on `coupled` and on whether the scan is systematic; record_slots and
 * trace_stride must be 0.  Outputs are concatenated in input order: instance i owns entries
 * offsets[i] .. offsets[i+1]-1 of est / se (its retained clones, ascending original index). */
typedef struct mcpd_batch mcpd_batch;

/* Build the batch.  designs, ys, params: [n_inst] host arrays (borrowed).  order_mode bits 0-7:
 * 0 keeps the instances in input order in the work list, 1 puts the instances with the longest
 * slots (largest horizon) first.  Bits 8-15: size classes, 0 for automatic, else 1..8.  The
 * instances are sorted by pair state (largest first) and cut into classes of about equal work
 * (slots x slot length); each class is its own launch of the sampling kernel, with a launch shape
 * fitted to its largest pair state, on its own stream forked from the context's stream (the
 * classes run concurrently; the finalize waits for all).  A fixed number cuts all instances
 * together.  Automatic takes as many classes as the total slots fill whole launches (at most
 * four) and, in a coupled batch, first groups the instances whose clones all sit in the same
 * number of pools (3 to 8) by that number, the others together, and cuts each group by size
 * into that many classes (at most one per instance), so that every class of a degree launches the
 * build compiled for it.  Results do not depend on the order or the classes. */
int mcpd_batch_create(mcpd_ctx *ctx, int32_t n_inst, const mcpd_design *designs,
                      const uint8_t *const *ys, const mcpd_params *params, int32_t order_mode,
                      mcpd_batch **out);
void mcpd_batch_destroy(mcpd_batch *batch);
/* The classes mcpd_batch_create would form, computed on the host (no device, no context):
 * class_of[n_inst] (caller-owned) receives each instance's class, numbered 0, 1, ... in launch
 * order, and *n_classes their number, for a GPU with sm_count multiprocessors (the automatic
 * class count depends on it).  The same validation of the inputs as mcpd_batch_create. */
int mcpd_batch_classes(int32_t n_inst, const mcpd_design *designs, const uint8_t *const *ys,
                       const mcpd_params *params, int32_t order_mode, int32_t sm_count,
                       int32_t *class_of, int32_t *n_classes);
/* info[0] total retained clones, [1] instances, [2] total slots, [3] largest n_active,
 * [4] warps per block, [5] blocks and [7] shared-memory bytes per block of the first class (the
 * largest pair state of its degree group), [6] resident pairs of the widest class, [8] lanes
 * per pair, [9] size
 * classes, [10] largest warps per block over the classes, [11] classes that launch the kernel
 * variant with meeting caps and lags > 1, [12] classes that launch a build with a compile-time
 * degree (coupled classes whose instances all sit in the same number of pools per clone, 3 to 8;
 * thresholds indexed by the mask of deciding pools up to 6). */
int mcpd_batch_info(const mcpd_batch *batch, int64_t info[16]);
/* offsets: [n_inst + 1] host array receiving each instance's first output index. */
int mcpd_batch_offsets(const mcpd_batch *batch, int64_t *offsets);
/* Choose the launch shape of every class: lanes per pair (1: one thread per pair; 8, 16 or 32: a
 * lane group per pair, coupled batches only; all give identical results) and at most
 * warps_per_block warps per block (0: as many as the kernel and the class's largest pair state
 * allow).  May reallocate the per-pair scratch; invalidates a captured graph. */
int mcpd_batch_set_shape(mcpd_ctx *ctx, mcpd_batch *batch, int32_t lanes_per_pair,
                         int32_t warps_per_block);
/* Enqueue one decode of every instance; est_dev, se_dev: device arrays [info[0]]. */
int mcpd_batch_run_async(mcpd_ctx *ctx, mcpd_batch *batch, double *est_dev, double *se_dev);
/* Extend the last decode of the batch, as mcpd_run_slots_async does for a plan: every instance i
 * with mask[i] != 0 (all if mask is NULL) runs its next P_i slots, the global slot ids after
 * those already in its N*_p buckets, and adds their sums; est_dev / se_dev receive every
 * instance's theta_CT and standard error over all slots in its buckets (an instance not extended
 * keeps its estimate).  For each instance the result is bit-identical to one decode over that
 * many slots with the same horizon.  Needs a previous mcpd_batch_run_async or
 * mcpd_batch_launch_graph (which start every instance again from its first slot).  Slots per
 * instance stay <= 2^31 and global slot ids < 2^32.  Asynchronous; mcpd_batch_collect reads this
 * extension's counters and kernel time. */
int mcpd_batch_extend_async(mcpd_ctx *ctx, mcpd_batch *batch, const int32_t *mask, double *est_dev,
                            double *se_dev);
/* Capture one decode (scratch clears, sampling kernel, finalize) into a CUDA graph on the
 * context's stream (which must not be the legacy default stream); replay it with
 * mcpd_batch_launch_graph. */
int mcpd_batch_capture_graph(mcpd_ctx *ctx, mcpd_batch *batch, double *est_dev, double *se_dev);
int mcpd_batch_launch_graph(mcpd_ctx *ctx, mcpd_batch *batch);
/* Wait for the last decode and read its counters (summed over instances). */
int mcpd_batch_collect(mcpd_ctx *ctx, mcpd_batch *batch, mcpd_stats *stats);
/* One instance's integer bucket sums (MCPD_FETCH_S1, _S2_LO, _S2_HI, _COUNT), sized as for a
 * plan of that instance alone. */
int mcpd_batch_fetch(mcpd_ctx *ctx, const mcpd_batch *batch, int32_t inst, int what,
                     void *host_dst, size_t bytes);
/* Autotuner: time each candidate shape (cand_lanes[c] lanes per pair, cand_warps[c] warps per
 * block; reps timed decodes after one warm-up each) and keep the fastest; best_index receives its
 * index, times[c] candidate c's mean milliseconds (-1 if it does not fit).  Runs that stop a
 * pair at its step limit still count as timings. */
int mcpd_batch_autotune(mcpd_ctx *ctx, mcpd_batch *batch, const int32_t *cand_lanes,
                        const int32_t *cand_warps, int32_t n_cand, int32_t reps, double *est_dev,
                        double *se_dev, int32_t *best_index, double *times);

/* ---- Learned scan weights and initial marginals ----------------------------------------------
 * Not in the paper, which proves that any fixed positive scan weights keep pi invariant
 * (Proposition 1) and that the coupled estimator is unbiased from any initial distribution
 * (Theorem 1).  These calls compute 16 per-clone features of a design, run a 16-64-64-2 MLP
 * (ReLU; parameters stored as bf16, arithmetic in fp32) and train it with Adam; its two heads give
 * scan weights w = 0.5 softmax(o_1) + 0.5/n per instance and initial marginals
 * nu = clamp(sigmoid(o_2), 1e-6, 1 - 1e-6), which mcpd_params.scan_weights / init_marginals
 * accept.  Parameter layout (mcpd_mlp_num_params() = 5378 values): W1 [64][16], b1 [64],
 * W2 [64][64], b2 [64], W3 [2][64], b3 [2].  All arrays are device arrays; work is enqueued on the
 * context's stream (mcpd_features_batch synchronises). */
int mcpd_mlp_num_params(void);
/* Features of every clone of every instance (no pruning), rows concatenated in instance order.
 * rates: [n_inst][3] host (fp, fn, prior_q); feat_dev: [sum n_clones][16] float.  Temporary
 * device buffers are allocated and freed inside. */
int mcpd_features_batch(mcpd_ctx *ctx, int32_t n_inst, const mcpd_design *designs,
                        const uint8_t *const *ys, const double *rates, float *feat_dev);
/* Out[r][2] = MLP(X[r][16]) for n_rows rows; W: [5378] bf16 bit patterns. */
int mcpd_mlp_forward(mcpd_ctx *ctx, int64_t n_rows, const float *X, const uint16_t *W, float *Out);
/* Per segment s (rows seg[s] .. seg[s+1]-1, one instance): loss_seg[s] = (cross-entropy of
 * softmax(o_1) to target_w + mean binary cross-entropy of sigmoid(o_2) to target_p) / n_seg and
 * dOut = its gradient.  seg_dev: [n_seg + 1] int64; loss_seg_dev: [n_seg] double. */
int mcpd_mlp_loss(mcpd_ctx *ctx, int32_t n_seg, const int64_t *seg_dev, const float *Out,
                  const float *target_w, const float *target_p, float *dOut, double *loss_seg_dev);
/* grad[5378] = gradient of sum(dOut * Out) with respect to the parameters (activations recomputed;
 * the row sum is taken in fixed chunks, so it is reproducible).  work: float workspace of at least
 * mcpd_mlp_backward_workspace(n_rows) values. */
int mcpd_mlp_backward(mcpd_ctx *ctx, int64_t n_rows, const float *X, const uint16_t *W,
                      const float *dOut, float *work, int64_t work_floats, float *grad);
int64_t mcpd_mlp_backward_workspace(int64_t n_rows);
/* One Adam step (step >= 1) on the fp32 master parameters; W receives them rounded to bf16. */
int mcpd_mlp_adam(mcpd_ctx *ctx, int32_t step, float lr, float beta1, float beta2, float eps,
                  float *master, float *m, float *v, const float *grad, uint16_t *W);
/* W = bf16(master), round to nearest even. */
int mcpd_mlp_cast(mcpd_ctx *ctx, const float *master, uint16_t *W);
/* Heads per segment: w_dev, nu_dev [seg[n_seg]] doubles. */
int mcpd_mlp_heads(mcpd_ctx *ctx, int32_t n_seg, const int64_t *seg_dev, const float *Out,
                   double *w_dev, double *nu_dev);

/* Decode without any device allocation.  The paper has no counterpart: this entry point exists for
 * callers that may not call cudaMalloc or cudaFree themselves, such as a component running under
 * a host application or server that owns all device memory through its own pool allocator and
 * hands out fixed budgets, or a host loop that cannot afford the device-wide synchronisation those
 * calls can imply.  The caller passes the host inputs (as for mcpd_decode) and two device arrays
 * it owns, est_dev and se_dev, each [n_active] in active order (mcpd_inspect gives n_active and the
 * active ids).  All other device memory comes from one 64 MiB array compiled into this library,
 * held on every GPU that loads it until the process exits.  Problems whose tables, N*_p buckets
 * and one warp of pair accumulators do not fit in it fail with MCPD_ETOO_LARGE; problems that fit
 * run with as many resident pairs as fit (stats->resident_pairs) and give the same results as
 * mcpd_run_async.  record_slots and trace_stride must be 0.  est_dev and se_dev must be device
 * (or managed) memory of the context's device in the runtime's primary context, else MCPD_EINVAL.
 * Every call looks the array's address up with the context's device current (so a reset of the
 * primary context leaves no stale address); the first call on a device may load the library's
 * device code, so make it before any stream capture.  Every call clears and reuses the same array:
 * calls whose GPU work overlaps on one device race, so serialise them.  Synchronous on the
 * context's stream; stats may be NULL (kernel_ms is left 0). */
int mcpd_decode_noalloc(mcpd_ctx *ctx, const mcpd_design *design, const uint8_t *y,
                        const mcpd_params *params, double *est_dev, double *se_dev,
                        mcpd_stats *stats);

/* Philox4x32-10 blocks computed by the device generator the sampler uses: out[4 i .. 4 i + 3] =
 * Philox(ctr[4 i .. 4 i + 3], key).  ctr, out: device arrays of 4 n words. */
int mcpd_philox_device(mcpd_ctx *ctx, const uint32_t *ctr_dev, uint32_t key0, uint32_t key1,
                       uint32_t *out_dev, int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* MCPD_H */
