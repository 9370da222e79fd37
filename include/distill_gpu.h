/*
 * distill_gpu.h - C ABI of a GB300 (sm_103a) library that runs the data-parallel
 * hot path of the cognitive models compiled by Distill (arXiv 2110.15425):
 * many independent stochastic trials of a PsyNeuLink-style composition, and
 * the grid search of an optimization-control mechanism.
 *
 * The calls follow the paper's statement of the problem:
 *   - compose a model graph of nodes (mechanisms) and edges (projections)
 *     (Sec. 2.1);
 *   - run it for a number of trials, iterating each trial until its end
 *     condition (Sec. 2.2, Listing 1);
 *   - let the Control node simulate every allocation of a grid and pick the
 *     best one (Sec. 2.1, Sec. 3.6).
 * Dynamic structures become static ones with integer ids (Sec. 3.3), and the
 * sanitization run of Sec. 2.2 becomes compose-time shape validation.
 *
 * Conventions (every entry point):
 *   - Returns dg_status; nothing throws across the ABI. On an error the
 *     outputs are left unwritten and dg_last_error() describes the failure.
 *   - "device" pointers are CUDA global-memory addresses (e.g. a torch
 *     tensor's data_ptr()); "host" pointers are ordinary CPU memory.
 *   - Inputs and outputs are owned by the caller. A model owns the device
 *     copies of its weights from dg_compose until dg_model_free.
 *   - Work on a `stream` (a cudaStream_t, NULL = legacy default stream) is
 *     asynchronous and ordered on that stream; outputs are valid once the
 *     stream has reached that point.
 *   - Random draws: Philox4x32-10 keyed by (seed lo, seed hi) with counter
 *     (trial, candidate, block, 0). Normal d of a (trial, candidate) stream
 *     is lane d&3 of the Box-Muller output of block d>>2; the uniform of word
 *     w is ((w >> 9) + 1/2) 2^-23. Results depend only on (inputs, seed), never
 *     on launch shape, so any trial can be replayed alone.
 */
#ifndef DISTILL_GPU_H
#define DISTILL_GPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_E_ARG = -1,          /* null pointer, bad enum value, size out of range */
  DG_E_SHAPE = -2,        /* model graph or sizes fail compose-time validation */
  DG_E_BUDGET = -3,       /* request larger than the context's HBM budget */
  DG_E_CUDA = -4,         /* a CUDA call failed (message has the CUDA error) */
  DG_E_TIMEOUT = -5,      /* dg_wait ran out of time, or a device wait gave up */
  DG_E_UNSUPPORTED = -6,  /* valid graph that no kernel implements */
  DG_E_STATE = -7         /* call not valid in the object's current state */
} dg_status;

typedef enum {
  DG_INPUT = 0,             /* clamped input layer: y = the trial's input values */
  DG_TRANSFER_LOGISTIC = 1, /* time-averaging logistic layer (Sec. 2.1, 5 Stroop) */
  DG_DDM = 2,               /* drift-diffusion integrator (Sec. 4.4) */
  DG_LCA = 3,               /* leaky competing accumulator (Sec. 4.4, 5 Multitasking) */
  DG_PP_OBSERVE = 4,        /* Obs nodes: noisy view of 3 entity positions (Sec. 2.1) */
  DG_PP_ACTION = 5,         /* Action node: one unit step (Sec. 2.1) */
  DG_PP_OBJECTIVE = 6       /* Objective node: -distance to prey - allocation cost (Sec. 2.1) */
} dg_mech_kind;

/* dg_mechanism.flags (DG_LCA only) */
#define DG_LCA_NO_RECTIFY 1 /* do not clamp accumulators at 0 */
#define DG_LCA_TWO_SIDED 2  /* size 1 only: stop at |x| >= threshold, choice = (x > 0) */

/* dg_projection.dtype: precision of the device copy of the weights */
#define DG_F32 0
#define DG_BF16 1 /* round-to-nearest-even bfloat16; only the wide hidden->response edge */

/* dg_run_desc.mode */
#define DG_MODE_BATCHED 0 /* persistent kernel, trials refilled as others finish, autotuned */
#define DG_MODE_PLAIN 1   /* one thread per trial, one launch, no refill (comparison form) */

/* dg_grid_desc.tie_break: which of several exactly equal best means is chosen */
#define DG_TIE_LOWEST 0    /* the lowest candidate index */
#define DG_TIE_RESERVOIR 1 /* uniformly at random by reservoir sampling (Sec. 3.3), see
                              dg_argmax_f64_reservoir */

typedef struct {
  int32_t kind;       /* dg_mech_kind */
  int32_t size;       /* number of units */
  double gain, bias;  /* TRANSFER_LOGISTIC: y = 1 / (1 + exp(-gain (s + bias))) */
  double rate;        /* TRANSFER_LOGISTIC: s <- (1 - rate) s + rate net + noise eps */
  double noise;       /* TRANSFER_LOGISTIC: sd added to s each step;
                         DDM, LCA: sigma, scaled by sqrt(dt) */
  double dt;          /* DDM, LCA: Euler step */
  double leak;        /* LCA: k */
  double inhibition;  /* LCA: beta (lateral inhibition) */
  double start;       /* DDM: x0 */
  double offset;      /* PP_OBSERVE: perception sd = 1 / (offset + allocation) */
  double weight;      /* PP_ACTION: act = unit(unit(prey - player) - weight unit(predator - player)) */
  int32_t flags;      /* DG_LCA_* */
  int32_t reserved;
  double threshold;   /* DDM node of a TRANSFER graph: bound z (> 0) */
  int32_t max_steps;  /* DDM node of a TRANSFER graph: steps at most (>= 1) */
  int32_t reserved2;
} dg_mechanism;

typedef struct {
  int32_t sender;        /* index into the mechanism array */
  int32_t receiver;
  const float* weights;  /* host, FP32 [receiver size][sender size] row-major; copied at compose.
                            NULL with lo < hi: drawn from the compose call's weight_seed, see
                            dg_compose; NULL with lo = hi = 0: the graph's structural edge
                            (identity, predator-prey chain) */
  int32_t dtype;         /* DG_F32 or DG_BF16 */
  int32_t reserved;
  double lo, hi;         /* range of seeded weights (weights NULL) */
} dg_projection;

typedef struct {
  int32_t mech;          /* mechanism whose outputs decide the end of a trial */
  int32_t max_steps;     /* iterations per trial at most (>= 1) */
  double threshold;      /* LCA: max_i x_i >= threshold; TRANSFER: top1 - top2 > threshold;
                            DDM: unused (per-trial threshold) */
} dg_stop;

typedef struct dg_ctx dg_ctx;
typedef struct dg_model dg_model;

/* Per-trial work of dg_run. */
typedef struct {
  int64_t n_trials;           /* >= 0; at most 2^31 - 1 */
  int64_t trial_offset;       /* global id of trial 0 of this call (>= 0, offset + n_trials
                                 <= 2^32): the random stream and the condition of local trial t
                                 are those of trial offset + t, so a job split across calls or
                                 GPUs, or resumed at any trial, reproduces the whole job */
  uint64_t seed;              /* Philox key */
  const float* trial_params;  /* device. DDM: [2][n_trials] (row 0 drift A, row 1 threshold z);
                                 LCA: [n_trials][N] inputs I; TRANSFER: unused (NULL) */
  const float* cond_inputs;   /* device. TRANSFER: [n_cond][input units of all DG_INPUT
                                 layers in mechanism order]; else unused */
  int32_t n_cond;             /* TRANSFER: global trial g takes condition (g / cond_block) % n_cond */
  int32_t cond_block;
  int32_t mode;               /* DG_MODE_* */
  int32_t reserved;
} dg_run_desc;

/* Control grid of dg_grid_search (predator-prey models). */
typedef struct {
  int32_t n_levels[3];        /* levels per control signal (player, predator, prey) */
  int32_t n_trials;           /* noisy trials per candidate, 1 .. 1024 */
  const float* levels[3];     /* device, allocation values of each signal */
  const float* positions;     /* device, [n_trials][6]: player xy, predator xy, prey xy */
  uint64_t seed;
  int32_t mode;               /* DG_MODE_* */
  int32_t tie_break;          /* DG_TIE_*; the reservoir draws use `seed` */
  int64_t cand_begin;         /* evaluate candidates cand_begin .. cand_begin + cand_count - 1 */
  int64_t cand_count;         /* (0 = all); cand_means[i] is candidate cand_begin + i, and
                                 best_index is a global candidate index */
} dg_grid_desc;

typedef struct {
  int64_t best_index;         /* c = (l0 * L1 + l1) * L2 + l2; on exact ties as tie_break says */
  double best_value;          /* FP64 mean outcome of the best candidate */
  double runner_up_gap;       /* best_value - second best value (0 on a tie) */
} dg_grid_result;

/* ---------------------------------------------------------------- context --- */

/* Create a context on CUDA device `device`. hbm_budget_bytes bounds the device
   memory the serving loop may hold for admitted jobs (0 = 150 GB). */
dg_status dg_create(dg_ctx** out, int device, size_t hbm_budget_bytes);
dg_status dg_destroy(dg_ctx* ctx);

/* Thread-local description of the last error on the calling thread; never NULL. */
const char* dg_last_error(void);

/* Library version, e.g. "distill-gpu 0.1 sm_103a". */
const char* dg_version(void);

/* ---------------------------------------------------------------- compose --- */

/* Validate a model graph (Sec. 2.2 sanitization) and lay it out statically
   (Sec. 3.3). Recognised graphs:
     - DDM:      one DG_DDM mechanism of size 1; no projections.
     - LCA:      one DG_LCA mechanism, size 1..16 (optionally fed by one DG_INPUT of
                 the same size through an identity projection with NULL weights).
     - TRANSFER: DG_INPUT and DG_TRANSFER_LOGISTIC layers; every projection runs
                 from an earlier mechanism to a logistic layer; the stop mechanism is
                 a logistic layer of size 2..16. Extended Stroop form (Sec. 5): up to
                 8 DG_DDM units in total (any number of DDM mechanisms) fed only by
                 F32 projections from the stop layer; when the network stops, DDM
                 unit q (mechanisms in array order, units in order) integrates
                 drift_q = bias + sum_i W[q][i] y_i with its mechanism's dt, noise,
                 threshold and max_steps from 0 (start must be 0), noise stream
                 (trial, cand 1 + q). Graphs that list the same DDM units through
                 different mechanisms or projections compose to the same layout. Up to 32 logistic units run on the
                 small-network kernel; the wide form (two one-hot input layers ->
                 hidden of 64..256 units, multiple of 64 -> response of 16 units with a
                 DG_BF16 hidden->response projection) runs on the tensor-core kernel.
     - PREDATOR_PREY: DG_INPUT(6) -> DG_PP_OBSERVE(6) -> DG_PP_ACTION(2) ->
                 DG_PP_OBJECTIVE(1), chained by projections with NULL weights.
   Static read-only parameters (Sec. 3.3): a projection with NULL weights and
   lo < hi gets weights drawn from weight_seed: weight w (row-major index)
   of projection p (its index in projs) is lo + (hi - lo) u, formed in FP64
   and rounded to FP32, u = ((x >> 9) + 1/2) 2^-23 with x word (w & 3) of
   Philox4x32-10(key = (weight_seed lo, weight_seed hi), counter = (p, 0,
   w >> 2, 2)) (purpose 2 keeps these draws apart from all noise).
   Weights are copied to the device (synchronously) before return.
   Errors: DG_E_ARG (null/invalid values), DG_E_SHAPE (graph not valid),
   DG_E_UNSUPPORTED (valid but outside the kernels' limits), DG_E_CUDA. */
dg_status dg_compose(dg_ctx* ctx, const dg_mechanism* mechs, int32_t n_mech,
                     const dg_projection* projs, int32_t n_proj, const dg_stop* stop,
                     uint64_t weight_seed, dg_model** out);
dg_status dg_model_free(dg_model* model);

/* The FP32 weights a model was composed with for projection `proj` (its index
   in the compose call's projs): the given ones, or those drawn from the seed
   (before any BF16 rounding of the device copy). out: host, n floats, n =
   receiver size x sender size (0 for a structural edge).
   Errors: DG_E_ARG (proj out of range, n not the projection's size). */
dg_status dg_model_weights(const dg_model* model, int32_t proj, float* out, int64_t n);

/* Model kind (0 DDM, 1 LCA, 2 TRANSFER small, 3 TRANSFER wide, 4 PREDATOR_PREY)
   and the number of floats dg_run writes per trial into final_state. */
dg_status dg_model_info(const dg_model* model, int32_t* kind, int32_t* state_size);

/* -------------------------------------------------------------------- run --- */

/* Run desc->n_trials independent trials of a DDM, LCA or TRANSFER model, each
   until its stop condition or stop.max_steps (Sec. 2.2, Listing 1).
   Outputs (device, caller-owned, n_trials entries):
     choice: DDM 1 = upper bound, 0 = lower; LCA winner index; TRANSFER index
             of the largest stop-layer output; -1 = no decision by max_steps.
             Extended Stroop: 2 q + (upper bound) of the first DDM unit q to
             reach a bound (fewest steps, lower q on equal steps), -1 if none.
     step:   iteration at which the trial ended (1-based), max_steps on timeout.
             Extended Stroop: network steps + that unit's steps (+ the largest
             DDM max_steps if none decided).
     final_state (may be NULL): [n_trials][state_size] FP32 state at the end
             (DDM x; LCA x_0..x_{N-1}; TRANSFER stop-layer outputs; Extended
             Stroop: stop-layer outputs, then per DDM unit x, choice, steps).
   Errors: DG_E_ARG, DG_E_UNSUPPORTED (PREDATOR_PREY model), DG_E_CUDA. */
dg_status dg_run(dg_model* model, const dg_run_desc* desc, int8_t* choice, int32_t* step,
                 float* final_state, void* stream);

/* Several jobs of one DDM, LCA or small TRANSFER model (at most 8 logistic
   units, no DDM nodes) in one persistent launch: Sec. 3.6's
   parallel evaluations taken across jobs as well as within one, so that jobs
   too small to fill the GPU share its lanes and the launch's ramp and drain.
   Job i is exactly dg_run(model, &descs[i], choice[i], step[i],
   final_state ? final_state[i] : NULL): the same trials, random streams and
   results, bit for bit. Each desc is checked as dg_run checks it and must use
   DG_MODE_BATCHED; jobs may differ in n_trials (0 allowed), trial_offset, seed
   and trial_params (networks: cond_inputs, n_cond and cond_block). choice, step
   (and final_state when not NULL) are host
   arrays of n_jobs device pointers; an entry of final_state may be NULL.
   n_jobs: 1 .. 256; at most 2^31 - 1 trials in all.
   Errors: DG_E_ARG, DG_E_UNSUPPORTED (another model), DG_E_CUDA. */
dg_status dg_run_jobs(dg_model* model, int32_t n_jobs, const dg_run_desc* descs,
                      int8_t* const* choice, int32_t* const* step, float* const* final_state,
                      void* stream);

/* Predator-prey grid search (Sec. 2.1, 3.6): simulate every candidate
   allocation over desc->n_trials noisy trials, average the outcomes in FP64,
   and take the argmax. Exact ties of the best mean go to the lowest index, or
   with desc->tie_break = DG_TIE_RESERVOIR to a random one of them, drawn as
   dg_argmax_f64_reservoir does over the evaluated candidates (indices
   cand_begin ..) in order.
   result: device pointer to one dg_grid_result.
   cand_means (may be NULL): device, FP64 mean outcome per evaluated candidate
   ([cand_count], [L0 L1 L2] for the whole grid). A candidate's mean has the
   same bits whatever range of candidates a call evaluates and whatever launch
   shape the library picks, so a search split across calls or GPUs reassembles
   exactly.
   Errors: DG_E_ARG, DG_E_UNSUPPORTED (not a PREDATOR_PREY model), DG_E_CUDA. */
dg_status dg_grid_search(dg_model* model, const dg_grid_desc* desc, dg_grid_result* result,
                         double* cand_means, void* stream);

/* A batch of independent grid searches of one PREDATOR_PREY model in one
   launch: the Control node's search (Sec. 2.1) for n_searches situations at
   once, every evaluation of every search in parallel (Sec. 3.6). Search i is
   exactly dg_grid_search(model, &descs[i], &results[i], cand_means[i]): the
   same candidates, noise streams, FP64 means (bit for bit) and lowest-index
   argmax. All searches share the grid shape (n_levels) and n_trials; each has
   its own level values, positions and seed; whole grids only (cand_begin =
   cand_count = 0), DG_TIE_LOWEST, DG_MODE_BATCHED.
   descs: host array [n_searches] (device pointers inside, as for
   dg_grid_search); results: device array [n_searches]; cand_means: NULL, or a
   host array [n_searches] of device pointers ([L0 L1 L2] each, or NULL).
   n_searches 1 .. 256. The first call on a stream with a given size
   allocates scratch (not inside stream capture).
   Errors: DG_E_ARG, DG_E_UNSUPPORTED (not a PREDATOR_PREY model), DG_E_STATE
   (scratch must grow inside capture), DG_E_CUDA. */
dg_status dg_grid_search_batch(dg_model* model, int32_t n_searches, const dg_grid_desc* descs,
                               dg_grid_result* results, double* const* cand_means, void* stream);

/* Time-stepped predator-prey episodes (Sec. 2.1: the whole search over
   allocations is repeated at every time step until the prey or the player is
   caught; the positions carried between steps are the sequential state of
   Sec. 2.1 that caps the parallelism of such models). Episode e starts from
   start[e] = (player xy, predator xy, prey xy). At step t = 0, 1, ...:
     - every allocation c (layout as dg_grid_search) is simulated on n_trials
       perceptions of the current positions, noise stream (trial t n_trials + j,
       cand c) at Philox blocks 2e and 2e + 1 (e the global episode index,
       episode_offset + row); FP64 mean; best = argmax
       (lowest index on exact ties);
     - the player perceives once more with the best allocation (stream
       (trial t, cand 0xFFFFFFFF), same blocks) and moves speed[0] times the
       Action node's unit step; the predator moves speed[1] unit(P - D) toward
       the player and the prey speed[2] unit(Y - P) away from it, all from the
       positions at the start of the step. The simulations run in FP32 with
       FP64 means; this one perception and the moves are computed in FP64
       from the FP32 positions and rounded to FP32 (the positions' format);
     - then |P - Y| <= radius ends the episode with +1 (prey caught), else
       |P - D| <= radius with -1 (player caught); after max_steps steps, 0. */
typedef struct {
  int32_t n_episodes;         /* E >= 1 */
  int32_t max_steps;          /* T >= 1, with T n_trials <= 2^32 */
  int32_t n_levels[3];        /* levels per signal, 1 .. 4096 */
  int32_t n_trials;           /* perceptions per candidate and step, 1 .. 1024 */
  const float* levels[3];     /* device, allocation values of each signal */
  const float* start;         /* device, [E][6] start positions */
  uint64_t seed;
  double speed[3];            /* step lengths of player, predator, prey (>= 0) */
  double capture_radius;      /* >= 0 */
  int64_t episode_offset;     /* global index of episode 0 (its noise), >= 0; with
                                 offset + E <= 2^31 - 1 a call reproduces episodes
                                 offset .. offset + E - 1 of a larger run */
} dg_episode_desc;

/* Outputs of dg_run_episodes (device pointers, caller-owned). */
typedef struct {
  int8_t* outcome;            /* [E] +1 prey caught, -1 player caught, 0 none by T */
  int32_t* steps;             /* [E] steps taken (the capture step, or T) */
  float* final_pos;           /* [E][6] positions at the end, or NULL */
  int32_t* best;              /* [E][T] best candidate of each step, -1 after the end, or NULL */
  double* value;              /* [E][T] its FP64 mean outcome (0 after the end), or NULL */
  float* pos;                 /* [E][T][6] positions after each step (0 after the end), or NULL */
} dg_episode_out;

/* Run E episodes of a PREDATOR_PREY model side by side: 1 + T kernel launches
   (one per time step over the episodes still running), no host
   synchronisation. Episodes are independent: an episode's results depend on
   its index and start only. The first call on a stream with a given E x
   candidates size allocates scratch (not inside stream capture).
   Errors: DG_E_ARG, DG_E_UNSUPPORTED (not a PREDATOR_PREY model), DG_E_STATE
   (first use inside capture), DG_E_CUDA. */
dg_status dg_run_episodes(dg_model* model, const dg_episode_desc* desc, const dg_episode_out* out,
                          void* stream);

/* Coarse-to-fine grid search: the refinement of the attention search in
   Sec. 4.3 ("adaptive mesh refinement"), done by simulating the model instead
   of by value-range analysis. Round r = 0 .. rounds-1 lays `points` (G) levels
   on each signal's interval [lo_e, hi_e]: level l = lo + (hi - lo) l / (G - 1),
   computed in FP64 and rounded to FP32. Its G^3 candidates c = (l0 G + l1) G + l2
   are simulated and averaged exactly as dg_grid_search does, with the noise
   stream of candidate r G^3 + c, and the best one (lowest index on exact ties)
   is taken. The next interval of each signal is the best level +- one grid
   spacing (hi - lo)/(G - 1), clipped to the domain (FP64, rounded to FP32): it
   shrinks by 2/(G - 1) per round. R rounds simulate R G^3 candidates instead
   of the (G-fold finer) full grid. */
typedef struct {
  int32_t points;             /* G: levels per signal in every round, 4 .. 64 */
  int32_t rounds;             /* R >= 1, with R G^3 <= 2^32 */
  int32_t n_trials;           /* noisy trials per candidate, 1 .. 1024 */
  int32_t reserved;           /* 0 */
  float lo[3], hi[3];         /* domain of each signal (player, predator, prey); lo <= hi */
  const float* positions;     /* device, [n_trials][6] as in dg_grid_desc */
  uint64_t seed;
} dg_refine_desc;

typedef struct {
  float alloc[3];             /* allocation of the round's best candidate */
  float lo[3], hi[3];         /* the round's interval of each signal */
  int32_t round;              /* r */
  int64_t best_index;         /* (l0 G + l1) G + l2 within the round */
  double best_value;          /* FP64 mean outcome of the best candidate */
  double runner_up_gap;       /* best - second best of the round (0 on a tie) */
} dg_refine_round;

/* Run a coarse-to-fine search on a PREDATOR_PREY model. rounds: device,
   dg_refine_round[desc->rounds], written in order (entry rounds-1 holds the
   answer). Up to 8,192 candidates per round (G <= 20) the search is one
   launch of one 8-CTA thread-block cluster; larger grids take 1 + 2 R
   launches. No host synchronisation (capturable).
   Errors: DG_E_ARG (bad sizes, domain or pointers), DG_E_UNSUPPORTED (not a
   PREDATOR_PREY model), DG_E_CUDA. */
dg_status dg_grid_refine(dg_model* model, const dg_refine_desc* desc, dg_refine_round* rounds,
                         void* stream);

/* Argmax over n FP64 values (device), lowest index on exact ties, into a
   device dg_grid_result. n >= 1. */
dg_status dg_argmax_f64(dg_ctx* ctx, const double* values, int64_t n, dg_grid_result* result,
                        void* stream);

/* Argmax over n FP64 values (device) with a uniformly random choice among the
   values equal to the maximum - the reservoir sampling of Sec. 3.3 (Vitter's
   Algorithm R, reservoir of one, values visited in index order): the k-th
   value equal to the running maximum, at index i, replaces the reservoir's
   element when w k < 2^32, w = word 0 of Philox4x32-10(key = (seed lo, seed
   hi), counter = (i lo, i hi, 0, 4)); a larger value restarts the count at 1.
   The choice is deterministic for a seed. result->runner_up_gap is 0 on a tie.
   Errors: DG_E_ARG (null pointers, n < 1), DG_E_CUDA. */
dg_status dg_argmax_f64_reservoir(dg_ctx* ctx, const double* values, int64_t n, uint64_t seed,
                                  dg_grid_result* result, void* stream);

/* Device-side status of the work enqueued on `stream` through this context:
   waits for the stream, then reports and clears the status word that kernels
   set when one of their bounded waits (the tensor-core kernel's mbarrier
   waits, about one second each) gives up instead of hanging. Returns DG_OK, or
   DG_E_TIMEOUT when a wait expired (the affected trials' outputs are not
   written), or DG_E_CUDA. */
dg_status dg_stream_status(dg_ctx* ctx, void* stream);

/* Exercise the device-side failure path on `stream`: a kernel waits on a
   barrier that nothing ever completes, gives up after about wait_us
   microseconds (1 .. 2,000,000) and records it in the stream's status word, as
   the tensor-core kernel does when one of its waits expires. A following
   dg_stream_status returns DG_E_TIMEOUT; the context stays usable. Test aid;
   the paper has no counterpart. */
dg_status dg_selftest_wait_timeout(dg_ctx* ctx, int32_t wait_us, void* stream);

/* The per-candidate reduction of dg_grid_search and dg_run_episodes applied to
   given values, so that it can be checked on its own against exact sums (the
   FP64 per-candidate means that feed the argmax, Sec. 3.6). Group g of
   per_group FP32 values values[g per_group .. (g + 1) per_group - 1] is reduced
   as a candidate's trial outcomes are: `lanes` (8 or 32) lanes each add every
   lanes-th value into a compensated FP32 pair (TwoSum), the group combines its
   pairs in a fixed butterfly order, and means[g] = (hi + lo) / per_group in
   FP64. values, means: device; per_group 1 .. 1024. Test aid; the paper
   describes the reduction only as per-evaluation results that are combined.
   Errors: DG_E_ARG, DG_E_CUDA. */
dg_status dg_selftest_pair_sum(const float* values, int64_t n_groups, int32_t per_group,
                               int32_t lanes, double* means, void* stream);

/* Allocation-free dg_grid_search. The paper has no counterpart: this entry
   point exists for callers that may not allocate device memory themselves or
   let a library do it behind their back - code that runs while someone else's
   CUDA graph capture is open (cudaMalloc is not a stream operation and breaks
   the capture), frameworks whose own allocator owns the whole device budget,
   and latency-bound loops where a device allocation would stall other work.
   dg_grid_search allocates its scratch (argmax ticket, per-block partials,
   and for the plain form without cand_means a per-candidate means buffer) on
   first use of each stream; this call uses a fixed array in the library's own
   device memory instead (280 KiB, present on every GPU that loads the library
   until the process exits) and calls no allocator.
   Same arguments, outputs and results as dg_grid_search, with these limits:
     - DG_MODE_PLAIN, or DG_TIE_RESERVOIR, without cand_means evaluates at
       most 32768 candidates per call (DG_E_ARG beyond that);
     - the first call on a device looks up the array's device address and
       keeps it for the life of the process; make that first call before any
       stream capture on that device. A reset of the device's primary context
       after that first call (cudaDeviceReset, or a framework doing one)
       reloads the library's device memory elsewhere and is not supported;
     - every call shares the one array and it keeps the last call's contents
       (the call clears what must start at zero), so calls that may overlap
       on the GPU, e.g. on two streams without ordering, race: order them. */
dg_status dg_grid_search_noalloc(dg_model* model, const dg_grid_desc* desc,
                                 dg_grid_result* result, double* cand_means, void* stream);

/* ------------------------------------------------------ RNG replay (parity) --- */

/* Raw Philox4x32-10 words of blocks block0 .. block0+nblocks-1 of
   counter (trial, cand, block, purpose), key (seed lo, seed hi).
   out: device, 4*nblocks uint32. */
dg_status dg_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                          uint32_t block0, int64_t nblocks, uint32_t* out, void* stream);

/* Normals d0 .. d0+n-1 of the noise stream of (seed, trial, cand), FP32, as the
   kernels draw them. out: device, n floats. */
dg_status dg_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                     float* out, void* stream);

/* ---------------------------------------------------------------- batching --- */

/* A batch is a fixed set of runs and grid searches launched together: the
   first dg_batch_launch captures them as parallel branches of one CUDA graph
   (each on its own forked stream, so their tails overlap on the device);
   later launches replay that graph. Pointers and sizes are fixed when added. */
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(dg_ctx* ctx, dg_batch** out);
dg_status dg_batch_add_run(dg_batch* b, dg_model* model, const dg_run_desc* desc,
                           int8_t* choice, int32_t* step, float* final_state);
dg_status dg_batch_add_grid(dg_batch* b, dg_model* model, const dg_grid_desc* desc,
                            dg_grid_result* result, double* cand_means);
dg_status dg_batch_launch(dg_batch* b, void* stream);
/* Kernel launches one dg_batch_launch makes: the kernel nodes of the batch's
   CUDA graph (trial-order sorts included; memsets are not kernels). Valid after
   the first dg_batch_launch; DG_E_STATE before. */
dg_status dg_batch_kernels(const dg_batch* b, int64_t* n_kernels);
dg_status dg_batch_free(dg_batch* b);

/* ---------------------------------------------------------------- serving --- */

/* A job for the serving loop. Inputs and outputs are HOST memory (pinned memory
   makes the copies asynchronous); the loop copies inputs to device memory it
   owns, runs the job, and copies the outputs back. */
typedef struct {
  dg_model* model;
  int32_t is_grid;            /* 0: dg_run job; 1: dg_grid_search job */
  int32_t reserved;
  dg_run_desc run;            /* trial_params / cond_inputs are HOST pointers here */
  dg_grid_desc grid;          /* levels / positions are HOST pointers here */
  int8_t* choice;             /* host outputs of a run job (final_state may be NULL) */
  int32_t* step;
  float* final_state;
  dg_grid_result* grid_result;  /* host output of a grid job */
  double* cand_means;           /* host, may be NULL */
} dg_job;

typedef struct {
  int32_t status;             /* dg_status of the job */
  int32_t reserved;
  double t_submit, t_admit, t_done;  /* seconds on the host's steady clock */
  uint64_t device_bytes;      /* device memory the job held */
} dg_job_result;

/* Queue a job; returns at once with a ticket. The serving loop admits queued
   jobs in arrival order while the HBM budget has room, runs admitted jobs
   concurrently (each launch on its own stream, continuous batching), and frees
   a job's memory when its results are on the host. A batched job of a model
   that dg_run_jobs takes, of at most 65,536 trials (environment
   DG_SERVE_GROUP_TRIALS; 0 turns this off), takes later queued batched jobs of
   the same model, up to that size
   each, 256 jobs and 2^23 trials in all, into one dg_run_jobs launch; results
   are those of the jobs run alone. Likewise whole-grid searches (lowest-index
   ties, batched mode, at most 65,536 candidates) of one model, grid shape and
   trial count share a dg_grid_search_batch launch (up to 256 searches). A
   grouped run job whose trial_params (or
   cond_inputs), choice, step (and final_state) are all pinned host memory (cudaHostAlloc, or
   cudaHostRegister'd) is read and written by the kernel in place through the
   memory's device mapping, without staging copies (DG_SERVE_ZERO_COPY=0 turns
   this off).
   Errors: DG_E_ARG; DG_E_BUDGET if the job alone exceeds the budget. */
dg_status dg_submit(dg_ctx* ctx, const dg_job* job, uint64_t* ticket);

/* Wait up to timeout_ms (< 0: no limit) for a ticket. DG_E_TIMEOUT if it is
   not done by then (the job keeps running; wait again later). On DG_OK the
   job's host outputs are written and *result describes it. A ticket can be
   waited for successfully once. */
dg_status dg_wait(dg_ctx* ctx, uint64_t ticket, int32_t timeout_ms, dg_job_result* result);

/* Autotuner counters: launch-shape keys (model kind, size bucket) with a tuned
   shape, and launches so far that ran the default shape because their key had
   none and tuning was not allowed where they ran (the serving thread and graph
   capture never time shapes). Either pointer may be NULL. */
dg_status dg_tune_stats(dg_ctx* ctx, int64_t* tuned_keys, int64_t* untuned_launches);

/* Serving counters: jobs queued, running, done; device bytes in use. */
dg_status dg_serve_stats(dg_ctx* ctx, int64_t* queued, int64_t* running, int64_t* done,
                         uint64_t* bytes_in_use);

#ifdef __cplusplus
}
#endif

#endif
