/*
 * Oracle: a plain, slow FP64 CPU simulator of the cognitive-model hot path of
 * "Distill: Domain-Specific Compilation for Cognitive Models" (arXiv 2110.15425).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link, import or
 * call this library: only the test suite, the smoke check in __graft_entry__
 * and the CPU-baseline leg of bench.py use it. It shares no code, header,
 * constant table or helper with the CUDA library.
 *
 * Every model is written step by step in the order the paper (and the reading
 * of it recorded in the design notes) describes, in double precision, with no
 * blocking, fusion or reordering. Random draws come from this file's own
 * Philox4x32-10 (Salmon et al., SC'11) and Box-Muller transform.
 *
 * Pinned by the tests under tests/test_oracle_*.py:
 *   - Philox words: cross-checked bitwise against an independent
 *     Philox4x32-10 (Triton's CPU interpreter) and statistical checks.
 *   - Box-Muller: moments, KS test, radius/angle identities.
 *   - DDM: closed-form choice probability and mean decision time.
 *   - LCA: DDM equivalence mapping (Sec. 4.4, Fig. clones), noise-free fixed
 *     point, closed-form leak-only crossing step, rectification invariant.
 *   - Transfer network: integrator closed form, synchronous-update delay,
 *     logistic range, stop-rule closed form.
 *   - Grid search: noise-free geometric limits, perception variance,
 *     candidate index layout, lowest-index argmax.
 *   - Coarse-to-fine grid: round 0 equals the full grid search; noise-free
 *     closed forms of the shrinking box; convergence to the known optimum.
 *   - Extended Stroop: its network part equals the Stroop run, its DDM part
 *     equals the DDM run on the network's drift; noise-free closed forms.
 *   - Episodes: one step equals the grid search on the start positions; the
 *     moves' geometry (pursuit, evasion, unit steps); capture rules.
 *   - Reservoir tie-break: a rank-based restatement (the last tied index whose
 *     draw accepts its rank), uniformity over the tie set, the no-tie case.
 */
#ifndef DISTILL_ORACLE_H
#define DISTILL_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- RNG --- */

/* One Philox4x32-10 block: out = Philox(ctr, key). Salmon et al. SC'11. */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Raw words of blocks block0 .. block0+nblocks-1 of the stream
   key = (seed lo, seed hi), counter = (trial, cand, block, purpose).
   out has 4*nblocks words. */
void or_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                     uint32_t block0, int64_t nblocks, uint32_t* out);

/* u = ((w >> 9) + 1/2) * 2^-23, in (0, 1); exact in binary32. */
double or_uniform(uint32_t w);
void or_weights(uint64_t seed, uint32_t proj, int64_t n, double lo, double hi, float* out);

/* Box-Muller on (w0,w1) and (w2,w3): z[0..3]. */
void or_box_muller(const uint32_t w[4], double z[4]);

/* Normals d0 .. d0+n-1 of the noise stream (purpose 0) of (seed, trial, cand). */
void or_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                double* out);

/* ---------------------------------------------------------------- DDM --- */

/* Drift-diffusion run to threshold (Sec. 4.4; config: batched DDM).
   For each k in 0..n_ids-1, trial t = trial_ids[k] uses A[t], z[t]:
     x_0 = x0;  x_j = x_{j-1} + (A dt + sigma sqrt(dt) eps_j)  (eps_j = normal j-1)
   stop at the first j with |x_j| >= z. choice = 1 if x_j > 0 else 0; step = j.
   No crossing within max_steps: choice = -1, step = max_steps.
   x_final = x at the stop step; margin = min over j <= stop of ||x_j| - z|.
   Any output pointer may be NULL. */
void or_ddm_run(const float* A, const float* z, const uint32_t* trial_ids, int64_t n_ids,
                uint64_t seed, double dt, double sigma, double x0, int32_t max_steps,
                int8_t* choice, int32_t* step, double* x_final, double* margin);

/* The same DDM trials for a run that starts at global trial id trial0:
   trial k uses A[k], z[k] and the noise stream of id trial0 + k (32-bit, so
   ids wrap as the device's counter word does). */
void or_ddm_run_offset(const float* A, const float* z, int64_t n, uint32_t trial0,
                       uint64_t seed, double dt, double sigma, double x0, int32_t max_steps,
                       int8_t* choice, int32_t* step, double* x_final, double* margin);

/* ---------------------------------------------------------------- LCA --- */

/* Leaky competing accumulator (Sec. 4.4; Usher-McClelland form). Trial t uses
   inputs I[t*N .. t*N+N-1]. All N units are updated synchronously:
     x_i <- x_i + ((I_i - k x_i - beta sum_{j!=i} x_j) dt + sigma sqrt(dt) eps_i)
     x_i <- max(0, x_i)                   when rectify != 0
   eps_i of step j (1-based) is normal (j-1)*N + i.
   one-sided (two_sided == 0): stop when max_i x_i >= threshold;
     choice = argmax_i x_i (lowest index on exact ties).
   two-sided (N == 1 only): stop when |x| >= threshold; choice = (x > 0).
   Timeout: choice = -1, step = max_steps.
   x_final: N values per trial (may be NULL); margin: min over j <= stop of
   |max_i x_i - threshold| (one-sided) or ||x| - threshold| (two-sided); in the
   one-sided case with N > 1 it also takes the gap between the largest and the
   second largest x at the stop step, since the winner is decided there. */
void or_lca_run(int N, const float* I, const uint32_t* trial_ids, int64_t n_ids,
                uint64_t seed, double leak, double inhibition, double sigma, double dt,
                double threshold, int32_t max_steps, int rectify, int two_sided,
                int8_t* choice, int32_t* step, double* x_final, double* margin);

/* ------------------------------------------------------ transfer network --- */

#define OR_MAX_LAYERS 16
#define OR_MAX_PROJ 32

typedef struct {
  int n_layers;
  int size[OR_MAX_LAYERS];
  int is_input[OR_MAX_LAYERS];   /* 1: clamped input layer; 0: logistic layer */
  double gain[OR_MAX_LAYERS];
  double bias[OR_MAX_LAYERS];
  double rate;                   /* time-averaging rate tau */
  double noise_sd;               /* sd of the noise added to the state */
  int n_proj;
  int proj_sender[OR_MAX_PROJ];
  int proj_receiver[OR_MAX_PROJ];
  const float* proj_w[OR_MAX_PROJ]; /* [receiver size][sender size], row-major */
  int stop_layer;
  double stop_threshold;         /* stop when top1 - top2 > threshold (strict) */
  int32_t max_steps;
} or_net;

/* Layered logistic time-averaging network (Sec. 2.2, 3.3; Botvinick Stroop).
   cond_inputs: [n_cond][total input units] (input layers in layer order).
   Trial t takes condition (t / cond_block) % n_cond.
   s(0) = 0, y(0) = logistic(gain*(0 + bias)); step j = 1..max_steps, all
   layers read the step j-1 outputs:
     s <- (1 - rate) s + rate net + noise_sd eps,  y = 1 / (1 + exp(-gain (s + bias)))
   eps of noisy unit u (logistic units numbered in layer order) at step j is
   normal (j-1)*U + u, U = number of logistic units.
   Stop at the first j where top1 - top2 of the stop layer > threshold:
   choice = index of top1 (lowest index on exact ties), step = j.
   Timeout: choice = -1, step = max_steps.
   y_final: stop-layer outputs at the stop step ([n_ids][stop size], may be NULL).
   margin: min over j <= stop of |(top1 - top2) - threshold|.
   trace (may be NULL): outputs of every unit (all layers, in layer order) at
   steps 0..trace_steps, [n_ids][trace_steps+1][total units]; the trace keeps
   running past the stop step so closed forms can be checked at any j. */
void or_transfer_run(const or_net* net, const float* cond_inputs, int n_cond, int cond_block,
                     const uint32_t* trial_ids, int64_t n_ids, uint64_t seed,
                     int8_t* choice, int32_t* step, double* y_final, double* margin,
                     double* trace, int32_t trace_steps);

/* Extended Stroop (Sec. 5): the Stroop network adds DDM nodes (colour naming,
   finger pointing) on its response layer. For each trial: the network runs
   to its own stop (or_transfer_run); then DDM q is driven by
   drift_q = bias_q + sum_i W[q][i] y_i of the stop layer's outputs y at that
   step (FP64), starts at 0 and runs x_j = x_{j-1} + drift dt_q +
   sigma_q sqrt(dt_q) eps_j to |x| >= bound_q or ddm_max[q] steps, with noise
   stream (seed, trial, cand 1 + q). The trial's response is the first DDM to
   reach a bound (fewest steps, lower q on equal steps):
   choice = 2 q + (upper bound), step = network steps + that DDM's steps; with
   none, choice = -1 and step = network steps + max_q ddm_max[q].
   Per trial: s_choice, s_step, y_final [ss], s_margin of the network;
   per (trial, q): drift, d_choice, d_step, d_x, d_margin. n_ddm <= 8. */
void or_extended_run(const or_net* net, const float* cond_inputs, int n_cond, int cond_block,
                     const uint32_t* trial_ids, int64_t n_ids, uint64_t seed, int n_ddm,
                     const float* W, const float* bias, const double* dt, const double* sigma,
                     const double* bound, const int32_t* ddm_max, int8_t* choice, int32_t* step,
                     int8_t* s_choice, int32_t* s_step, double* y_final, double* s_margin,
                     double* drift, int8_t* d_choice, int32_t* d_step, double* d_x,
                     double* d_margin);

/* ------------------------------------------------- predator-prey grid --- */

/* One evaluation of the predator-prey model (Sec. 2.1, Fig. pp_eg) for
   allocation a[0..2] (player, predator, prey) on trial `trial` of candidate
   `cand`. pos = true positions (player xy, predator xy, prey xy).
   Perceived X^_e = X_e + eps_{2e+c} / (obs_offset + a_e), eps from stream
   (seed, trial, cand). u_prey = unit(Y^ - P^), u_pred = unit(D^ - P^),
   act = unit(u_prey - pred_weight u_pred), unit(0) = 0.
   outcome = -|P + act - Y| - sum_e a_e^2. perceived (may be NULL) gets X^. */
double or_pp_outcome(const float pos[6], const double a[3], uint64_t seed, uint32_t trial,
                     uint32_t cand, double obs_offset, double pred_weight, double* perceived);

/* Per-candidate mean outcome over trials 0..n_trials-1 (summed in index order)
   for candidates cand_ids[0..n_ids-1]. Candidate c has levels
   (l0, l1, l2) with c = (l0*L1 + l1)*L2 + l2 and allocation
   (lv0[l0], lv1[l1], lv2[l2]). pos: [n_trials][6]. */
void or_pp_means(const float* pos, int32_t n_trials, const float* lv0, int32_t L0,
                 const float* lv1, int32_t L1, const float* lv2, int32_t L2,
                 const uint32_t* cand_ids, int64_t n_ids, uint64_t seed,
                 double obs_offset, double pred_weight, double* means);

/* argmax with lowest index on exact ties; gap = best - second best (0 on a tie;
   0 when n == 1). */
void or_argmax(const double* v, int64_t n, int64_t* best, double* best_value, double* gap);

/* argmax with a uniformly random choice among exact ties (the reservoir
   sampling of Sec. 3.3; Vitter, ACM TOMS 1985, Algorithm R with a reservoir of
   one). One pass over v in index order: a value above the running maximum
   empties the reservoir and becomes its element (k = 1); the k-th value equal
   to the running maximum, at index i, replaces the element with probability
   1/k, decided by word 0 w of Philox4x32-10(key = (seed lo, seed hi),
   counter = (i lo, i hi, 0, 4)): replace iff w k < 2^32. Purpose 4 keeps these
   draws apart from every noise stream (purpose 0). n_ties = number of values
   equal to the maximum; gap as or_argmax (0 on a tie). */
void or_argmax_reservoir(const double* v, int64_t n, uint64_t seed, int64_t* best,
                         double* best_value, double* gap, int64_t* n_ties);

/* Coarse-to-fine grid search (the refinement of the prey-attention search of
   Sec. 4.3, done by simulation instead of value-range analysis). Round r =
   0..R-1 lays G points on each signal's interval [lo_e, hi_e]:
   level l = lo + (hi - lo) l / (G - 1) (FP64, rounded to FP32); candidate
   c = (l0 G + l1) G + l2 is simulated over n_trials trials exactly as in
   or_pp_means but with noise stream (seed, trial, r G^3 + c); best = argmax
   (lowest index on ties). The next interval of each signal is the best level
   +- one grid spacing (hi - lo)/(G - 1), clipped to the domain [lo0, hi0]
   (FP64, rounded to FP32), so it shrinks by 2/(G - 1) per round (G >= 4).
   Outputs per round: best[r], value[r], gap[r], box[r][6] = (lo[3], hi[3])
   of the round, alloc[r][3] = allocation of the best candidate. G <= 64. */
void or_pp_refine(const float* pos, int32_t n_trials, const float lo0[3], const float hi0[3],
                  int32_t G, int32_t R, uint64_t seed, double obs_offset, double pred_weight,
                  int64_t* best, double* value, double* gap, float* box, float* alloc);

/* One time-stepped predator-prey episode (Sec. 2.1: the search over
   allocations is repeated at every time step until the prey or the player is
   caught). State S = (P, D, Y) in FP32. At step t = 0, 1, ...:
     - every candidate allocation c (layout as or_pp_means) is simulated on
       n_trials perceptions of the current S, perception noise from stream
       (seed, trial t n_trials + j, cand c) at Philox blocks 2 episode + {0, 1};
       FP64 mean; best = argmax (lowest index on ties);
     - the player perceives S once more with the best allocation (stream
       (seed, t, 0xFFFFFFFF), same blocks) and moves by speed[0] act; the
       predator moves speed[1] unit(P - D) toward the player and the prey
       speed[2] unit(Y - P) away from it, all from the positions at the start
       of the step (FP64, rounded to FP32);
     - with the new positions, |P - Y| <= radius ends the episode with
       outcome +1 (prey caught), else |P - D| <= radius with -1 (player
       caught); after max_steps steps without either, outcome 0.
   steps = steps taken. Per step t (may be NULL): traj_best[t], its mean
   traj_value[t], the runner-up gap traj_gap[t], positions after the step
   traj_pos[t][6], and
   traj_margin[t] = min(| |P-Y| - radius |, | |P-D| - radius |). */
void or_pp_episode(const float start[6], uint32_t episode, const float* lv0, int32_t L0,
                   const float* lv1, int32_t L1, const float* lv2, int32_t L2, int32_t n_trials,
                   int32_t max_steps, uint64_t seed, double obs_offset, double pred_weight,
                   const double speed[3], double radius, int8_t* outcome, int32_t* steps,
                   float final_pos[6], int64_t* traj_best, double* traj_value,
                   double* traj_gap, float* traj_pos, double* traj_margin);

#ifdef __cplusplus
}
#endif

#endif
