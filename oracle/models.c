/*
 * Oracle models: DDM, LCA, layered logistic transfer network, predator-prey
 * grid search. Plain FP64, one trial at a time, steps in the paper's order.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

/* Noise stream of one (seed, trial, candidate): normal d is lane d&3 of the
   Box-Muller output of Philox block d>>2 (purpose 0). Keeps the last block so
   consecutive draws do not recompute it. */
typedef struct {
  uint64_t seed;
  uint32_t trial, cand;
  uint32_t block0; /* block of normal 0 (episodes give each episode its own blocks) */
  int64_t block;
  double z[4];
} noise_stream;

static void noise_open(noise_stream* s, uint64_t seed, uint32_t trial, uint32_t cand) {
  s->seed = seed;
  s->trial = trial;
  s->cand = cand;
  s->block0 = 0u;
  s->block = -1;
}

static double noise_at(noise_stream* s, uint64_t d) {
  int64_t block = (int64_t)(d >> 2);
  if (block != s->block) {
    uint32_t w[4];
    or_philox_words(s->seed, s->trial, s->cand, 0u, s->block0 + (uint32_t)block, 1, w);
    or_box_muller(w, s->z);
    s->block = block;
  }
  return s->z[d & 3];
}

/* ------------------------------------------------------------------ DDM --- */

/* One DDM trial on noise stream (seed, trial, cand): x_j = x_{j-1} +
   (drift dt + sigma sqrt(dt) eps_j) until |x_j| >= bound or max_steps;
   margin = min_j | |x_j| - bound |. */
static void ddm_trial(double drift, double bound, uint64_t seed, uint32_t trial, uint32_t cand,
                      double dt, double sigma, double x0, int32_t max_steps, int8_t* choice,
                      int32_t* step, double* x_final, double* margin) {
  const double diffusion = sigma * sqrt(dt);
  noise_stream ns;
  noise_open(&ns, seed, trial, cand);
  double x = x0;
  double m = INFINITY;
  int8_t c = -1;
  int32_t s = max_steps;
  for (int32_t j = 1; j <= max_steps; ++j) {
    double eps = noise_at(&ns, (uint64_t)(j - 1));
    x = x + (drift * dt + diffusion * eps);
    double d = fabs(fabs(x) - bound);
    if (d < m) m = d;
    if (fabs(x) >= bound) {
      c = (x > 0.0) ? 1 : 0;
      s = j;
      break;
    }
  }
  *choice = c;
  *step = s;
  *x_final = x;
  *margin = m;
}

void or_ddm_run(const float* A, const float* z, const uint32_t* trial_ids, int64_t n_ids,
                uint64_t seed, double dt, double sigma, double x0, int32_t max_steps,
                int8_t* choice, int32_t* step, double* x_final, double* margin) {
  for (int64_t k = 0; k < n_ids; ++k) {
    uint32_t t = trial_ids[k];
    int8_t c;
    int32_t st;
    double x, m;
    ddm_trial((double)A[t], (double)z[t], seed, t, 0u, dt, sigma, x0, max_steps, &c, &st, &x, &m);
    if (choice) choice[k] = c;
    if (step) step[k] = st;
    if (x_final) x_final[k] = x;
    if (margin) margin[k] = m;
  }
}

void or_ddm_run_offset(const float* A, const float* z, int64_t n, uint32_t trial0,
                       uint64_t seed, double dt, double sigma, double x0, int32_t max_steps,
                       int8_t* choice, int32_t* step, double* x_final, double* margin) {
  for (int64_t k = 0; k < n; ++k)
    ddm_trial((double)A[k], (double)z[k], seed, trial0 + (uint32_t)k, 0u, dt, sigma, x0,
              max_steps, &choice[k], &step[k], &x_final[k], &margin[k]);
}

/* ------------------------------------------------------------------ LCA --- */

void or_lca_run(int N, const float* I, const uint32_t* trial_ids, int64_t n_ids,
                uint64_t seed, double leak, double inhibition, double sigma, double dt,
                double threshold, int32_t max_steps, int rectify, int two_sided,
                int8_t* choice, int32_t* step, double* x_final, double* margin) {
  const double diffusion = sigma * sqrt(dt);
  double* x = (double*)malloc(sizeof(double) * (size_t)N);
  double* xn = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t k = 0; k < n_ids; ++k) {
    uint32_t t = trial_ids[k];
    const float* in = I + (size_t)t * (size_t)N;
    noise_stream ns;
    noise_open(&ns, seed, t, 0u);
    for (int i = 0; i < N; ++i) x[i] = 0.0;
    double m = INFINITY;
    int8_t c = -1;
    int32_t s = max_steps;
    for (int32_t j = 1; j <= max_steps; ++j) {
      /* synchronous update: every unit reads the step j-1 values */
      for (int i = 0; i < N; ++i) {
        double others = 0.0;
        for (int q = 0; q < N; ++q)
          if (q != i) others += x[q];
        double eps = noise_at(&ns, (uint64_t)(j - 1) * (uint64_t)N + (uint64_t)i);
        double v = x[i] + (((double)in[i] - leak * x[i] - inhibition * others) * dt +
                           diffusion * eps);
        if (rectify && v < 0.0) v = 0.0;
        xn[i] = v;
      }
      memcpy(x, xn, sizeof(double) * (size_t)N);
      if (two_sided) {
        double d = fabs(fabs(x[0]) - threshold);
        if (d < m) m = d;
        if (fabs(x[0]) >= threshold) {
          c = (x[0] > 0.0) ? 1 : 0;
          s = j;
          break;
        }
      } else {
        int best = 0;
        for (int i = 1; i < N; ++i)
          if (x[i] > x[best]) best = i;
        double d = fabs(x[best] - threshold);
        if (d < m) m = d;
        if (x[best] >= threshold) {
          double second = -INFINITY;
          for (int i = 0; i < N; ++i)
            if (i != best && x[i] > second) second = x[i];
          if (N > 1 && x[best] - second < m) m = x[best] - second;
          c = (int8_t)best;
          s = j;
          break;
        }
      }
    }
    if (choice) choice[k] = c;
    if (step) step[k] = s;
    if (x_final)
      for (int i = 0; i < N; ++i) x_final[(size_t)k * (size_t)N + (size_t)i] = x[i];
    if (margin) margin[k] = m;
  }
  free(x);
  free(xn);
}

/* ------------------------------------------------------ transfer network --- */

static double logistic(double gain, double bias, double s) {
  return 1.0 / (1.0 + exp(-gain * (s + bias)));
}

/* top1 - top2 and the index of top1 (lowest index on exact ties) */
static double top_gap(const double* y, int n, int* arg) {
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (y[i] > y[best]) best = i;
  double second = -INFINITY;
  for (int i = 0; i < n; ++i)
    if (i != best && y[i] > second) second = y[i];
  *arg = best;
  if (n == 1) return y[best];
  return y[best] - second;
}

void or_transfer_run(const or_net* net, const float* cond_inputs, int n_cond, int cond_block,
                     const uint32_t* trial_ids, int64_t n_ids, uint64_t seed,
                     int8_t* choice, int32_t* step, double* y_final, double* margin,
                     double* trace, int32_t trace_steps) {
  int L = net->n_layers;
  int off[OR_MAX_LAYERS + 1];     /* unit offset of each layer (all units) */
  int noisy_off[OR_MAX_LAYERS];   /* offset among logistic units, -1 for inputs */
  int n_in = 0, U = 0;
  off[0] = 0;
  for (int l = 0; l < L; ++l) {
    off[l + 1] = off[l] + net->size[l];
    if (net->is_input[l]) {
      noisy_off[l] = -1;
      n_in += net->size[l];
    } else {
      noisy_off[l] = U;
      U += net->size[l];
    }
  }
  int total = off[L];
  double* y = (double*)malloc(sizeof(double) * (size_t)total);
  double* yn = (double*)malloc(sizeof(double) * (size_t)total);
  double* s = (double*)malloc(sizeof(double) * (size_t)total);
  double* sn = (double*)malloc(sizeof(double) * (size_t)total);
  int sl = net->stop_layer;
  int ssize = net->size[sl];
  int32_t run_steps = net->max_steps;
  if (trace && trace_steps > run_steps) run_steps = trace_steps;

  for (int64_t k = 0; k < n_ids; ++k) {
    uint32_t t = trial_ids[k];
    int cond = (int)((t / (uint32_t)cond_block) % (uint32_t)n_cond);
    const float* cin = cond_inputs + (size_t)cond * (size_t)n_in;
    noise_stream ns;
    noise_open(&ns, seed, t, 0u);
    /* step 0: inputs clamped, logistic units at s = 0 */
    int in_pos = 0;
    for (int l = 0; l < L; ++l) {
      for (int i = 0; i < net->size[l]; ++i) {
        int u = off[l] + i;
        if (net->is_input[l]) {
          y[u] = (double)cin[in_pos++];
          s[u] = 0.0;
        } else {
          s[u] = 0.0;
          y[u] = logistic(net->gain[l], net->bias[l], 0.0);
        }
      }
    }
    double* tr = trace ? trace + (size_t)k * (size_t)(trace_steps + 1) * (size_t)total : NULL;
    if (tr) memcpy(tr, y, sizeof(double) * (size_t)total);

    double m = INFINITY;
    int8_t c = -1;
    int32_t st = net->max_steps;
    int stopped = 0;
    double yst[64];
    for (int32_t j = 1; j <= run_steps; ++j) {
      /* synchronous update (Sec. 3.3): all layers read the step j-1 outputs y */
      for (int l = 0; l < L; ++l) {
        for (int i = 0; i < net->size[l]; ++i) {
          int u = off[l] + i;
          if (net->is_input[l]) {
            sn[u] = s[u];
            yn[u] = y[u];
            continue;
          }
          double nt = 0.0;
          for (int p = 0; p < net->n_proj; ++p) {
            if (net->proj_receiver[p] != l) continue;
            int snd = net->proj_sender[p];
            const float* w = net->proj_w[p] + (size_t)i * (size_t)net->size[snd];
            for (int q = 0; q < net->size[snd]; ++q) nt += (double)w[q] * y[off[snd] + q];
          }
          double eps = noise_at(&ns, (uint64_t)(j - 1) * (uint64_t)U +
                                         (uint64_t)(noisy_off[l] + i));
          sn[u] = (1.0 - net->rate) * s[u] + net->rate * nt + net->noise_sd * eps;
          yn[u] = logistic(net->gain[l], net->bias[l], sn[u]);
        }
      }
      memcpy(s, sn, sizeof(double) * (size_t)total);
      memcpy(y, yn, sizeof(double) * (size_t)total);
      if (tr && j <= trace_steps) memcpy(tr + (size_t)j * (size_t)total, y, sizeof(double) * (size_t)total);
      if (!stopped && j <= net->max_steps) {
        int arg;
        double gap = top_gap(y + off[sl], ssize, &arg);
        double d = fabs(gap - net->stop_threshold);
        if (d < m) m = d;
        if (gap > net->stop_threshold) {
          stopped = 1;
          c = (int8_t)arg;
          st = j;
          for (int i = 0; i < ssize && i < 64; ++i) yst[i] = y[off[sl] + i];
        }
      }
      if (stopped && (!tr || j >= trace_steps)) break;
      if (!stopped && j >= net->max_steps && (!tr || j >= trace_steps)) break;
    }
    if (!stopped)
      for (int i = 0; i < ssize && i < 64; ++i) yst[i] = y[off[sl] + i];
    /* with a trace longer than max_steps, y has moved on; the timeout value is
       the one at max_steps, which the trace holds */
    if (!stopped && tr && trace_steps > net->max_steps)
      for (int i = 0; i < ssize && i < 64; ++i)
        yst[i] = tr[(size_t)net->max_steps * (size_t)total + (size_t)(off[sl] + i)];
    if (choice) choice[k] = c;
    if (step) step[k] = st;
    if (margin) margin[k] = m;
    if (y_final)
      for (int i = 0; i < ssize && i < 64; ++i) y_final[(size_t)k * (size_t)ssize + (size_t)i] = yst[i];
  }
  free(y);
  free(yn);
  free(s);
  free(sn);
}

/* ------------------------------------------------- predator-prey grid --- */

static void unit2(double vx, double vy, double* ox, double* oy) {
  double n = sqrt(vx * vx + vy * vy);
  if (n > 0.0) {
    *ox = vx / n;
    *oy = vy / n;
  } else {
    *ox = 0.0;
    *oy = 0.0;
  }
}

/* Perceived positions X^_e = X_e + eps_{2e+c} / (obs_offset + a_e) with the
   normals of stream (seed, trial, cand) starting at block block0, and the
   Action node's unit step act = unit(unit(Y^ - P^) - w unit(D^ - P^)). */
static void pp_perceive_act(const float pos[6], const double a[3], uint64_t seed,
                            uint32_t trial, uint32_t cand, uint32_t block0, double obs_offset,
                            double pred_weight, double ph[6], double* ax, double* ay) {
  noise_stream ns;
  noise_open(&ns, seed, trial, cand);
  ns.block0 = block0;
  for (int e = 0; e < 3; ++e) {
    double sd = 1.0 / (obs_offset + a[e]);
    for (int c = 0; c < 2; ++c) {
      int d = 2 * e + c;
      ph[d] = (double)pos[d] + sd * noise_at(&ns, (uint64_t)d);
    }
  }
  double uyx, uyy, udx, udy;
  unit2(ph[4] - ph[0], ph[5] - ph[1], &uyx, &uyy);
  unit2(ph[2] - ph[0], ph[3] - ph[1], &udx, &udy);
  unit2(uyx - pred_weight * udx, uyy - pred_weight * udy, ax, ay);
}

/* Objective node: -|P + act - Y| - sum_e a_e^2 with true P, Y. */
static double pp_outcome_b(const float pos[6], const double a[3], uint64_t seed,
                           uint32_t trial, uint32_t cand, uint32_t block0, double obs_offset,
                           double pred_weight) {
  double ph[6], ax, ay;
  pp_perceive_act(pos, a, seed, trial, cand, block0, obs_offset, pred_weight, ph, &ax, &ay);
  double nx = (double)pos[0] + ax - (double)pos[4];
  double ny = (double)pos[1] + ay - (double)pos[5];
  double cost = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
  return -sqrt(nx * nx + ny * ny) - cost;
}

double or_pp_outcome(const float pos[6], const double a[3], uint64_t seed, uint32_t trial,
                     uint32_t cand, double obs_offset, double pred_weight, double* perceived) {
  if (perceived) {
    double ax, ay;
    pp_perceive_act(pos, a, seed, trial, cand, 0u, obs_offset, pred_weight, perceived, &ax, &ay);
  }
  return pp_outcome_b(pos, a, seed, trial, cand, 0u, obs_offset, pred_weight);
}

void or_pp_means(const float* pos, int32_t n_trials, const float* lv0, int32_t L0,
                 const float* lv1, int32_t L1, const float* lv2, int32_t L2,
                 const uint32_t* cand_ids, int64_t n_ids, uint64_t seed,
                 double obs_offset, double pred_weight, double* means) {
  (void)L0;
  for (int64_t k = 0; k < n_ids; ++k) {
    uint32_t c = cand_ids[k];
    uint32_t l2 = c % (uint32_t)L2;
    uint32_t l1 = (c / (uint32_t)L2) % (uint32_t)L1;
    uint32_t l0 = c / ((uint32_t)L2 * (uint32_t)L1);
    double a[3] = {(double)lv0[l0], (double)lv1[l1], (double)lv2[l2]};
    double sum = 0.0;
    for (int32_t j = 0; j < n_trials; ++j)
      sum += or_pp_outcome(pos + 6 * (size_t)j, a, seed, (uint32_t)j, c, obs_offset,
                           pred_weight, NULL);
    means[k] = sum / (double)n_trials;
  }
}

void or_argmax(const double* v, int64_t n, int64_t* best, double* best_value, double* gap) {
  int64_t b = 0;
  for (int64_t i = 1; i < n; ++i)
    if (v[i] > v[b]) b = i;
  double second = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (i != b && v[i] > second) second = v[i];
  *best = b;
  *best_value = v[b];
  *gap = (n > 1) ? v[b] - second : 0.0;
}

void or_argmax_reservoir(const double* v, int64_t n, uint64_t seed, int64_t* best,
                         double* best_value, double* gap, int64_t* n_ties) {
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  int64_t choice = 0; /* the reservoir's one element */
  int64_t k = 1;      /* values equal to the running maximum seen so far */
  double top = v[0];
  for (int64_t i = 1; i < n; ++i) {
    if (v[i] > top) {
      top = v[i];
      choice = i;
      k = 1;
    } else if (v[i] == top) {
      k += 1;
      const uint32_t ctr[4] = {(uint32_t)i, (uint32_t)((uint64_t)i >> 32), 0u, 4u};
      uint32_t w[4];
      or_philox4x32_10(ctr, key, w);
      if ((uint64_t)w[0] * (uint64_t)k < ((uint64_t)1 << 32)) choice = i;
    }
  }
  double second = -INFINITY;
  for (int64_t i = 0; i < n; ++i)
    if (i != choice && v[i] > second) second = v[i];
  *best = choice;
  *best_value = top;
  *gap = (n > 1) ? top - second : 0.0;
  *n_ties = k;
}

/* Level l of G on [lo, hi]: lo + (hi - lo) l / (G - 1) in FP64, rounded to FP32. */
static float refine_level(float lo, float hi, int l, int G) {
  double w = (double)hi - (double)lo;
  double t = (w * (double)l) / (double)(G - 1);
  return (float)((double)lo + t);
}

void or_pp_refine(const float* pos, int32_t n_trials, const float lo0[3], const float hi0[3],
                  int32_t G, int32_t R, uint64_t seed, double obs_offset, double pred_weight,
                  int64_t* best, double* value, double* gap, float* box, float* alloc) {
  float lo[3] = {lo0[0], lo0[1], lo0[2]};
  float hi[3] = {hi0[0], hi0[1], hi0[2]};
  const int64_t n_cand = (int64_t)G * G * G;
  double* means = (double*)malloc(sizeof(double) * (size_t)n_cand);
  float lv[3][64];
  for (int32_t r = 0; r < R; ++r) {
    /* the grid of this round */
    for (int e = 0; e < 3; ++e) {
      box[6 * r + e] = lo[e];
      box[6 * r + 3 + e] = hi[e];
      for (int l = 0; l < G; ++l) lv[e][l] = refine_level(lo[e], hi[e], l, G);
    }
    /* simulate every candidate; its noise stream is candidate r G^3 + c */
    for (int64_t c = 0; c < n_cand; ++c) {
      const int l2 = (int)(c % G), l1 = (int)((c / G) % G), l0 = (int)(c / ((int64_t)G * G));
      const double a[3] = {(double)lv[0][l0], (double)lv[1][l1], (double)lv[2][l2]};
      const uint32_t stream = (uint32_t)((int64_t)r * n_cand + c);
      double sum = 0.0;
      for (int32_t j = 0; j < n_trials; ++j)
        sum += or_pp_outcome(pos + 6 * (size_t)j, a, seed, (uint32_t)j, stream, obs_offset,
                             pred_weight, NULL);
      means[c] = sum / (double)n_trials;
    }
    int64_t b;
    or_argmax(means, n_cand, &b, &value[r], &gap[r]);
    best[r] = b;
    const int lb[3] = {(int)(b / ((int64_t)G * G)), (int)((b / G) % G), (int)(b % G)};
    /* next box: the best point +- one grid spacing, inside the domain */
    for (int e = 0; e < 3; ++e) {
      const float center = lv[e][lb[e]];
      alloc[3 * r + e] = center;
      const double s = ((double)hi[e] - (double)lo[e]) / (double)(G - 1);
      double nlo = (double)center - s, nhi = (double)center + s;
      if (nlo < (double)lo0[e]) nlo = (double)lo0[e];
      if (nhi > (double)hi0[e]) nhi = (double)hi0[e];
      lo[e] = (float)nlo;
      hi[e] = (float)nhi;
    }
  }
  free(means);
}

void or_pp_episode(const float start[6], uint32_t episode, const float* lv0, int32_t L0,
                   const float* lv1, int32_t L1, const float* lv2, int32_t L2, int32_t n_trials,
                   int32_t max_steps, uint64_t seed, double obs_offset, double pred_weight,
                   const double speed[3], double radius, int8_t* outcome, int32_t* steps,
                   float final_pos[6], int64_t* traj_best, double* traj_value,
                   double* traj_gap, float* traj_pos, double* traj_margin) {
  const int64_t n_cand = (int64_t)L0 * L1 * L2;
  double* means = (double*)malloc(sizeof(double) * (size_t)n_cand);
  float S[6];
  for (int d = 0; d < 6; ++d) S[d] = start[d];
  const uint32_t block0 = 2u * episode;
  int8_t out = 0;
  int32_t t = 0;
  for (t = 0; t < max_steps; ++t) {
    /* Control: simulate every allocation on n_trials perceptions of the
       current positions (Sec. 2.1) and keep the best */
    for (int64_t c = 0; c < n_cand; ++c) {
      const int l2 = (int)(c % L2), l1 = (int)((c / L2) % L1), l0 = (int)(c / ((int64_t)L2 * L1));
      const double a[3] = {(double)lv0[l0], (double)lv1[l1], (double)lv2[l2]};
      double sum = 0.0;
      for (int32_t j = 0; j < n_trials; ++j)
        sum += pp_outcome_b(S, a, seed, (uint32_t)t * (uint32_t)n_trials + (uint32_t)j,
                            (uint32_t)c, block0, obs_offset, pred_weight);
      means[c] = sum / (double)n_trials;
    }
    int64_t b;
    double bv, gap;
    or_argmax(means, n_cand, &b, &bv, &gap);
    const int l2 = (int)(b % L2), l1 = (int)((b / L2) % L1), l0 = (int)(b / ((int64_t)L2 * L1));
    const double a[3] = {(double)lv0[l0], (double)lv1[l1], (double)lv2[l2]};
    /* Act: one more perception with the chosen allocation moves the player;
       the predator steps toward the player, the prey away from it */
    double ph[6], ax, ay, ux, uy, vx, vy;
    pp_perceive_act(S, a, seed, (uint32_t)t, 0xFFFFFFFFu, block0, obs_offset, pred_weight, ph,
                    &ax, &ay);
    unit2((double)S[0] - (double)S[2], (double)S[1] - (double)S[3], &ux, &uy);
    unit2((double)S[4] - (double)S[0], (double)S[5] - (double)S[1], &vx, &vy);
    float N[6];
    N[0] = (float)((double)S[0] + speed[0] * ax);
    N[1] = (float)((double)S[1] + speed[0] * ay);
    N[2] = (float)((double)S[2] + speed[1] * ux);
    N[3] = (float)((double)S[3] + speed[1] * uy);
    N[4] = (float)((double)S[4] + speed[2] * vx);
    N[5] = (float)((double)S[5] + speed[2] * vy);
    for (int d = 0; d < 6; ++d) S[d] = N[d];
    const double py = sqrt(((double)S[0] - S[4]) * ((double)S[0] - S[4]) +
                           ((double)S[1] - S[5]) * ((double)S[1] - S[5]));
    const double pd = sqrt(((double)S[0] - S[2]) * ((double)S[0] - S[2]) +
                           ((double)S[1] - S[3]) * ((double)S[1] - S[3]));
    if (traj_best) traj_best[t] = b;
    if (traj_value) traj_value[t] = bv;
    if (traj_gap) traj_gap[t] = gap;
    if (traj_pos)
      for (int d = 0; d < 6; ++d) traj_pos[6 * (size_t)t + d] = S[d];
    if (traj_margin) traj_margin[t] = fmin(fabs(py - radius), fabs(pd - radius));
    if (py <= radius) {
      out = 1;
      break;
    }
    if (pd <= radius) {
      out = -1;
      break;
    }
  }
  *outcome = out;
  *steps = (t < max_steps) ? t + 1 : max_steps;
  for (int d = 0; d < 6; ++d) final_pos[d] = S[d];
  free(means);
}

void or_extended_run(const or_net* net, const float* cond_inputs, int n_cond, int cond_block,
                     const uint32_t* trial_ids, int64_t n_ids, uint64_t seed, int n_ddm,
                     const float* W, const float* bias, const double* dt, const double* sigma,
                     const double* bound, const int32_t* ddm_max, int8_t* choice, int32_t* step,
                     int8_t* s_choice, int32_t* s_step, double* y_final, double* s_margin,
                     double* drift, int8_t* d_choice, int32_t* d_step, double* d_x,
                     double* d_margin) {
  const int ss = net->size[net->stop_layer];
  double y[64];
  for (int64_t k = 0; k < n_ids; ++k) {
    /* the Stroop network to its own stop */
    int8_t sc;
    int32_t st;
    double sm;
    or_transfer_run(net, cond_inputs, n_cond, cond_block, trial_ids + k, 1, seed, &sc, &st, y,
                    &sm, NULL, 0);
    s_choice[k] = sc;
    s_step[k] = st;
    s_margin[k] = sm;
    for (int i = 0; i < ss; ++i) y_final[k * ss + i] = y[i];
    /* the DDM nodes, driven by the response layer at that step */
    int first = -1;
    for (int q = 0; q < n_ddm; ++q) {
      double A = (double)bias[q];
      for (int i = 0; i < ss; ++i) A += (double)W[q * ss + i] * y[i];
      drift[k * n_ddm + q] = A;
      const size_t o = (size_t)k * n_ddm + q;
      ddm_trial(A, bound[q], seed, trial_ids[k], 1u + (uint32_t)q, dt[q], sigma[q], 0.0, ddm_max[q],
                &d_choice[o], &d_step[o], &d_x[o], &d_margin[o]);
      if (d_choice[o] >= 0 && (first < 0 || d_step[o] < d_step[(size_t)k * n_ddm + first]))
        first = q;
    }
    /* the trial's response: the first DDM to reach a bound (lower index on
       equal steps) */
    if (first >= 0) {
      choice[k] = (int8_t)(2 * first + d_choice[(size_t)k * n_ddm + first]);
      step[k] = st + d_step[(size_t)k * n_ddm + first];
    } else {
      int32_t mx = 0;
      for (int q = 0; q < n_ddm; ++q) mx = ddm_max[q] > mx ? ddm_max[q] : mx;
      choice[k] = -1;
      step[k] = st + mx;
    }
  }
}
