/*
 * Oracle RNG: Philox4x32-10 and Box-Muller, in plain C / FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
 * "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4x32-bit counter is
 * passed through 10 rounds; each round multiplies words 0 and 2 by two fixed
 * odd constants, and the high halves of the products are xor-ed with words 1
 * and 3 and the two key words; the key is advanced by two Weyl constants
 * before every round after the first.
 *
 * The paper uses one stateful PRNG per evaluation whose state is restored on
 * every call (Sec. 3.6); a counter-based generator reaches the same goal (every
 * evaluation draws reproducible, independent numbers) with no state at all.
 */
#include <math.h>
#include "oracle.h"

#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0;
    x1 = y1;
    x2 = y2;
    x3 = y3;
  }
  out[0] = x0;
  out[1] = x1;
  out[2] = x2;
  out[3] = x3;
}

void or_philox_words(uint64_t seed, uint32_t trial, uint32_t cand, uint32_t purpose,
                     uint32_t block0, int64_t nblocks, uint32_t* out) {
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  for (int64_t b = 0; b < nblocks; ++b) {
    uint32_t ctr[4] = {trial, cand, (uint32_t)(block0 + b), purpose};
    or_philox4x32_10(ctr, key, out + 4 * b);
  }
}

double or_uniform(uint32_t w) {
  /* top 23 bits plus one half, times 2^-23: strictly inside (0, 1), and
     exactly representable in binary32 as well as binary64 */
  return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

void or_box_muller(const uint32_t w[4], double z[4]) {
  const double two_pi = 6.283185307179586476925286766559;
  for (int pair = 0; pair < 2; ++pair) {
    double ua = or_uniform(w[2 * pair]);
    double ub = or_uniform(w[2 * pair + 1]);
    double r = sqrt(-2.0 * log(ua));
    z[2 * pair] = r * cos(two_pi * ub);
    z[2 * pair + 1] = r * sin(two_pi * ub);
  }
}

void or_normals(uint64_t seed, uint32_t trial, uint32_t cand, uint64_t d0, int64_t n,
                double* out) {
  uint32_t w[4];
  double z[4];
  int64_t cached_block = -1;
  for (int64_t k = 0; k < n; ++k) {
    uint64_t d = d0 + (uint64_t)k;
    int64_t block = (int64_t)(d >> 2);
    if (block != cached_block) {
      or_philox_words(seed, trial, cand, 0u, (uint32_t)block, 1, w);
      or_box_muller(w, z);
      cached_block = block;
    }
    out[k] = z[d & 3];
  }
}

/* Static weights drawn from a seed (Sec. 3.3's read-only parameters): weight w
   of projection `proj` is lo + (hi - lo) u in FP64, rounded to binary32, where
   u is the uniform of word (w mod 4) of the Philox block with counter
   (proj, 0, w div 4, purpose 2). */
void or_weights(uint64_t seed, uint32_t proj, int64_t n, double lo, double hi, float* out) {
  uint32_t w[4];
  for (int64_t i = 0; i < n; ++i) {
    if ((i & 3) == 0) or_philox_words(seed, proj, 0u, 2u, (uint32_t)(i >> 2), 1, w);
    const double u = or_uniform(w[i & 3]);
    out[i] = (float)(lo + (hi - lo) * u);
  }
}
