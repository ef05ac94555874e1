/*
 * Oracle: the random inputs xi of the KL expansion (Sec. 3.1.1, Eq. KL-expansion;
 * the workloads draw xi ~ N(0,1) from a counter-based Philox stream).
 * TEST INFRASTRUCTURE ONLY -- see oracle.h.
 *
 * Philox4x32-10 is written from its published definition (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds
 * of two 32x32->64 multiplies with the Weyl key schedule.
 *
 * The normal transform is Box-Muller (Box & Muller 1958).  Its ln and sin/cos
 * are written here from their Taylor / atanh series, using only IEEE-exact
 * operations (+ - * / sqrt, frexp) and compiled with -ffp-contract=off, so the
 * bits are fixed by the algorithm and not by any math library.
 *
 * Counter layout: for level pair l, sample id i, seed s and mode pair j
 *   counter = (j, lo32(i), hi32(i), l),  key = (lo32(s), hi32(s));
 * the four words give u1 = (k1 + 1) 2^-53 in (0,1] from words (0,1) and
 * u2 = k2 2^-53 in [0,1) from words (2,3), k = (w_a >> 5) 2^26 + (w_b >> 6);
 * xi[2j] = r cos(2 pi u2), xi[2j+1] = r sin(2 pi u2), r = sqrt(-2 ln u1).
 */
#include <math.h>
#include "oracle.h"

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)x0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)x2;
    uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
    uint32_t y1 = (uint32_t)p1;
    uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
    uint32_t y3 = (uint32_t)p0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ln x for finite x > 0:  x = f 2^e with f in [1/sqrt2, sqrt2), and
 * ln f = 2 atanh(s), s = (f-1)/(f+1), |s| <= 0.1716, summed to s^25. */
double or_log(double x) {
  int e;
  double f = frexp(x, &e);
  if (f < 0.70710678118654752440) { f = f * 2.0; e = e - 1; }
  double s = (f - 1.0) / (f + 1.0);
  double s2 = s * s;
  double p = 1.0 / 25.0;
  for (int j = 11; j >= 0; --j) p = p * s2 + 1.0 / (double)(2 * j + 1);
  double lnf = (2.0 * s) * p;
  return (double)e * 0.69314718055994530942 + lnf;
}

/* sin and cos of 2 pi u for u in [0,1): exact quadrant split of 4u, reflection
 * onto [0, pi/4], then the Maclaurin series to the phi^21 / phi^20 terms. */
void or_sincos_2pi(double u, double* s_out, double* c_out) {
  double t = 4.0 * u;
  int q = (int)t;
  double w = t - (double)q;
  int swap = 0;
  if (w > 0.5) { w = 1.0 - w; swap = 1; }
  double phi = w * 1.57079632679489661923;
  double p2 = phi * phi;
  /* coefficients (-1)^j/(2j+1)! and (-1)^j/(2j)!, j = 0..10 */
  double fs[11], fc[11];
  double fact = 1.0; /* running k! */
  for (int k = 0; k <= 21; ++k) {
    if (k > 0) fact = fact * (double)k;
    double coef = 1.0 / fact;
    int j = k / 2;
    double sg = (j % 2) ? -1.0 : 1.0;
    if (k % 2) fs[j] = sg * coef; else fc[j] = sg * coef;
  }
  double ps = fs[10], pc = fc[10];
  for (int j = 9; j >= 0; --j) { ps = ps * p2 + fs[j]; pc = pc * p2 + fc[j]; }
  double sp = phi * ps, cp = pc;
  double sq, cq;
  if (swap) { sq = cp; cq = sp; } else { sq = sp; cq = cp; }
  switch (q & 3) {
    case 0: *s_out = sq; *c_out = cq; break;
    case 1: *s_out = cq; *c_out = -sq; break;
    case 2: *s_out = -sq; *c_out = -cq; break;
    default: *s_out = -cq; *c_out = sq; break;
  }
}

void or_xi(uint64_t seed, int level, uint64_t sample_id, int M, double* xi) {
  const double two_m53 = 1.0 / 9007199254740992.0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; 2 * j < M; ++j) {
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)sample_id, (uint32_t)(sample_id >> 32),
                       (uint32_t)level};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    uint64_t k1 = ((uint64_t)(w[0] >> 5) << 26) | (uint64_t)(w[1] >> 6);
    uint64_t k2 = ((uint64_t)(w[2] >> 5) << 26) | (uint64_t)(w[3] >> 6);
    double u1 = (double)(k1 + 1) * two_m53;
    double u2 = (double)k2 * two_m53;
    double r = sqrt(-2.0 * or_log(u1));
    double sn, cs;
    or_sincos_2pi(u2, &sn, &cs);
    xi[2 * j] = r * cs;
    if (2 * j + 1 < M) xi[2 * j + 1] = r * sn;
  }
}

/* The paper's uniform KL inputs psi_k ~ U(-1, 1) (Sec. 3.1.1) from the same
 * Philox words as or_xi: psi_2j = 2 u1 - 1 in (-1, 1], psi_2j+1 = 2 u2 - 1 in
 * [-1, 1), exact in binary arithmetic. */
void or_psi_uniform(uint64_t seed, int level, uint64_t sample_id, int M, double* psi) {
  const double two_m52 = 1.0 / 4503599627370496.0;
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (int j = 0; 2 * j < M; ++j) {
    uint32_t ctr[4] = {(uint32_t)j, (uint32_t)sample_id, (uint32_t)(sample_id >> 32),
                       (uint32_t)level};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    uint64_t k1 = ((uint64_t)(w[0] >> 5) << 26) | (uint64_t)(w[1] >> 6);
    uint64_t k2 = ((uint64_t)(w[2] >> 5) << 26) | (uint64_t)(w[3] >> 6);
    psi[2 * j] = (double)(k1 + 1) * two_m52 - 1.0;
    if (2 * j + 1 < M) psi[2 * j + 1] = (double)k2 * two_m52 - 1.0;
  }
}
