/*
 * Oracle utilities (test infrastructure; see orc.h).
 *
 * Philox4x32-10 is written from its published definition (Salmon et al., SC'11,
 * "Parallel random numbers: as easy as 1, 2, 3"): ten rounds of two 32x32->64
 * multiplications with a Weyl-sequence key schedule.  The Poisson thresholds are
 * the plain cumulative sum of the Poisson probabilities.  The geometry helpers
 * spell out the canonical cell order that numbers graph vertices.
 */
#include "orc.h"
#include <math.h>
#include <stdint.h>

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

void orc_poisson_thresholds(double mu, uint64_t T[ORC_KMAX]) {
  /* P(K = 0) = e^{-mu}, P(K = k) = P(K = k-1) * mu / k; T[k] = floor(2^64 CDF(k)). */
  double p = exp(-mu);
  double cdf = 0.0;
  for (int k = 0; k < ORC_KMAX; ++k) {
    if (k > 0) p = p * mu / (double)k;
    cdf += p;
    double x = ldexp(cdf, 64);
    if (x >= 18446744073709551616.0)
      T[k] = UINT64_MAX;
    else
      T[k] = (uint64_t)x;
  }
}

int64_t orc_nsub(const orc_params *p) { return p->L * p->Q; }
int64_t orc_nbond(const orc_params *p) { return p->L * p->Q * p->Q; }

int64_t orc_nwin(const orc_params *p) {
  double w = 16.0 / p->J;
  double q = ceil(p->beta / w);
  int64_t nw = (int64_t)q;
  return nw < 1 ? 1 : nw;
}

int64_t orc_ncell(const orc_params *p) { return orc_nbond(p) * orc_nwin(p); }

int64_t orc_cell_index(const orc_params *p, int64_t b, int64_t j) {
  /* Cells are grouped in blocks of ORC_TW windows; inside a block, bond-major. */
  int64_t NB = orc_nbond(p), NW = orc_nwin(p);
  int64_t blk = j / ORC_TW, jj = j % ORC_TW;
  int64_t tw = NW - blk * ORC_TW;
  if (tw > ORC_TW) tw = ORC_TW;
  return blk * NB * ORC_TW + b * tw + jj;
}

int orc_fixed_exponent(const orc_params *p) {
  /* F = 60 - ceil(log2(Q L beta)), so every loop's sum of lengths is < 2^60. */
  double total = (double)p->Q * (double)p->L * p->beta;
  int e;
  double m = frexp(total, &e);
  int cl = (m == 0.5) ? e - 1 : e;
  int F = 60 - cl;
  if (F < 0) F = 0;
  if (F > 62) F = 62;
  return F;
}

void orc_neel(const orc_params *p, uint8_t *s0, int64_t *op_ptr) {
  int64_t ns = orc_nsub(p), nc = orc_ncell(p);
  for (int64_t u = 0; u < ns; ++u) s0[u] = (uint8_t)((u / p->Q) & 1);
  for (int64_t c = 0; c <= nc; ++c) op_ptr[c] = 0;
}
