/*
 * Swendsen-Wang update of the two-dimensional Ising model (test infrastructure;
 * see orc.h).  Sec. 4.1 of the paper benchmarks its union-find on this update:
 * classical spins on an L x L square lattice, a bond between equal nearest
 * neighbours is activated with probability p = 1 - exp(-2K), and every cluster
 * of activated bonds is flipped with probability 1/2.
 *
 * Plain restatement, one step after another: all bond draws, then clusters by
 * breadth-first search in increasing site order (so the site that starts a
 * search is the smallest of its cluster: every smaller site already belongs
 * to an earlier cluster), then one coin per cluster, then the estimators.
 * No union-find, nothing shared with the CUDA library.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "orc.h"

uint64_t orc_sw_threshold(double K) {
  /* T = round(2^32 p), p = 1 - e^{-2K}: a bond is active when its 32-bit
   * draw w satisfies w < T, i.e. with probability T / 2^32. */
  double p = -expm1(-2.0 * K);
  double x = floor(ldexp(p, 32) + 0.5);
  if (x <= 0.0) return 0;
  if (x >= 4294967296.0) return (uint64_t)1 << 32;
  return (uint64_t)x;
}

static void sw_draws(uint64_t seed, uint32_t sweep, int64_t i, uint32_t w[4]) {
  const uint32_t ctr[4] = {ORC_TAG_SWBOND << 24, (uint32_t)i, 0u, sweep};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, w);
}

static int sw_coin(uint64_t seed, uint32_t sweep, int64_t r) {
  /* 128 coins per Philox block: coin r is bit (r mod 128) of block r / 128. */
  const uint32_t ctr[4] = {ORC_TAG_SWFLIP << 24, (uint32_t)(r >> 7), 0u, sweep};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  int b = (int)(r & 127);
  return (int)((o[b >> 5] >> (b & 31)) & 1u);
}

int orc_sw_update(int64_t L, double K, uint64_t seed, uint32_t sweep, uint8_t *s,
                  int64_t *root_out, uint8_t *bond_out, orc_sw_record *rec) {
  if (L < 2) return -2;
  const int64_t N = L * L;
  const uint64_t T = orc_sw_threshold(K);
  uint8_t *bond = (uint8_t *)malloc((size_t)(2 * N));
  int64_t *root = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  uint8_t *coin = (uint8_t *)malloc((size_t)N);
  if (!bond || !root || !queue || !coin) {
    free(bond);
    free(root);
    free(queue);
    free(coin);
    return -1;
  }
  /* 1. bonds: R(i) = (i, right of i), D(i) = (i, below i); periodic */
  int64_t n_eq = 0, n_act = 0;
  for (int64_t i = 0; i < N; ++i) {
    const int64_t x = i % L, y = i / L;
    const int64_t r = y * L + (x + 1) % L, d = ((y + 1) % L) * L + x;
    uint32_t w[4];
    sw_draws(seed, sweep, i, w);
    const int eqr = s[i] == s[r], eqd = s[i] == s[d];
    bond[2 * i] = (uint8_t)(eqr && (uint64_t)w[0] < T);
    bond[2 * i + 1] = (uint8_t)(eqd && (uint64_t)w[1] < T);
    n_eq += eqr + eqd;
    n_act += bond[2 * i] + bond[2 * i + 1];
  }
  /* 2. clusters by breadth-first search from the smallest unvisited site */
  for (int64_t i = 0; i < N; ++i) root[i] = -1;
  int64_t n_cl = 0, max_c = 0;
  uint64_t sum_c2 = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (root[i] >= 0) continue;
    int64_t head = 0, tail = 0;
    root[i] = i;
    queue[tail++] = i;
    while (head < tail) {
      const int64_t v = queue[head++];
      const int64_t x = v % L, y = v / L;
      const int64_t nb[4] = {y * L + (x + 1) % L, ((y + 1) % L) * L + x,
                             y * L + (x + L - 1) % L, ((y + L - 1) % L) * L + x};
      const int on[4] = {bond[2 * v], bond[2 * v + 1], bond[2 * nb[2]], bond[2 * nb[3] + 1]};
      for (int k = 0; k < 4; ++k) {
        if (on[k] && root[nb[k]] < 0) {
          root[nb[k]] = i;
          queue[tail++] = nb[k];
        }
      }
    }
    /* tail = the cluster's size */
    ++n_cl;
    sum_c2 += (uint64_t)tail * (uint64_t)tail;
    if (tail > max_c) max_c = tail;
    coin[i] = (uint8_t)sw_coin(seed, sweep, i);
  }
  /* 3. flip every cluster whose coin is 1 */
  int64_t mag = 0;
  for (int64_t v = 0; v < N; ++v) {
    s[v] = (uint8_t)(s[v] ^ coin[root[v]]);
    mag += s[v] ? -1 : 1;
  }
  if (root_out)
    for (int64_t v = 0; v < N; ++v) root_out[v] = root[v];
  if (bond_out)
    for (int64_t k = 0; k < 2 * N; ++k) bond_out[k] = bond[k];
  rec->n_eq = n_eq;
  rec->n_act = n_act;
  rec->n_clusters = n_cl;
  rec->max_cluster = max_c;
  rec->sum_c2 = sum_c2;
  rec->mag = mag;
  /* E / N = -(1/N) sum over the 2N bonds of sigma_i sigma_j = (2N - 2 n_eq) / N */
  rec->energy = (double)(2 * N - 2 * n_eq) / (double)N;
  rec->chi = (double)sum_c2 / (double)N;
  free(bond);
  free(root);
  free(queue);
  free(coin);
  return 0;
}

int orc_sw_run(int64_t L, double K, uint64_t seed, uint32_t sweep0, int64_t n, uint8_t *s,
               orc_sw_record *recs) {
  for (int64_t t = 0; t < n; ++t) {
    int rc = orc_sw_update(L, K, seed, sweep0 + (uint32_t)t, s, NULL, NULL, recs + t);
    if (rc) return rc;
  }
  return 0;
}
