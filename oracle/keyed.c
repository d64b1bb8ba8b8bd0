/*
 * Keyed form of one loop-cluster update (test infrastructure; see orc.h).
 *
 * Steps, in the order of the Monte Carlo step of Sec. 2:
 *  1. labeling (rules i-iii, Sec. 2): every old off-diagonal operator is a
 *     horizontal graph; on each bond and each time window, candidate graphs form
 *     a Poisson process of rate J/2 (rule ii in the continuum limit) and a
 *     candidate is kept iff the two spins of the bond are antiparallel there
 *     (rule iii otherwise).  Candidate counts and positions come from Philox
 *     keyed by (seed; tag, draw, bond, window, sweep).
 *  2. cluster identification: the world line is cut at every graph leg into
 *     pieces; a horizontal graph joins its two lower legs and its two upper legs
 *     (Fig. 1); loops are found by walking this 2-regular piece graph.
 *  3. each loop is flipped with probability 1/2 (Sec. 2), the coin drawn from
 *     Philox keyed by the loop's smallest vertex id.
 *  4. s(tau=0) and the operator list are rewritten (step 7 of the MC step).
 *  5. measurement: energy from the number of graphs; staggered susceptibility
 *     and chi(pi + 2 pi/L) from the loop lengths (improved estimators).
 * For S=1 (Q=2) each site holds two subspins and each bond four sub-bonds
 * (Sec. 5); at tau=0 the subspins are joined by a permutation drawn uniformly
 * among those that map every top spin onto an equal bottom spin.
 */
#include "orc.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double tau;
  int64_t bond;
} ev_t;

typedef struct {
  double tau;
  int64_t bond, cell, id;
  uint8_t flag;
} vtx_t;

typedef struct {
  uint64_t u53;
  int k;
  double tau;
} cand_t;

static void bond_ends(const orc_params *p, int64_t b, int64_t *ul, int64_t *ur) {
  int64_t Q = p->Q;
  int64_t i = b / (Q * Q), a = (b / Q) % Q, a2 = b % Q;
  *ul = i * Q + a;
  *ur = ((i + 1) % p->L) * Q + a2;
}

static int ev_cmp(const void *x, const void *y) {
  const ev_t *a = (const ev_t *)x, *b = (const ev_t *)y;
  if (a->tau < b->tau) return -1;
  if (a->tau > b->tau) return 1;
  return (a->bond > b->bond) - (a->bond < b->bond);
}

/* Number of events with key (tau_e, bond_e) < (tau, bond). */
static int64_t count_before(const ev_t *e, int64_t n, double tau, int64_t bond) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    int less = (e[mid].tau < tau) || (e[mid].tau == tau && e[mid].bond < bond);
    if (less)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

static int cand_cmp(const void *x, const void *y) {
  const cand_t *a = (const cand_t *)x, *b = (const cand_t *)y;
  if (a->u53 != b->u53) return a->u53 < b->u53 ? -1 : 1;
  return (a->k > b->k) - (a->k < b->k);
}

static const vtx_t *g_vtx; /* for the leg-end comparator */
static int leg_cmp(const void *x, const void *y) {
  int64_t a = *(const int64_t *)x, b = *(const int64_t *)y;
  if (g_vtx[a].tau < g_vtx[b].tau) return -1;
  if (g_vtx[a].tau > g_vtx[b].tau) return 1;
  return (a > b) - (a < b);
}

static int coin(const orc_params *p, uint32_t tag, int64_t index, uint32_t sweep) {
  uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  uint32_t ctr[4] = {tag << 24, (uint32_t)(index >> 7), 0u, sweep};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  int bit = (int)(index & 127);
  return (int)((out[bit >> 5] >> (bit & 31)) & 1u);
}

static int poisson_sample(const uint64_t T[ORC_KMAX], uint64_t U) {
  int K = 0;
  while (K < ORC_KMAX - 1 && U >= T[K]) ++K;
  return K;
}

/*
 * Labeling of one cell (bond b, window j): the old operators of the cell are
 * horizontal graphs (rule i); candidates of a Poisson process of rate J/2 are
 * kept where the bond's spins are antiparallel (rules ii, iii).  ev_l / ev_r
 * are the old operators touching the bond's left / right subsite, sorted by
 * (tau, bond).  Writes the cell's vertices in (tau, old-first, draw) order and
 * returns their number.
 */
static int64_t label_cell(const orc_params *p, uint32_t sweep, int64_t b, int64_t j,
                          const uint8_t *s0, const ev_t *ev_l, int64_t n_l, const ev_t *ev_r,
                          int64_t n_r, const int64_t *op_ptr, const double *op_tau,
                          const uint64_t *T_full, const uint64_t *T_last, double *out_tau,
                          uint8_t *out_flag) {
  const int64_t NW = orc_nwin(p);
  const double beta = p->beta, w = 16.0 / p->J;
  const uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  int64_t ul, ur;
  bond_ends(p, b, &ul, &ur);
  const int64_t c = orc_cell_index(p, b, j);
  double t0 = (double)j * w;
  double t_end = (j == NW - 1) ? beta : (double)(j + 1) * w;
  double d = t_end - t0;
  const uint64_t *T = (j == NW - 1) ? T_last : T_full;
  cand_t cand[ORC_KMAX];
  /* Draws: call 0 gives K and candidate 0; call m >= 1 gives 2m-1, 2m. */
  uint32_t ctr[4] = {(ORC_TAG_INSERT << 24) | 0u, (uint32_t)b, (uint32_t)j, sweep};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  uint64_t U = (uint64_t)out[0] | ((uint64_t)out[1] << 32);
  int K = poisson_sample(T, U);
  int nk = 0;
  for (int k = 0; k < K; ++k) {
    uint64_t bits;
    if (k == 0) {
      bits = (uint64_t)out[2] | ((uint64_t)out[3] << 32);
    } else {
      uint32_t m = (uint32_t)((k + 1) / 2);
      uint32_t c2[4] = {(ORC_TAG_INSERT << 24) | m, (uint32_t)b, (uint32_t)j, sweep};
      uint32_t o2[4];
      orc_philox4x32_10(c2, key, o2);
      bits = (k & 1) ? ((uint64_t)o2[0] | ((uint64_t)o2[1] << 32))
                     : ((uint64_t)o2[2] | ((uint64_t)o2[3] << 32));
    }
    uint64_t u53 = bits >> 11;
    double tau = fma(d, ldexp((double)u53, -53), t0);
    if (!(tau < t_end)) continue;
    /* Rule ii/iii: keep iff the bond's spins are antiparallel at tau. */
    int64_t pl = count_before(ev_l, n_l, tau, b);
    int64_t pr = count_before(ev_r, n_r, tau, b);
    int sl = s0[ul] ^ (int)(pl & 1), sr = s0[ur] ^ (int)(pr & 1);
    if (sl == sr) continue;
    cand[nk].u53 = u53;
    cand[nk].k = k;
    cand[nk].tau = tau;
    ++nk;
  }
  qsort(cand, (size_t)nk, sizeof(cand_t), cand_cmp);
  /* Merge with the cell's old operators; an old one goes first at equal tau. */
  int64_t q = op_ptr[c], qe = op_ptr[c + 1], r = 0;
  int ki = 0;
  while (q < qe || ki < nk) {
    if (q < qe && (ki >= nk || op_tau[q] <= cand[ki].tau)) {
      out_tau[r] = op_tau[q++];
      out_flag[r] = 1;
    } else {
      out_tau[r] = cand[ki++].tau;
      out_flag[r] = 0;
    }
    ++r;
  }
  return r;
}

static int64_t gather_events(const orc_params *p, int64_t u, const int64_t *op_ptr,
                             const double *op_tau, ev_t **out) {
  /* Old operators on the bonds touching subsite u, sorted by (tau, bond). */
  const int64_t NW = orc_nwin(p), Q = p->Q, i = u / Q, a = u % Q;
  int64_t cnt = 0, cap = 1024;
  ev_t *e = (ev_t *)malloc(sizeof(ev_t) * (size_t)cap);
  for (int64_t k = 0; k < 2 * Q; ++k) {
    /* bonds (i, a, k) with u at the left end, bonds (i-1, k-Q, a) at the right */
    int64_t b = (k < Q) ? i * Q * Q + a * Q + k : ((i - 1 + p->L) % p->L) * Q * Q + (k - Q) * Q + a;
    for (int64_t j = 0; j < NW; ++j) {
      int64_t c = orc_cell_index(p, b, j);
      for (int64_t q = op_ptr[c]; q < op_ptr[c + 1]; ++q) {
        if (cnt == cap) {
          cap *= 2;
          e = (ev_t *)realloc(e, sizeof(ev_t) * (size_t)cap);
        }
        e[cnt].tau = op_tau[q];
        e[cnt].bond = b;
        ++cnt;
      }
    }
  }
  qsort(e, (size_t)cnt, sizeof(ev_t), ev_cmp);
  *out = e;
  return cnt;
}

int orc_keyed_cell(const orc_params *p, uint32_t sweep, const uint8_t *s0, const int64_t *op_ptr,
                   const double *op_tau, int64_t b, int64_t j, double *out_tau, uint8_t *out_flag,
                   int64_t cap, int64_t *n_out) {
  const int64_t NW = orc_nwin(p);
  const double w = 16.0 / p->J;
  uint64_t T_full[ORC_KMAX], T_last[ORC_KMAX];
  orc_poisson_thresholds(ORC_CELL_MEAN, T_full);
  {
    double t0 = (double)(NW - 1) * w;
    double d = p->beta - t0;
    orc_poisson_thresholds(d > 0.0 ? p->J * d * 0.5 : 0.0, T_last);
  }
  int64_t ul, ur;
  bond_ends(p, b, &ul, &ur);
  ev_t *el, *er;
  int64_t nl = gather_events(p, ul, op_ptr, op_tau, &el);
  int64_t nr = gather_events(p, ur, op_ptr, op_tau, &er);
  const int64_t c = orc_cell_index(p, b, j);
  const int64_t nold = op_ptr[c + 1] - op_ptr[c];
  double *t = (double *)malloc(sizeof(double) * (size_t)(nold + ORC_KMAX + 1));
  uint8_t *f = (uint8_t *)malloc((size_t)(nold + ORC_KMAX + 1));
  int64_t m = label_cell(p, sweep, b, j, s0, el, nl, er, nr, op_ptr, op_tau, T_full, T_last, t, f);
  int rc = 0;
  if (m > cap) {
    rc = -1;
  } else {
    memcpy(out_tau, t, sizeof(double) * (size_t)m);
    memcpy(out_flag, f, (size_t)m);
  }
  *n_out = m;
  free(t);
  free(f);
  free(el);
  free(er);
  return rc;
}

typedef unsigned __int128 u128;

/* floor((v c + 2^31) / 2^32): v c / 2^32 rounded to nearest, ties up (exact). */
/* Phase factors for the temporal moment (Sec. 5: the gap from the
   imaginary-time moment of the staggered correlation). */
#define PH_BITS 16
static int64_t ph_cos[(1 << PH_BITS) + 1], ph_sin[(1 << PH_BITS) + 1];
static int ph_ready;

static void ph_init(void) {
  if (ph_ready) return;
  for (int64_t k = 0; k <= (1 << PH_BITS); ++k) {
    double ang = (2.0 * M_PI * (double)k) / (double)(1 << PH_BITS);
    ph_cos[k] = llrint(ldexp(cos(ang), 30));
    ph_sin[k] = llrint(ldexp(sin(ang), 30));
  }
  ph_ready = 1;
}

static int64_t floor_div_2_32(int64_t x) { /* floor(x / 2^32) */
  return x >= 0 ? x / 4294967296LL : -((-x + 4294967295LL) / 4294967296LL);
}

uint64_t orc_phase_recip(int64_t qbeta, int *sh) {
  int k = 63;
  while (k > 0 && !(((uint64_t)qbeta >> k) & 1u)) --k;
  *sh = k; /* 2^k <= qbeta < 2^(k+1) */
  return (uint64_t)(((((u128)1) << (64 + k)) - 1) / (u128)(uint64_t)qbeta);
}

void orc_phase(uint64_t q, uint64_t R, int sh, int64_t *c, int64_t *s) {
  ph_init();
  uint64_t X = (uint64_t)(((u128)q * R) >> sh); /* fraction of the period, modulo 2^64 */
  uint64_t k = X >> (64 - PH_BITS);
  int64_t t = (int64_t)((X >> (32 - PH_BITS)) & 0xffffffffULL);
  *c = ph_cos[k] + floor_div_2_32((ph_cos[k + 1] - ph_cos[k]) * t);
  *s = ph_sin[k] + floor_div_2_32((ph_sin[k + 1] - ph_sin[k]) * t);
}

static int64_t mul_q32(int64_t v, int64_t c) {
  __int128 p = (__int128)v * (__int128)c + ((__int128)1 << 31);
  return (int64_t)(p >> 32);
}

int orc_keyed_update(const orc_params *p, uint32_t sweep, const uint8_t *s0,
                     const int64_t *op_ptr, const double *op_tau, uint8_t *s0_out,
                     int64_t *op_ptr_out, double *op_tau_out, int64_t op_cap,
                     orc_record *rec, int64_t cap_vtx, double *vtx_tau_o, uint8_t *vtx_flag_o,
                     int64_t *vtx_bond_o, int64_t *vtx_pl_o, int64_t *vtx_pr_o,
                     int64_t *vtx_root_o) {
  const int64_t L = p->L, Q = p->Q, NS = orc_nsub(p), NB = orc_nbond(p);
  const int64_t NW = orc_nwin(p), NC = orc_ncell(p);
  const double beta = p->beta, w = 16.0 / p->J;
  int rc = 0;

  /* Windows: [j w, (j+1) w) and the last one [(NW-1) w, beta). */
  uint64_t T_full[ORC_KMAX], T_last[ORC_KMAX];
  orc_poisson_thresholds(ORC_CELL_MEAN, T_full);
  {
    double t0 = (double)(NW - 1) * w;
    double d = beta - t0;
    double mu = d > 0.0 ? p->J * d * 0.5 : 0.0;
    orc_poisson_thresholds(mu, T_last);
  }

  /* Old operators: per-subsite event lists sorted by (tau, bond). */
  int64_t n_old = op_ptr[NC];
  int64_t *ev_cnt = (int64_t *)calloc((size_t)NS + 1, sizeof(int64_t));
  for (int64_t b = 0; b < NB; ++b) {
    int64_t ul, ur;
    bond_ends(p, b, &ul, &ur);
    for (int64_t j = 0; j < NW; ++j) {
      int64_t c = orc_cell_index(p, b, j);
      int64_t m = op_ptr[c + 1] - op_ptr[c];
      ev_cnt[ul + 1] += m;
      ev_cnt[ur + 1] += m;
    }
  }
  for (int64_t u = 0; u < NS; ++u) ev_cnt[u + 1] += ev_cnt[u];
  ev_t *ev = (ev_t *)malloc(sizeof(ev_t) * (size_t)(ev_cnt[NS] + 1));
  int64_t *ev_fill = (int64_t *)calloc((size_t)NS, sizeof(int64_t));
  for (int64_t b = 0; b < NB; ++b) {
    int64_t ul, ur;
    bond_ends(p, b, &ul, &ur);
    for (int64_t j = 0; j < NW; ++j) {
      int64_t c = orc_cell_index(p, b, j);
      for (int64_t q = op_ptr[c]; q < op_ptr[c + 1]; ++q) {
        ev_t e = {op_tau[q], b};
        ev[ev_cnt[ul] + ev_fill[ul]++] = e;
        ev[ev_cnt[ur] + ev_fill[ur]++] = e;
      }
    }
  }
  for (int64_t u = 0; u < NS; ++u)
    qsort(ev + ev_cnt[u], (size_t)(ev_cnt[u + 1] - ev_cnt[u]), sizeof(ev_t), ev_cmp);

  /* 1. Labeling: build each cell's vertex list in canonical cell order. */
  int64_t vcap = n_old + 1024, n = 0;
  vtx_t *vtx = (vtx_t *)malloc(sizeof(vtx_t) * (size_t)vcap);
  int64_t max_cell = 0;
  for (int64_t c = 0; c < NC; ++c)
    if (op_ptr[c + 1] - op_ptr[c] > max_cell) max_cell = op_ptr[c + 1] - op_ptr[c];
  double *cell_tau = (double *)malloc(sizeof(double) * (size_t)(max_cell + ORC_KMAX));
  uint8_t *cell_flag = (uint8_t *)malloc((size_t)(max_cell + ORC_KMAX));
  int64_t nblk = (NW + ORC_TW - 1) / ORC_TW;
  int64_t c_expect = 0;
  for (int64_t blk = 0; blk < nblk; ++blk) {
    int64_t tw = NW - blk * ORC_TW;
    if (tw > ORC_TW) tw = ORC_TW;
    for (int64_t b = 0; b < NB; ++b) {
      int64_t ul, ur;
      bond_ends(p, b, &ul, &ur);
      for (int64_t jj = 0; jj < tw; ++jj) {
        int64_t j = blk * ORC_TW + jj;
        int64_t c = orc_cell_index(p, b, j);
        if (c != c_expect) { rc = -3; goto done; }
        ++c_expect;
        int64_t m = label_cell(p, sweep, b, j, s0, ev + ev_cnt[ul], ev_cnt[ul + 1] - ev_cnt[ul],
                               ev + ev_cnt[ur], ev_cnt[ur + 1] - ev_cnt[ur], op_ptr, op_tau, T_full,
                               T_last, cell_tau, cell_flag);
        if (n + m > vcap) {
          while (n + m > vcap) vcap *= 2;
          vtx = (vtx_t *)realloc(vtx, sizeof(vtx_t) * (size_t)vcap);
        }
        for (int64_t r = 0; r < m; ++r) {
          vtx[n].tau = cell_tau[r];
          vtx[n].flag = cell_flag[r];
          vtx[n].bond = b;
          vtx[n].cell = c;
          vtx[n].id = n;
          ++n;
        }
      }
    }
  }

  /* 2. Leg ends per subsite, ordered by (tau, vertex id). */
  int64_t *leg_cnt = (int64_t *)calloc((size_t)NS + 1, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) {
    int64_t ul, ur;
    bond_ends(p, vtx[v].bond, &ul, &ur);
    leg_cnt[ul + 1]++;
    leg_cnt[ur + 1]++;
  }
  for (int64_t u = 0; u < NS; ++u) leg_cnt[u + 1] += leg_cnt[u];
  int64_t *leg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * n + 1));
  int64_t *leg_fill = (int64_t *)calloc((size_t)NS, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) {
    int64_t ul, ur;
    bond_ends(p, vtx[v].bond, &ul, &ur);
    leg[leg_cnt[ul] + leg_fill[ul]++] = v;
    leg[leg_cnt[ur] + leg_fill[ur]++] = v;
  }
  g_vtx = vtx;
  for (int64_t u = 0; u < NS; ++u)
    qsort(leg + leg_cnt[u], (size_t)(leg_cnt[u + 1] - leg_cnt[u]), sizeof(int64_t), leg_cmp);
  /* Position of each vertex in its two subsites' lists. */
  int64_t *pos_l = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int64_t *pos_r = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  for (int64_t u = 0; u < NS; ++u) {
    for (int64_t m = leg_cnt[u]; m < leg_cnt[u + 1]; ++m) {
      int64_t v = leg[m], ul, ur;
      bond_ends(p, vtx[v].bond, &ul, &ur);
      if (ul == u) pos_l[v] = m - leg_cnt[u];
      if (ur == u) pos_r[v] = m - leg_cnt[u];
    }
  }

  /* Cut at tau = 0: permutation of subspins per site (identity for Q = 1),
     drawn uniformly among those that join every top to a bottom of the same
     spin (heat bath of the symmetrization, Sec. 5). */
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS); /* top subsite -> bottom subsite */
  for (int64_t i = 0; i < L; ++i) {
    if (Q == 1) {
      perm[i] = i;
      continue;
    }
    if (Q > 2) {
      /* Tops and bottoms of spin 1, then of spin 0, in subspin order; a
         uniform shuffle of each bottom list (Fisher-Yates from the last
         place down, place j drawn as floor(w (j+1) / 2^32) with w the next
         word of Philox(ctr = ((ORC_TAG_PERM << 24) | 1, i, 0, sweep))); the
         m-th top of each spin continues into the m-th shuffled bottom. */
      int64_t tops[2][ORC_QMAX], bots[2][ORC_QMAX];
      int nt[2] = {0, 0}, nb[2] = {0, 0};
      for (int a = 0; a < Q; ++a) {
        int64_t u = i * Q + a;
        int t = s0[u] ^ (int)((ev_cnt[u + 1] - ev_cnt[u]) & 1);
        int g = t ? 0 : 1; /* group 0: spin 1 */
        tops[g][nt[g]++] = a;
        int gb = s0[u] ? 0 : 1;
        bots[gb][nb[gb]++] = a;
      }
      if (nt[0] != nb[0]) {
        rc = -2;
        goto done2;
      }
      uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
      uint32_t ctr[4] = {(ORC_TAG_PERM << 24) | 1u, (uint32_t)i, 0u, sweep};
      uint32_t w[4];
      orc_philox4x32_10(ctr, key, w);
      int d = 0;
      for (int g = 0; g < 2; ++g) {
        for (int j = nb[g] - 1; j >= 1; --j) {
          int r = (int)(((uint64_t)w[d++] * (uint64_t)(j + 1)) >> 32);
          int64_t tmp = bots[g][j];
          bots[g][j] = bots[g][r];
          bots[g][r] = tmp;
        }
        for (int m = 0; m < nt[g]; ++m) perm[i * Q + tops[g][m]] = i * Q + bots[g][m];
      }
      continue;
    }
    int64_t u0 = i * Q, u1 = i * Q + 1;
    int t0 = s0[u0] ^ (int)((ev_cnt[u0 + 1] - ev_cnt[u0]) & 1);
    int t1 = s0[u1] ^ (int)((ev_cnt[u1 + 1] - ev_cnt[u1]) & 1);
    int ok_id = (t0 == s0[u0]) && (t1 == s0[u1]);
    int ok_sw = (t0 == s0[u1]) && (t1 == s0[u0]);
    int swap;
    if (ok_id && ok_sw)
      swap = coin(p, ORC_TAG_PERM, i, sweep);
    else if (ok_sw)
      swap = 1;
    else if (ok_id)
      swap = 0;
    else {
      rc = -2;
      goto done2;
    }
    perm[u0] = swap ? u1 : u0;
    perm[u1] = swap ? u0 : u1;
  }

  {
    /* Pieces: subsite u with k legs has pieces 0..k; piece m runs from leg m-1
       (or the cut) to leg m (or the cut). */
    int64_t *poff = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NS + 1));
    poff[0] = 0;
    for (int64_t u = 0; u < NS; ++u) poff[u + 1] = poff[u] + (leg_cnt[u + 1] - leg_cnt[u]) + 1;
    int64_t NP = poff[NS];
    int64_t *bot_v = (int64_t *)malloc(sizeof(int64_t) * (size_t)NP);
    int64_t *top_v = (int64_t *)malloc(sizeof(int64_t) * (size_t)NP);
    int64_t *psub = (int64_t *)malloc(sizeof(int64_t) * (size_t)NP);
    int64_t *partner = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * NP));
    for (int64_t u = 0; u < NS; ++u) {
      int64_t k = leg_cnt[u + 1] - leg_cnt[u];
      for (int64_t m = 0; m <= k; ++m) {
        int64_t pc = poff[u] + m;
        bot_v[pc] = (m == 0) ? -1 : leg[leg_cnt[u] + m - 1];
        top_v[pc] = (m == k) ? -1 : leg[leg_cnt[u] + m];
        psub[pc] = u;
      }
    }
    for (int64_t e = 0; e < 2 * NP; ++e) partner[e] = -1;
    for (int64_t v = 0; v < n; ++v) {
      int64_t ul, ur;
      bond_ends(p, vtx[v].bond, &ul, &ur);
      int64_t bl = poff[ul] + pos_l[v], br = poff[ur] + pos_r[v]; /* pieces below */
      partner[2 * bl + 1] = 2 * br + 1;                          /* lower legs */
      partner[2 * br + 1] = 2 * bl + 1;
      partner[2 * (bl + 1)] = 2 * (br + 1); /* upper legs */
      partner[2 * (br + 1)] = 2 * (bl + 1);
    }
    for (int64_t u = 0; u < NS; ++u) {
      int64_t last = poff[u + 1] - 1, first = poff[perm[u]];
      partner[2 * last + 1] = 2 * first;
      partner[2 * first] = 2 * last + 1;
    }
    for (int64_t e = 0; e < 2 * NP; ++e)
      if (partner[e] < 0) { rc = -4; }
    int64_t *loop = (int64_t *)malloc(sizeof(int64_t) * (size_t)NP);
    for (int64_t q = 0; q < NP; ++q) loop[q] = -1;
    int64_t nloop = 0;
    int64_t *canon = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NP + 1));
    int *is_free = (int *)malloc(sizeof(int) * (size_t)(NP + 1));
    int64_t *npieces = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NP + 1));
    if (rc == 0) {
      for (int64_t q0 = 0; q0 < NP; ++q0) {
        if (loop[q0] >= 0) continue;
        int64_t id = nloop++;
        int64_t best_v = -1, best_s = -1, cnt = 0;
        int64_t entry = 2 * q0;
        int64_t guard = 0;
        do {
          int64_t q = entry / 2;
          if (loop[q] >= 0) { rc = -5; break; }
          loop[q] = id;
          ++cnt;
          if (bot_v[q] >= 0 && (best_v < 0 || bot_v[q] < best_v)) best_v = bot_v[q];
          if (best_s < 0 || psub[q] < best_s) best_s = psub[q];
          entry = partner[entry ^ 1];
          if (++guard > 2 * NP + 2) { rc = -6; break; }
        } while (entry != 2 * q0);
        if (rc) break;
        is_free[id] = best_v < 0;
        canon[id] = best_v >= 0 ? best_v : best_s;
        npieces[id] = cnt;
      }
    }
    if (rc == 0) {
      /* 3. One coin per loop. */
      uint8_t *flip = (uint8_t *)malloc((size_t)nloop + 1);
      int64_t n_free = 0;
      for (int64_t l = 0; l < nloop; ++l) {
        flip[l] = (uint8_t)coin(p, is_free[l] ? ORC_TAG_FREE : ORC_TAG_FLIP, canon[l], sweep);
        n_free += is_free[l];
      }
      /* 4. Rewrite: s(0) and the operators. */
      for (int64_t u = 0; u < NS; ++u) s0_out[u] = (uint8_t)(s0[u] ^ flip[loop[poff[u]]]);
      uint8_t *newflag = (uint8_t *)malloc((size_t)n + 1);
      for (int64_t v = 0; v < n; ++v) {
        int64_t ul, ur;
        bond_ends(p, vtx[v].bond, &ul, &ur);
        int64_t below = poff[ul] + pos_l[v], above = below + 1;
        newflag[v] = (uint8_t)(vtx[v].flag ^ flip[loop[below]] ^ flip[loop[above]]);
      }
      for (int64_t c = 0; c <= NC; ++c) op_ptr_out[c] = 0;
      int64_t n_new = 0;
      for (int64_t v = 0; v < n; ++v) {
        if (!newflag[v]) continue;
        op_ptr_out[vtx[v].cell + 1]++;
        if (n_new < op_cap) op_tau_out[n_new] = vtx[v].tau;
        ++n_new;
      }
      for (int64_t c = 0; c < NC; ++c) op_ptr_out[c + 1] += op_ptr_out[c];
      if (n_new > op_cap) rc = -1;

      /* 5. Measurement: per loop, fixed-point sums over fragments.  Times are
         measured in ticks of 2^-F: q(x) = rint(x 2^F); a fragment from time a up
         to time b across c cuts at tau = beta has length q(b) - q(a) + c q(beta),
         and contributes rint(len cos(kx) 2^32) / 2^32 (ties up) to the Fourier
         sums, with cos(kx) itself rounded to 32 fractional bits. */
      int F = orc_fixed_exponent(p);
      const int64_t qbeta = llrint(ldexp(beta, F));
      int64_t *Wq = (int64_t *)calloc((size_t)nloop + 1, sizeof(int64_t));
      int64_t *Cq = (int64_t *)calloc((size_t)nloop + 1, sizeof(int64_t));
      int64_t *Sq = (int64_t *)calloc((size_t)nloop + 1, sizeof(int64_t));
      int64_t *Zr = (int64_t *)calloc((size_t)nloop + 1, sizeof(int64_t));
      int64_t *Zi = (int64_t *)calloc((size_t)nloop + 1, sizeof(int64_t));
      int rsh;
      const uint64_t rbeta = orc_phase_recip(qbeta, &rsh);
      int64_t *cx = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
      int64_t *sx = (int64_t *)malloc(sizeof(int64_t) * (size_t)L);
      for (int64_t x = 0; x < L; ++x) {
        double ang = (2.0 * M_PI * (double)x) / (double)L;
        cx[x] = llrint(ldexp(cos(ang), 32));
        sx[x] = llrint(ldexp(sin(ang), 32));
      }
      for (int64_t v = 0; v < n; ++v) {
        int64_t ul, ur;
        bond_ends(p, vtx[v].bond, &ul, &ur);
        for (int side = 0; side < 2; ++side) {
          int64_t u = side ? ur : ul;
          int64_t q = poff[u] + (side ? pos_r[v] : pos_l[v]) + 1; /* piece above v */
          int64_t cross = 0, guard = 0;
          while (top_v[q] < 0) {
            ++cross;
            q = partner[2 * q + 1] / 2;
            if (++guard > NS + 2) { rc = -7; break; }
          }
          int64_t qt = llrint(ldexp(vtx[top_v[q]].tau, F)), qb = llrint(ldexp(vtx[v].tau, F));
          int64_t len = qt - qb + cross * qbeta;
          int64_t x = u / Q;
          int64_t l = loop[poff[u] + (side ? pos_r[v] : pos_l[v]) + 1];
          Wq[l] += len;
          Cq[l] += mul_q32(len, cx[x]);
          Sq[l] += mul_q32(len, sx[x]);
          /* int over the fragment of e^{i w1 t} dt = (e(top) - e(bottom)) / (i w1):
             the same across the cut, since e(t + beta) = e(t) */
          int64_t ct, st_, cb, sb;
          orc_phase((uint64_t)qt, rbeta, rsh, &ct, &st_);
          orc_phase((uint64_t)qb, rbeta, rsh, &cb, &sb);
          Zr[l] += ct - cb;
          Zi[l] += st_ - sb;
        }
      }
      for (int64_t l = 0; l < nloop; ++l) {
        if (!is_free[l]) continue;
        int64_t len = npieces[l] * qbeta;
        int64_t x = canon[l] / Q;
        Wq[l] += len;
        Cq[l] += mul_q32(len, cx[x]);
        Sq[l] += mul_q32(len, sx[x]);
      }
      /* (vertex-free loops are whole periods: their temporal sums are 0) */
      u128 sw2 = 0, sf2 = 0, sz2 = 0;
      for (int64_t l = 0; l < nloop; ++l) {
        uint64_t aw = (uint64_t)(Wq[l] < 0 ? -Wq[l] : Wq[l]);
        uint64_t ac = (uint64_t)(Cq[l] < 0 ? -Cq[l] : Cq[l]);
        uint64_t as = (uint64_t)(Sq[l] < 0 ? -Sq[l] : Sq[l]);
        uint64_t ar = (uint64_t)(Zr[l] < 0 ? -Zr[l] : Zr[l]);
        uint64_t ai = (uint64_t)(Zi[l] < 0 ? -Zi[l] : Zi[l]);
        sw2 += (u128)aw * aw;
        sf2 += (u128)ac * ac + (u128)as * as;
        sz2 += (u128)ar * ar + (u128)ai * ai;
      }
      if (rec) {
        rec->n = n;
        rec->n_off_old = n_old;
        rec->n_off_new = n_new;
        rec->n_free = n_free;
        rec->n_clusters = nloop;
        rec->n_seg = 2 * n + n_free;
        rec->F = F;
        rec->pad = 0;
        rec->sw2_lo = (uint64_t)sw2;
        rec->sw2_hi = (uint64_t)(sw2 >> 64);
        rec->sf2_lo = (uint64_t)sf2;
        rec->sf2_hi = (uint64_t)(sf2 >> 64);
        rec->sz2_lo = (uint64_t)sz2;
        rec->sz2_hi = (uint64_t)(sz2 >> 64);
        double dsw = (double)rec->sw2_hi * 18446744073709551616.0 + (double)rec->sw2_lo;
        double dsf = (double)rec->sf2_hi * 18446744073709551616.0 + (double)rec->sf2_lo;
        double dsz = (double)rec->sz2_hi * 18446744073709551616.0 + (double)rec->sz2_lo;
        rec->energy = (double)(Q * Q) * p->J * 0.25 - (double)n / (beta * (double)L);
        rec->chi_s = ldexp(dsw, -2 * F) / (4.0 * beta * (double)L);
        rec->chi_q = ldexp(dsf, -2 * F) / (4.0 * beta * (double)L);
        /* |int e^{i w1 t} dt|^2 = |Z|^2 2^-60 / w1^2, w1 = 2 pi / beta */
        rec->chi_w = ldexp(dsz, -60) * beta / (16.0 * M_PI * M_PI * (double)L);
      }
      /* Debug graph export. */
      if (cap_vtx >= n) {
        for (int64_t v = 0; v < n; ++v) {
          int64_t ul, ur;
          bond_ends(p, vtx[v].bond, &ul, &ur);
          if (vtx_tau_o) vtx_tau_o[v] = vtx[v].tau;
          if (vtx_flag_o) vtx_flag_o[v] = vtx[v].flag;
          if (vtx_bond_o) vtx_bond_o[v] = vtx[v].bond;
          for (int side = 0; side < 2; ++side) {
            int64_t u = side ? ur : ul;
            int64_t q = poff[u] + (side ? pos_r[v] : pos_l[v]); /* piece below v */
            int64_t guard = 0;
            while (bot_v[q] < 0) {
              q = partner[2 * q] / 2;
              if (++guard > NS + 2) break;
            }
            int64_t node = bot_v[q];
            if (side == 0 && vtx_pl_o) vtx_pl_o[v] = node;
            if (side == 1 && vtx_pr_o) vtx_pr_o[v] = node;
          }
          if (vtx_root_o) vtx_root_o[v] = canon[loop[poff[ul] + pos_l[v] + 1]];
        }
      } else if (vtx_tau_o || vtx_flag_o || vtx_bond_o || vtx_pl_o || vtx_pr_o || vtx_root_o) {
        if (rc == 0) rc = -1;
      }
      free(Wq);
      free(Cq);
      free(Sq);
      free(Zr);
      free(Zi);
      free(cx);
      free(sx);
      free(newflag);
      free(flip);
    }
    free(loop);
    free(canon);
    free(is_free);
    free(npieces);
    free(poff);
    free(bot_v);
    free(top_v);
    free(psub);
    free(partner);
  }
done2:
  free(perm);
  free(leg_cnt);
  free(leg);
  free(leg_fill);
  free(pos_l);
  free(pos_r);
done:
  free(cell_tau);
  free(cell_flag);
  free(ev_cnt);
  free(ev);
  free(ev_fill);
  free(vtx);
  return rc;
}

int orc_keyed_run(const orc_params *p, uint32_t sweep0, int64_t n_updates, uint8_t *s0,
                  int64_t *op_ptr, double *op_tau, int64_t op_cap, orc_record *recs) {
  int64_t NS = orc_nsub(p), NC = orc_ncell(p);
  uint8_t *s1 = (uint8_t *)malloc((size_t)NS);
  int64_t *p1 = (int64_t *)malloc(sizeof(int64_t) * (size_t)(NC + 1));
  double *t1 = (double *)malloc(sizeof(double) * (size_t)(op_cap > 0 ? op_cap : 1));
  int rc = 0;
  for (int64_t t = 0; t < n_updates; ++t) {
    rc = orc_keyed_update(p, sweep0 + (uint32_t)t, s0, op_ptr, op_tau, s1, p1, t1, op_cap,
                          recs ? &recs[t] : NULL, 0, NULL, NULL, NULL, NULL, NULL, NULL);
    if (rc) break;
    memcpy(s0, s1, (size_t)NS);
    memcpy(op_ptr, p1, sizeof(int64_t) * (size_t)(NC + 1));
    memcpy(op_tau, t1, sizeof(double) * (size_t)p1[NC]);
  }
  free(s1);
  free(p1);
  free(t1);
  return rc;
}
