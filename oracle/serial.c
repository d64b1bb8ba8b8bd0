/*
 * Paper-literal form of one loop-cluster update (test infrastructure; see orc.h).
 *
 * Follows the enumerated continuous-time Monte Carlo step of Sec. 2 one step at
 * a time: tau advances by exponential gaps -(2/(J N_b)) log r with r in (0,1];
 * off-diagonal operators passed on the way are kept as horizontal graphs and
 * flip the spins; at each new tau' a bond is drawn uniformly and a horizontal
 * graph is inserted if its spins are antiparallel.  Loops are built while
 * scanning with union-find (union by weight, path compression; Sec. 2, last
 * paragraph), flipped with probability 1/2, and s(tau=0) and the operator list
 * are rewritten.  For S=1 (Q=2) the same scan runs on the subspin lattice of
 * Sec. 5 and the subspins are joined at tau=0 by a permutation drawn uniformly
 * among those consistent with the spins there.
 *
 * Its random numbers are a sequential Philox stream; it is compared with the
 * keyed form and with exact diagonalization only statistically.
 */
#include "orc.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint32_t key[2];
  uint32_t sweep;
  uint64_t ctr;
  uint32_t buf[4];
  int left;
} stream_t;

static uint64_t next_u64(stream_t *s) {
  if (s->left == 0) {
    uint32_t c[4] = {ORC_TAG_SERIAL << 24, (uint32_t)s->ctr, (uint32_t)(s->ctr >> 32), s->sweep};
    orc_philox4x32_10(c, s->key, s->buf);
    s->ctr++;
    s->left = 2;
  }
  int i = 2 - s->left;
  s->left--;
  return (uint64_t)s->buf[2 * i] | ((uint64_t)s->buf[2 * i + 1] << 32);
}

/* r uniform in (0, 1]. */
static double next_r(stream_t *s) { return ldexp((double)((next_u64(s) >> 11) + 1), -53); }

static int64_t next_index(stream_t *s, int64_t n) {
  return (int64_t)(((unsigned __int128)next_u64(s) * (unsigned __int128)(uint64_t)n) >> 64);
}

typedef struct {
  int64_t *parent, *weight;
  int64_t n, cap;
} uf_t;

static int64_t uf_add(uf_t *u) {
  if (u->n == u->cap) {
    u->cap = u->cap ? 2 * u->cap : 1024;
    u->parent = (int64_t *)realloc(u->parent, sizeof(int64_t) * (size_t)u->cap);
    u->weight = (int64_t *)realloc(u->weight, sizeof(int64_t) * (size_t)u->cap);
  }
  u->parent[u->n] = u->n;
  u->weight[u->n] = 1;
  return u->n++;
}

static int64_t uf_find(uf_t *u, int64_t x) {
  int64_t r = x;
  while (u->parent[r] != r) r = u->parent[r];
  while (u->parent[x] != r) { /* path compression */
    int64_t nx = u->parent[x];
    u->parent[x] = r;
    x = nx;
  }
  return r;
}

static void uf_union(uf_t *u, int64_t a, int64_t b) {
  int64_t ra = uf_find(u, a), rb = uf_find(u, b);
  if (ra == rb) return;
  if (u->weight[ra] < u->weight[rb]) { /* union by weight */
    int64_t t = ra;
    ra = rb;
    rb = t;
  }
  u->parent[rb] = ra;
  u->weight[ra] += u->weight[rb];
}

typedef struct {
  int64_t sub;
  double t0, t1;
  int from_vertex;
} seg_t;

typedef struct {
  double tau;
  int64_t bond, below, above;
  int flag;
} sv_t;

int orc_serial_update(const orc_params *p, uint32_t sweep, uint8_t *s0, int64_t *n_ops,
                      double *ops_tau, int64_t *ops_bond, int64_t op_cap, orc_record *rec) {
  const int64_t L = p->L, Q = p->Q, NS = orc_nsub(p), NB = orc_nbond(p);
  const double beta = p->beta;
  stream_t rs = {{(uint32_t)p->seed, (uint32_t)(p->seed >> 32)}, sweep, 0, {0, 0, 0, 0}, 0};
  uf_t uf = {NULL, NULL, 0, 0};
  int64_t scap = 2 * NS + 1024, ns = 0;
  seg_t *seg = (seg_t *)malloc(sizeof(seg_t) * (size_t)scap);
  int64_t vcap = *n_ops + 1024, nv = 0;
  sv_t *vs = (sv_t *)malloc(sizeof(sv_t) * (size_t)vcap);
  int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
  int64_t *first = (int64_t *)malloc(sizeof(int64_t) * (size_t)NS);
  uint8_t *s = (uint8_t *)malloc((size_t)NS);
  int rc = 0;

#define NEW_SEG(SUB, T0, FV)                                                 \
  do {                                                                       \
    if (ns == scap) {                                                        \
      scap *= 2;                                                             \
      seg = (seg_t *)realloc(seg, sizeof(seg_t) * (size_t)scap);             \
    }                                                                        \
    seg[ns].sub = (SUB);                                                     \
    seg[ns].t0 = (T0);                                                       \
    seg[ns].t1 = beta;                                                       \
    seg[ns].from_vertex = (FV);                                              \
    uf_add(&uf);                                                             \
    ++ns;                                                                    \
  } while (0)

  /* Step 1: tau <- 0, s <- s(0); one open segment per subsite. */
  for (int64_t u = 0; u < NS; ++u) {
    s[u] = s0[u];
    NEW_SEG(u, 0.0, 0);
    cur[u] = first[u] = ns - 1;
  }

  double tau = 0.0;
  int64_t q = 0;
  for (;;) {
    /* Step 2: tau' <- tau - (2 / (J N_b)) log r. */
    double r = next_r(&rs);
    double tau2 = tau - (2.0 / (p->J * (double)NB)) * log(r);
    /* Step 3: operators in (tau, tau'] become horizontal graphs and flip s. */
    while (q < *n_ops && ops_tau[q] <= tau2) {
      double tv = ops_tau[q];
      int64_t b = ops_bond[q];
      int64_t i = b / (Q * Q), a = (b / Q) % Q, a2 = b % Q;
      int64_t ul = i * Q + a, ur = ((i + 1) % L) * Q + a2;
      if (nv == vcap) {
        vcap *= 2;
        vs = (sv_t *)realloc(vs, sizeof(sv_t) * (size_t)vcap);
      }
      seg[cur[ul]].t1 = tv;
      seg[cur[ur]].t1 = tv;
      uf_union(&uf, cur[ul], cur[ur]); /* lower legs */
      vs[nv].tau = tv;
      vs[nv].bond = b;
      vs[nv].below = cur[ul];
      vs[nv].flag = 1;
      NEW_SEG(ul, tv, 1);
      cur[ul] = ns - 1;
      NEW_SEG(ur, tv, 1);
      cur[ur] = ns - 1;
      uf_union(&uf, cur[ul], cur[ur]); /* upper legs */
      vs[nv].above = cur[ul];
      ++nv;
      s[ul] ^= 1;
      s[ur] ^= 1;
      ++q;
    }
    /* Step 4: stop at the end of the time interval. */
    if (tau2 >= beta) break;
    /* Step 5: a uniformly drawn bond gets a graph iff antiparallel. */
    int64_t b = next_index(&rs, NB);
    int64_t i = b / (Q * Q), a = (b / Q) % Q, a2 = b % Q;
    int64_t ul = i * Q + a, ur = ((i + 1) % L) * Q + a2;
    if (s[ul] != s[ur]) {
      if (nv == vcap) {
        vcap *= 2;
        vs = (sv_t *)realloc(vs, sizeof(sv_t) * (size_t)vcap);
      }
      seg[cur[ul]].t1 = tau2;
      seg[cur[ur]].t1 = tau2;
      uf_union(&uf, cur[ul], cur[ur]);
      vs[nv].tau = tau2;
      vs[nv].bond = b;
      vs[nv].below = cur[ul];
      vs[nv].flag = 0;
      NEW_SEG(ul, tau2, 1);
      cur[ul] = ns - 1;
      NEW_SEG(ur, tau2, 1);
      cur[ur] = ns - 1;
      uf_union(&uf, cur[ul], cur[ur]);
      vs[nv].above = cur[ul];
      ++nv;
    }
    /* Step 6. */
    tau = tau2;
  }

  /* Close the world lines at tau = beta: join each top to a bottom at tau = 0. */
  for (int64_t i = 0; i < L; ++i) {
    if (Q == 1) {
      uf_union(&uf, cur[i], first[i]);
      continue;
    }
    if (Q > 2) {
      /* uniform among the permutations joining equal spins: shuffle the
         bottoms of each spin value (Fisher-Yates) and pair them in order */
      int64_t tops[2][ORC_QMAX], bots[2][ORC_QMAX];
      int nt[2] = {0, 0}, nb[2] = {0, 0};
      for (int a = 0; a < Q; ++a) {
        int64_t u = i * Q + a;
        tops[s[u] ? 0 : 1][nt[s[u] ? 0 : 1]++] = u;
        bots[s0[u] ? 0 : 1][nb[s0[u] ? 0 : 1]++] = u;
      }
      if (nt[0] != nb[0]) {
        rc = -2;
        goto out;
      }
      for (int g = 0; g < 2; ++g) {
        for (int j = nb[g] - 1; j >= 1; --j) {
          int r = (int)(next_u64(&rs) % (uint64_t)(j + 1));
          int64_t tmp = bots[g][j];
          bots[g][j] = bots[g][r];
          bots[g][r] = tmp;
        }
        for (int m = 0; m < nt[g]; ++m) uf_union(&uf, cur[tops[g][m]], first[bots[g][m]]);
      }
      continue;
    }
    int64_t u0 = i * Q, u1 = i * Q + 1;
    int ok_id = (s[u0] == s0[u0]) && (s[u1] == s0[u1]);
    int ok_sw = (s[u0] == s0[u1]) && (s[u1] == s0[u0]);
    int swap;
    if (ok_id && ok_sw)
      swap = (int)(next_u64(&rs) & 1u);
    else if (ok_sw)
      swap = 1;
    else if (ok_id)
      swap = 0;
    else {
      rc = -2;
      goto out;
    }
    uf_union(&uf, cur[u0], first[swap ? u1 : u0]);
    uf_union(&uf, cur[u1], first[swap ? u0 : u1]);
  }

  {
    /* Step 7: flip every loop with probability 1/2 and rewrite. */
    uint8_t *flip = (uint8_t *)malloc((size_t)ns);
    uint8_t *seen = (uint8_t *)calloc((size_t)ns, 1);
    uint8_t *hasv = (uint8_t *)calloc((size_t)ns, 1);
    int64_t nclu = 0, nfree = 0;
    for (int64_t x = 0; x < ns; ++x) {
      int64_t rt = uf_find(&uf, x);
      if (!seen[rt]) {
        seen[rt] = 1;
        flip[rt] = (uint8_t)(next_u64(&rs) & 1u);
        ++nclu;
      }
      if (seg[x].from_vertex) hasv[rt] = 1;
    }
    for (int64_t x = 0; x < ns; ++x)
      if (uf_find(&uf, x) == x && !hasv[x]) ++nfree;
    for (int64_t u = 0; u < NS; ++u) s0[u] = (uint8_t)(s0[u] ^ flip[uf_find(&uf, first[u])]);
    int64_t nn = 0, n_old = *n_ops;
    for (int64_t v = 0; v < nv; ++v) {
      int f = vs[v].flag ^ flip[uf_find(&uf, vs[v].below)] ^ flip[uf_find(&uf, vs[v].above)];
      if (!f) continue;
      if (nn < op_cap) {
        ops_tau[nn] = vs[v].tau;
        ops_bond[nn] = vs[v].bond;
      }
      ++nn;
    }
    if (nn > op_cap) rc = -1;
    *n_ops = nn;

    /* Step 8: measurement from the loop lengths. */
    double *W = (double *)calloc((size_t)ns, sizeof(double));
    double *C = (double *)calloc((size_t)ns, sizeof(double));
    double *S = (double *)calloc((size_t)ns, sizeof(double));
    double *ZR = (double *)calloc((size_t)ns, sizeof(double));
    double *ZI = (double *)calloc((size_t)ns, sizeof(double));
    const double w1 = 2.0 * M_PI / beta; /* first Matsubara frequency */
    for (int64_t x = 0; x < ns; ++x) {
      int64_t rt = uf_find(&uf, x);
      double len = seg[x].t1 - seg[x].t0;
      double ang = (2.0 * M_PI * (double)(seg[x].sub / Q)) / (double)L;
      W[rt] += len;
      C[rt] += len * cos(ang);
      S[rt] += len * sin(ang);
      /* int_{t0}^{t1} e^{i w1 t} dt = (e^{i w1 t1} - e^{i w1 t0}) / (i w1) */
      ZR[rt] += cos(w1 * seg[x].t1) - cos(w1 * seg[x].t0);
      ZI[rt] += sin(w1 * seg[x].t1) - sin(w1 * seg[x].t0);
    }
    double sw2 = 0.0, sf2 = 0.0, sz2 = 0.0;
    for (int64_t x = 0; x < ns; ++x) {
      if (uf_find(&uf, x) != x) continue;
      sw2 += W[x] * W[x];
      sf2 += C[x] * C[x] + S[x] * S[x];
      sz2 += ZR[x] * ZR[x] + ZI[x] * ZI[x];
    }
    if (rec) {
      memset(rec, 0, sizeof(*rec));
      rec->n = nv;
      rec->n_off_old = n_old;
      rec->n_off_new = nn;
      rec->n_free = nfree;
      rec->n_clusters = nclu;
      rec->n_seg = 2 * nv + nfree;
      rec->energy = (double)(Q * Q) * p->J * 0.25 - (double)nv / (beta * (double)L);
      rec->chi_s = sw2 / (4.0 * beta * (double)L);
      rec->chi_q = sf2 / (4.0 * beta * (double)L);
      rec->chi_w = sz2 / (w1 * w1 * 4.0 * beta * (double)L);
    }
    free(ZR);
    free(ZI);
    free(W);
    free(C);
    free(S);
    free(flip);
    free(seen);
    free(hasv);
  }
out:
#undef NEW_SEG
  free(seg);
  free(vs);
  free(cur);
  free(first);
  free(s);
  free(uf.parent);
  free(uf.weight);
  return rc;
}

int orc_serial_run(const orc_params *p, uint32_t sweep0, int64_t n_updates, uint8_t *s0,
                   int64_t *n_ops, double *ops_tau, int64_t *ops_bond, int64_t op_cap,
                   orc_record *recs) {
  for (int64_t t = 0; t < n_updates; ++t) {
    int rc = orc_serial_update(p, sweep0 + (uint32_t)t, s0, n_ops, ops_tau, ops_bond, op_cap,
                               recs ? &recs[t] : NULL);
    if (rc) return rc;
  }
  return 0;
}
