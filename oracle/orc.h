/*
 * CPU oracle for the continuous-time loop-cluster update (test infrastructure).
 *
 * This directory is TEST INFRASTRUCTURE.  Only the tests, the smoke entry point
 * and the benchmark's CPU-baseline leg may load it.  It shares no code with the
 * CUDA library: it is a plain, slow, obviously-correct restatement of the method
 * in fp64 / exact integer arithmetic.
 *
 * Two forms of one Monte Carlo step of the S=1/2 (Q=2S=1) or S=1 (Q=2, subspin)
 * antiferromagnetic Heisenberg chain, H = J sum_j S_j . S_{j+1}  (Eq. 1, Sec. 2):
 *
 *   orc_serial_update  -- the paper's sequential 8-step scan (Sec. 2, the
 *                         enumerated MC step): global exponential gaps, a
 *                         uniformly drawn bond per gap, union-find by weight with
 *                         path compression.  Its random stream is its own; it is
 *                         compared with everything else only statistically.
 *
 *   orc_keyed_update   -- the same Markov chain written per bond and per time
 *                         window with Philox keys (a reading of the insertion
 *                         step: superposition of per-bond Poisson processes of
 *                         rate J/2, Sec. 2 rule ii).  Clusters are found by
 *                         walking the loops of the segment graph (no
 *                         union-find).  Given the same state, seed and sweep it
 *                         defines every integer output of the update exactly.
 *
 * And the Swendsen-Wang update of the 2D Ising model on which the paper
 * benchmarks its union-find (Sec. 4.1): orc_sw_update (sw.c).
 */
#ifndef ORC_H
#define ORC_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Poisson thresholds per window: K <= ORC_KMAX-1 candidates per cell. */
#define ORC_KMAX 48
/* Mean number of candidate graphs per full window: window width w = 16/J. */
#define ORC_CELL_MEAN 8.0
/* Windows per time block in the canonical cell order. */
#define ORC_TW 4
/* Largest 2S (S = 2). */
#define ORC_QMAX 4

/* Philox tags (high byte of counter word 0). */
#define ORC_TAG_INSERT 1u
#define ORC_TAG_FLIP 2u
#define ORC_TAG_FREE 3u
#define ORC_TAG_PERM 4u
#define ORC_TAG_SERIAL 9u
#define ORC_TAG_SWBOND 5u
#define ORC_TAG_SWFLIP 6u

typedef struct {
  int64_t L;      /* original sites (even, >= 2) */
  int Q;          /* 2S subspins per site: 1 to ORC_QMAX */
  double J;       /* coupling, > 0 */
  double beta;    /* inverse temperature, > 0 */
  uint64_t seed;  /* Philox key */
} orc_params;

/* One update's measurements. Integer sums are exact. */
typedef struct {
  int64_t n;            /* graph vertices (old off-diagonal + new diagonal) */
  int64_t n_off_old;    /* off-diagonal operators before the update */
  int64_t n_off_new;    /* off-diagonal operators after the update */
  int64_t n_free;       /* loops that carry no vertex (empty cut cycles) */
  int64_t n_clusters;   /* loops in total */
  int64_t n_seg;        /* world-line fragments (pieces between vertices) */
  int32_t F;            /* fixed-point exponent of the per-loop sums */
  int32_t pad;
  /* Loop sums in ticks of 2^-F (fragment length = q(top) - q(bottom) + crossings
     x q(beta), q(x) = rint(x 2^F)); Fourier terms with cos, sin in 2^-32 units. */
  uint64_t sw2_lo, sw2_hi;  /* sum over loops of Wq^2 (128-bit) */
  uint64_t sf2_lo, sf2_hi;  /* sum over loops of Cq^2 + Sq^2 (128-bit) */
  /* Temporal moment: per fragment Z = e(top) - e(bottom), e(t) = exp(i w1 t) in
     2^-30 units (w1 = 2 pi / beta, evaluated as in orc_phase); per loop the sum
     of Z; here the sum over loops of |sum Z|^2 (128-bit). */
  uint64_t sz2_lo, sz2_hi;
  double energy;        /* E/L = (Q^2 J/4) - n/(beta L) */
  double chi_s;         /* sum_c W_c^2 / (4 beta L) */
  double chi_q;         /* sum_c |sum e^{ikx} len|^2 / (4 beta L), k = 2 pi/L */
  double chi_w;         /* sum_c |sum over fragments of int e^{i w1 t} dt|^2 / (4 beta L) */
} orc_record;

/* exp(i 2 pi q / qbeta) in units of 2^-30 for a tick count q of a time in
   [0, beta]: the fraction q / qbeta in 64-bit fixed point, X = (q R) >> sh
   modulo 2^64 with sh = floor(log2 qbeta) and R = floor((2^(64+sh) - 1) / qbeta)
   (error below 3 units of 2^-64); cos and sin at 2^16 points of the period
   (rounded to 30 fractional bits); linear interpolation in integers (floor of
   the 2^-32-scaled correction).  Error below 2e-9 of the unit. */
void orc_phase(uint64_t q, uint64_t R, int sh, int64_t *c, int64_t *s);
uint64_t orc_phase_recip(int64_t qbeta, int *sh);

/* Derived chain geometry (both forms use it). */
int64_t orc_nsub(const orc_params *p);
int64_t orc_nbond(const orc_params *p);
int64_t orc_nwin(const orc_params *p);
int64_t orc_ncell(const orc_params *p);
int64_t orc_cell_index(const orc_params *p, int64_t b, int64_t j);
int orc_fixed_exponent(const orc_params *p);

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Poisson(mu) thresholds: T[k] = floor(2^64 * P(K <= k)), saturated. */
void orc_poisson_thresholds(double mu, uint64_t T[ORC_KMAX]);

/* Neel start: s0[(i,a)] = i & 1, no operators. op_ptr has ncell+1 entries. */
void orc_neel(const orc_params *p, uint8_t *s0, int64_t *op_ptr);

/*
 * Keyed update.  Inputs: s0 [nsub], op_ptr [ncell+1] (canonical cell order),
 * op_tau [op_ptr[ncell]] sorted within each cell.  Outputs: s0_out, op_ptr_out,
 * op_tau_out (capacity op_cap).  Optional debug outputs (may be NULL):
 *   vtx_tau[n], vtx_flag[n] (1 = off-diagonal before the update),
 *   vtx_bond[n], vtx_pl[n], vtx_pr[n] (node of the piece below the vertex on its
 *   left / right subsite), vtx_root[n] (canonical id of the loop through the
 *   vertex's upper legs), cap_vtx the capacity of these arrays.
 * Returns 0, or -1 (capacity) / -2 (invalid configuration).
 */
int orc_keyed_update(const orc_params *p, uint32_t sweep, const uint8_t *s0,
                     const int64_t *op_ptr, const double *op_tau, uint8_t *s0_out,
                     int64_t *op_ptr_out, double *op_tau_out, int64_t op_cap,
                     orc_record *rec, int64_t cap_vtx, double *vtx_tau, uint8_t *vtx_flag,
                     int64_t *vtx_bond, int64_t *vtx_pl, int64_t *vtx_pr, int64_t *vtx_root);

/* Labeling step of one cell (bond b, window j) of the keyed update: writes the
 * cell's vertices (tau, flag) in vertex-id order; *n_out their number.
 * Returns -1 if cap is too small. */
int orc_keyed_cell(const orc_params *p, uint32_t sweep, const uint8_t *s0, const int64_t *op_ptr,
                   const double *op_tau, int64_t b, int64_t j, double *out_tau, uint8_t *out_flag,
                   int64_t cap, int64_t *n_out);

/* Run n keyed updates in place (state arrays must have room: op_cap). */
int orc_keyed_run(const orc_params *p, uint32_t sweep0, int64_t n_updates, uint8_t *s0,
                  int64_t *op_ptr, double *op_tau, int64_t op_cap, orc_record *recs);

/*
 * Serial (paper-literal) update on a time-ordered operator list.
 * ops_tau[n_ops], ops_bond[n_ops] sorted by tau; outputs replace them
 * (capacity op_cap).  Random numbers: Philox keyed by seed, counter stream
 * (i, sweep, ORC_TAG_SERIAL).
 */
int orc_serial_update(const orc_params *p, uint32_t sweep, uint8_t *s0, int64_t *n_ops,
                      double *ops_tau, int64_t *ops_bond, int64_t op_cap, orc_record *rec);

int orc_serial_run(const orc_params *p, uint32_t sweep0, int64_t n_updates, uint8_t *s0,
                   int64_t *n_ops, double *ops_tau, int64_t *ops_bond, int64_t op_cap,
                   orc_record *recs);

/*
 * Swendsen-Wang update of the L x L periodic Ising model (Sec. 4.1 benchmark).
 * Site i = y L + x, spin s[i] in {0, 1} (sigma = 1 - 2 s).  Bonds R(i) = (i,
 * right neighbour) and D(i) = (i, lower neighbour): 2N bonds, N = L^2.  The
 * draws of site i are Philox(ctr = (ORC_TAG_SWBOND << 24, i, 0, sweep),
 * key = seed): word 0 for R(i), word 1 for D(i).  A bond is active iff its two
 * spins are equal and its draw w < T = orc_sw_threshold(K).  A cluster's id is
 * its smallest site index r; its coin is bit (r mod 128) of Philox(ctr =
 * (ORC_TAG_SWFLIP << 24, r / 128, 0, sweep)), words in order, low bit first.
 */
typedef struct {
  int64_t n_eq;        /* bonds whose spins are equal, before the update */
  int64_t n_act;       /* activated bonds */
  int64_t n_clusters;  /* clusters (isolated sites included) */
  int64_t max_cluster; /* sites of the largest cluster */
  uint64_t sum_c2;     /* sum over clusters of size^2 (< 2^62 for N < 2^31) */
  int64_t mag;         /* sum of sigma after the update */
  double energy;       /* (2N - 2 n_eq) / N: energy per site before the update */
  double chi;          /* sum_c2 / N: improved estimator of <M^2> / N */
} orc_sw_record;

uint64_t orc_sw_threshold(double K);

/* One update in place on s[N].  Optional outputs (may be NULL): root_out[N]
 * (cluster id of every site), bond_out[2N] (R(i) at 2i, D(i) at 2i+1).
 * Returns 0, -1 (memory) or -2 (L < 2). */
int orc_sw_update(int64_t L, double K, uint64_t seed, uint32_t sweep, uint8_t *s,
                  int64_t *root_out, uint8_t *bond_out, orc_sw_record *rec);

/* n updates in place, sweeps sweep0, sweep0+1, ... */
int orc_sw_run(int64_t L, double K, uint64_t seed, uint32_t sweep0, int64_t n, uint8_t *s,
               orc_sw_record *recs);

#ifdef __cplusplus
}
#endif
#endif
