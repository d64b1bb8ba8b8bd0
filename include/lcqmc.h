/*
 * lcqmc -- continuous-time loop-cluster quantum Monte Carlo update of the
 * antiferromagnetic Heisenberg chain on one GB300 GPU (sm_103a), C ABI.
 *
 * Method: Todo, Matsuo, Shitara, "Parallel loop cluster quantum Monte Carlo
 * simulation of quantum magnets based on global union-find graph algorithm"
 * (arXiv:1810.07485).  The model is H = J sum_j S_j . S_{j+1} with periodic
 * boundaries (Eq. 1, Sec. 2); one update is the continuous-time loop step of
 * Sec. 2 (labeling, cluster identification, flip, rewrite, measurement) with the
 * cluster identification done by a lock-free union-find (Sec. 3.2).  S = 1,
 * 3/2 and 2 are handled by the subspin representation of Sec. 5 (Q = 2S
 * S=1/2 subspins per site, Q^2 sub-bonds per bond, the subspins joined at
 * tau = 0 by a permutation drawn uniformly among those that join equal
 * spins).
 *
 * Conventions shared by every entry point:
 *   - Return value: LCQMC_OK (0) on success, LCQMC_PENDING (1) where stated,
 *     a negative LCQMC_E_* code on failure.  lcqmc_last_error() returns a
 *     thread-local message describing the last failure of the calling thread.
 *   - Host pointers are plain host memory owned by the caller; the library
 *     copies from / into them before returning.  The library owns every device
 *     buffer it allocates; handles own their state until destroyed.
 *   - A chain handle or batch handle must not be used from two threads at
 *     once.  Server calls are thread-safe.
 *   - Work is ordered on the handle's CUDA stream; lcqmc_update only enqueues,
 *     lcqmc_sync / lcqmc_measure wait for it.
 *   - The world-line state is the spin configuration at tau=0 plus the
 *     imaginary times of the off-diagonal operators (Sec. 2, world lines).  Its
 *     exchange format groups operators by cell = (bond, time window):
 *       bond b of the subspin lattice joins subsite (i*Q + a) and
 *       (((i+1) mod L)*Q + a') with b = i*Q*Q + a*Q + a', Q = 2S;
 *       window j covers [j*w, (j+1)*w) with w = 16/J, the last one ends at beta;
 *       cells are ordered in blocks of LCQMC_TW windows, bond-major inside a
 *       block: cell(b, j) = (j/TW)*nbond*TW + b*tw + (j mod TW), tw = the
 *       block's window count.
 *     op_ptr has ncell+1 entries (CSR offsets), op_tau the times, ascending
 *     inside each cell.
 */
#ifndef LCQMC_H
#define LCQMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LCQMC_OK 0
#define LCQMC_PENDING 1
#define LCQMC_E_INVAL (-1)          /* bad argument: L < 2 or odd, beta <= 0, J <= 0, 2S not in 1..4 */
#define LCQMC_E_NOMEM (-2)          /* device or host allocation failed */
#define LCQMC_E_TOO_LARGE (-3)      /* footprint above the budget / the server's HBM budget */
#define LCQMC_E_ID_OVERFLOW (-4)    /* more than 2^31-4096 graph vertices, or 2^31 cells, in one chain */
#define LCQMC_E_DEVICE_TIMEOUT (-5) /* a bounded device wait (union-find retry) ran out */
#define LCQMC_E_CUDA (-6)           /* a CUDA runtime call failed */
#define LCQMC_E_STATE (-7)          /* imported configuration is not a valid world-line state */
#define LCQMC_E_NOT_FOUND (-8)      /* unknown server ticket */
#define LCQMC_E_CANCELLED (-9)      /* request was cancelled or rejected at admission */
#define LCQMC_E_CAPACITY (-10)      /* caller-provided output buffer too small */

#define LCQMC_TW 4 /* windows per time block of the cell order */

typedef struct lcqmc_chain *lcqmc_handle;
typedef struct lcqmc_batch *lcqmc_batch_t;
typedef struct lcqmc_server *lcqmc_server_t;

/* Running averages since create / the last reset (caller-owned). Index k of
 * sum/sumsq: 0 E/L, 1 chi_s, 2 chi(pi+2pi/L), 3 n (graph vertices),
 * 4 n_off (off-diagonal operators after the update), 5 world-line fragments,
 * 6 loops, 7 vertices+edges of the cluster graph (fragments + 2n),
 * 8 chi(pi, w1) at the first Matsubara frequency w1 = 2pi/beta. */
typedef struct {
  int64_t n_updates;
  double sum[9];
  double sumsq[9];
  double xi;     /* (L/2pi) sqrt(<chi_s>/<chi(pi+2pi/L)> - 1), ratio of means */
  double xi_tau; /* (beta/2pi) sqrt(<chi_s>/<chi(pi,w1)> - 1): imaginary-time length */
  double gap;    /* 1/xi_tau (Sec. 5: gap from the second moment in time) */
} lcqmc_obs;

/* One update's measurements.  The sums of squared loop lengths are exact
 * 128-bit integers in units of 2^-2F (F = 60 - ceil(log2(Q L beta))): every
 * fragment length is rounded once to a multiple of 2^-F, then summed per loop
 * exactly.  energy = Q^2 J/4 - n/(beta L); chi_s = sw2 2^-2F/(4 beta L);
 * chi_q = sf2 2^-2F/(4 beta L) with q = pi + 2 pi / L.  Temporal moment: per
 * fragment Z = e(top) - e(bottom) with e(t) = exp(i w1 t) in units of 2^-30
 * (w1 = 2 pi / beta; the period fraction of the time's tick count in 64-bit
 * fixed point, cos/sin at 2^16 points rounded to 30 bits, integer linear
 * interpolation), summed per loop; sz2 = sum over loops of |sum Z|^2 (exact);
 * chi_w = sz2 2^-60 beta / (16 pi^2 L) = sum_c |int e^{i w1 t} dt|^2 / (4 beta L). */
typedef struct {
  int64_t n, n_off_old, n_off_new, n_free, n_clusters, n_seg;
  int32_t F, pad;
  uint64_t sw2_lo, sw2_hi, sf2_lo, sf2_hi, sz2_lo, sz2_hi;
  double energy, chi_s, chi_q, chi_w;
} lcqmc_record;

typedef struct {
  int64_t L, nsub, nbond, nwin, ncell;
  int32_t Q, F;
  double J, beta, w;
  uint64_t seed;
  uint32_t sweep;   /* updates completed (the Philox sweep counter) */
  uint32_t replays; /* updates re-run after a buffer had to grow, since the
                       handle was created (saturates at 2^32 - 1); a timer
                       that brackets updates sees such re-runs outside its
                       window only if it stops before lcqmc_sync */
} lcqmc_geometry;

/* Device memory allocator supplied by the caller (e.g. a framework's caching
 * allocator).  alloc returns device memory of at least `bytes` or NULL; free
 * releases it.  ctx is passed through. */
typedef struct {
  void *(*alloc)(size_t bytes, void *ctx);
  void (*free)(void *ptr, void *ctx);
  void *ctx;
} lcqmc_allocator;

/* --- single chain (Sec. 2 MC step on one chain) ----------------------------- */

/* Creates a chain of L sites (even, >= 2), spin S (0.5, 1, 1.5 or 2, checked exactly),
 * coupling J > 0, inverse temperature beta > 0, Philox seed.  Starts from the
 * Neel state with no operators, sweep 0, on device 0's default stream. */
int lcqmc_create(int64_t L, double S, double J, double beta, uint64_t seed, lcqmc_handle *out);

/* As lcqmc_create with a CUDA stream (cudaStream_t as void*, NULL = legacy
 * default) and an optional allocator (NULL = cudaMalloc/cudaFree). */
int lcqmc_create_ex(int64_t L, double S, double J, double beta, uint64_t seed, void *cuda_stream,
                    const lcqmc_allocator *alloc, lcqmc_handle *out);

/* Enqueues n loop updates on the chain's stream.  Returns at once. */
int lcqmc_update(lcqmc_handle h, int64_t n);

/* Waits for enqueued updates.  Grows device buffers and replays updates that
 * ran out of room (results are unchanged: the random numbers are keyed by the
 * sweep counter).  Returns LCQMC_E_DEVICE_TIMEOUT if a device wait ran out. */
int lcqmc_sync(lcqmc_handle h);

/* Syncs, then fills *out with averages since create or the last reset. */
int lcqmc_measure(lcqmc_handle h, lcqmc_obs *out);
int lcqmc_reset_obs(lcqmc_handle h);

/* Syncs, then copies up to max per-update records (oldest first) that were
 * produced since the previous call into out; *count receives the number.  The
 * device keeps the last 4096 records; older ones are dropped (count them with
 * lcqmc_obs.n_updates). */
int lcqmc_get_records(lcqmc_handle h, lcqmc_record *out, int64_t max, int64_t *count);

int lcqmc_get_geometry(lcqmc_handle h, lcqmc_geometry *out);

/* Syncs, then copies the state: s0[nsub] (0/1), op_ptr[ncell+1], op_tau[n_off].
 * op_tau may be NULL to query *n_off only; LCQMC_E_CAPACITY if op_cap < n_off. */
int lcqmc_export_config(lcqmc_handle h, uint8_t *s0, int32_t *op_ptr, double *op_tau,
                        int64_t op_cap, int64_t *n_off);

/* Replaces the state with the given one and sets the sweep counter.  Checks
 * that op_ptr is a non-decreasing CSR, every time lies in its cell's window,
 * times are ascending inside a cell, and every operator acts on antiparallel
 * spins (Sec. 2 world-line constraint); LCQMC_E_STATE otherwise. */
int lcqmc_import_config(lcqmc_handle h, const uint8_t *s0, const int32_t *op_ptr,
                        const double *op_tau, int64_t n_off, uint32_t sweep);

/* Debug: keep the graph of the most recent update for lcqmc_export_graph. */
int lcqmc_set_keep_graph(lcqmc_handle h, int keep);

/* Debug: after an update with keep_graph set, copies per-vertex arrays of that
 * update (chain-local vertex ids): tau, flag (1 = operator was off-diagonal
 * before the update), pl / pr (node of the fragment below the vertex on its
 * left / right subsite), root (smallest node id of its loop).  n_cap entries
 * each; *n receives the vertex count.  Any pointer may be NULL. */
int lcqmc_export_graph(lcqmc_handle h, double *tau, uint8_t *flag, int32_t *pl, int32_t *pr,
                       int32_t *root, int64_t n_cap, int64_t *n);

/* Debug: vertex offsets of every cell (ncell+1 entries, chain-local ids, in
 * the cell order above) of the most recent update: the vertices of cell c are
 * ids vptr[c] .. vptr[c+1]-1 of lcqmc_export_graph. */
int lcqmc_export_cells(lcqmc_handle h, int32_t *vptr, int64_t cap);

/* Checkpoint = geometry + seed + sweep + state.  lcqmc_checkpoint with
 * buf == NULL sets *len to the size needed.  Restoring continues the same
 * Markov chain bit for bit. */
int lcqmc_checkpoint(lcqmc_handle h, void *buf, size_t *len);
int lcqmc_restore(lcqmc_handle h, const void *buf, size_t len);

/* Per-phase device time (ms) accumulated over updates while enabled, in the
 * spirit of the cost table of Sec. 4.3: 0 random numbers and labeling
 * (insertion with vertex offsets), 1 tau=0 cut, 2 linking and union-find,
 * 3 loop ids (compression, coins), 4 loop properties and new flags,
 * 5 operator offsets, 6 operator rewrite, 7 spin rewrite and record. */
#define LCQMC_NPHASE 8
int lcqmc_set_phase_timing(lcqmc_handle h, int enable);

/* Turns the temporal moment on or off (off after create): chi(pi, w1) at the
 * first Matsubara frequency w1 = 2 pi / beta, the record's sz2 and chi_w and
 * the obs' sum[8], xi_tau and gap (Sec. 5: the gap from the second moment in
 * imaginary time).  Off, those are 0 and every other result is unchanged.
 * Waits for enqueued updates; applies to the following ones. */
int lcqmc_set_temporal(lcqmc_handle h, int enable);

/* Debug: bound of the global union-find walks and compare-and-swap retries
 * (Sec. 3.2) of the following updates: 1 .. 2^22 steps, 0 restores the default
 * 2^22.  A walk that needs more steps stops the update on the device with the
 * chain's state untouched (neither the spins, the operators nor the sweep
 * counter change), and lcqmc_sync returns LCQMC_E_DEVICE_TIMEOUT.  With a tiny
 * bound this exercises that failure path on a correct chain; the next update
 * at the default bound is the one that would have run.  Waits for enqueued
 * updates; LCQMC_E_INVAL out of range. */
int lcqmc_set_wait_limit(lcqmc_handle h, int64_t limit);

/* Block sizes of the union-find phases (Sec. 3.2 on the GPU): threads per
 * block of the tile linking and local union-find (128 or 256), warps per block
 * of the union of tile-crossing edges (1..8, one tile each) and threads per
 * block of the compression (32..128 in steps of 32).  Defaults 256, 8, 128.
 * Any choice gives bit-identical results; only the time changes. */
typedef struct {
  int32_t link_threads, link_x_warps, compress_threads, pad;
} lcqmc_tuning;
/* Current block sizes (host struct, caller-owned). */
int lcqmc_get_tuning(lcqmc_handle h, lcqmc_tuning *out);
/* Waits for enqueued updates, then sets the block sizes; LCQMC_E_INVAL out of
 * range. */
int lcqmc_set_tuning(lcqmc_handle h, const lcqmc_tuning *cfg);
/* Autotuner: times each candidate with the phase events over
 * updates_per_trial updates (a coordinate search: 128/256 x 2/4/8 for the
 * linking phase, then 64/128 for the compression; 8 trials) and keeps the
 * fastest.  The trial updates are ordinary updates of the chain (records and
 * running sums included).  out (may be NULL) receives the choice. */
int lcqmc_autotune(lcqmc_handle h, int64_t updates_per_trial, lcqmc_tuning *out);
int lcqmc_get_phase_times(lcqmc_handle h, double *ms, int nphase);

/* Raw CUDA stream of the handle (cudaStream_t as void*). */
void *lcqmc_stream(lcqmc_handle h);

int lcqmc_destroy(lcqmc_handle h);

/* --- batched form: many independent chains in one launch per phase ------- */

typedef struct {
  int64_t L;
  double S, J, beta;
  uint64_t seed;
} lcqmc_chain_spec;

/* Creates a batch of independent chains (Sec. 3: independent Markov chains),
 * updated together: every phase of an update is one kernel launch over all
 * chains' cells, and n updates are replayed from one captured CUDA graph. */
int lcqmc_batch_create(int64_t nchains, const lcqmc_chain_spec *specs, void *cuda_stream,
                       lcqmc_batch_t *out);
int lcqmc_batch_update(lcqmc_batch_t b, int64_t n);
int lcqmc_batch_sync(lcqmc_batch_t b);
int lcqmc_batch_set_temporal(lcqmc_batch_t b, int enable); /* as lcqmc_set_temporal, all chains */
/* As lcqmc_get_tuning / lcqmc_set_tuning / lcqmc_autotune for a batch (one
 * choice for all its chains; trial updates update every chain). */
int lcqmc_batch_get_tuning(lcqmc_batch_t b, lcqmc_tuning *out);
int lcqmc_batch_set_tuning(lcqmc_batch_t b, const lcqmc_tuning *cfg);
int lcqmc_batch_autotune(lcqmc_batch_t b, int64_t updates_per_trial, lcqmc_tuning *out);
int lcqmc_batch_measure(lcqmc_batch_t b, int64_t chain, lcqmc_obs *out);
int lcqmc_batch_get_records(lcqmc_batch_t b, int64_t chain, lcqmc_record *out, int64_t max,
                            int64_t *count);
int lcqmc_batch_destroy(lcqmc_batch_t b);

/* --- served form: continuous batching of simulation requests -------------- */

typedef struct {
  int64_t L;
  double S, J, beta;
  uint64_t seed;
  int64_t n_updates; /* updates to run, then read out */
} lcqmc_request;

typedef struct {
  int32_t status; /* LCQMC_OK, LCQMC_PENDING, or LCQMC_E_* */
  int32_t pad;
  lcqmc_obs obs;
  double t_submit, t_admit, t_done; /* seconds on the server's clock */
  int64_t vertices_edges;           /* total V+E processed for this request */
} lcqmc_result;

/* Device bytes one served chain holds (persistent state + its share of the
 * update's scratch), as used for admission.  Host-only; needs no GPU. */
int lcqmc_footprint(int64_t L, double S, double J, double beta, size_t *bytes);

/* A server keeps up to max_slots chains resident on the device within
 * hbm_budget bytes, admits queued requests as slots and memory free up, and
 * advances all resident chains together in ticks of updates. */
int lcqmc_server_create(size_t hbm_budget, int max_slots, lcqmc_server_t *out);
/* Queues a request; LCQMC_E_TOO_LARGE if its footprint alone exceeds the
 * budget, LCQMC_E_ID_OVERFLOW if it needs more than 2^31 graph vertices. */
int lcqmc_submit(lcqmc_server_t s, const lcqmc_request *req, uint64_t *ticket);
/* LCQMC_PENDING while queued or running; LCQMC_OK once out->status holds the
 * outcome (LCQMC_OK with obs filled, or an error / LCQMC_E_CANCELLED). */
int lcqmc_poll(lcqmc_server_t s, uint64_t ticket, lcqmc_result *out);
int lcqmc_cancel(lcqmc_server_t s, uint64_t ticket);
int lcqmc_server_destroy(lcqmc_server_t s);

/* Loop labelling with no device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not call cudaMalloc: code
 * that runs inside another framework's memory pool or under a device-memory
 * budget fixed when it started, which may not grow its footprint, and code
 * whose other streams must not be stalled by the device-wide synchronization
 * that cudaMalloc implies.  Input: n graph vertices, pl[n] / pr[n] = node of
 * the fragment below each vertex on its left / right subsite (device
 * pointers, node ids in [0, n), as lcqmc_export_graph returns them).
 * Output: root[n] (device pointer) = smallest node id of each node's loop.
 * The union-find forest lives in a fixed device array of 2^22 int32 parents
 * compiled into the library (reserved on every GPU that loads it, until
 * exit); n above 2^22 returns LCQMC_E_TOO_LARGE.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) and keeps it:
 * make that first call before any stream capture, and make no call after
 * cudaDeviceReset on that device (the kept address would be stale).  Work
 * runs on cuda_stream (NULL = legacy default); the call then waits for that
 * stream, to read back a status word.  All calls share the array and each
 * call resets what it uses; calls that overlap on the GPU race and must be
 * serialized by the caller.  LCQMC_E_INVAL if an id is outside [0, n). */
int lcqmc_loops_noalloc(const int32_t *pl, const int32_t *pr, int64_t n, int32_t *root,
                        void *cuda_stream);

/* Host-side self-test of the integer bit constructions the kernels use, against
 * the C library, on n random inputs from seed (which = 0: the unit factor
 * u53 2^-53 of a candidate time, Sec. 2 step 2; which = 1: the tick count
 * rint(x 2^F) of a time, used by the loop-length sums).  *mismatches receives
 * the count.  Needs no GPU. */
int lcqmc_selftest(int which, int64_t n, uint64_t seed, int64_t *mismatches);

/* Message of the calling thread's last failure ("" if none). */
const char *lcqmc_last_error(void);

/* ---- Swendsen-Wang update of the 2D Ising model ----------------------------
 * The benchmark on which the paper measures its union-find alone (Sec. 4.1):
 * classical spins sigma = +-1 on an L x L periodic square lattice, a bond
 * between equal nearest neighbours activated with probability
 * p = 1 - exp(-2K), every cluster of active bonds flipped with probability
 * 1/2 (Swendsen-Wang 1987); the paper's workload is L = 8192 at
 * K_c = ln(1 + sqrt 2)/2.
 *
 * Keyed definition (bit-exact, as the CPU oracle's): site i = y L + x, spin
 * s[i] in {0, 1} with sigma = 1 - 2 s.  Bonds R(i) = (i, (x+1 mod L, y)) and
 * D(i) = (i, (x, y+1 mod L)): 2 L^2 bonds.  The draws of site i are
 * Philox4x32-10(counter = (5 << 24, i, 0, sweep), key = seed): word 0 for
 * R(i), word 1 for D(i).  A bond is active iff its spins are equal and its
 * draw is below T = round(2^32 (1 - e^{-2K})).  A cluster is named by its
 * smallest site index r; it flips iff bit (r mod 128) of Philox4x32-10(
 * counter = (6 << 24, r / 128, 0, sweep), key = seed) is 1 (words in order,
 * low bit first).  Update t of a lattice created (or set) at sweep t0 uses
 * sweep t0 + t.  The handle owns all device memory (about 10.5 B per site);
 * calls on one handle are not thread-safe. */
typedef struct lcqmc_sw *lcqmc_sw_t;

typedef struct {
  int64_t sweep;        /* sweep counter of this update */
  int64_t n_eq;         /* bonds with equal spins, before the update */
  int64_t n_act;        /* active bonds */
  int64_t n_clusters;   /* clusters, single sites included */
  int64_t max_cluster;  /* sites of the largest cluster */
  uint64_t sum_c2;      /* sum over clusters of size^2 (exact) */
  int64_t mag;          /* sum of sigma after the update */
  double energy;        /* (2N - 2 n_eq) / N: -(1/N) sum_bonds sigma sigma before the update */
  double chi;           /* sum_c2 / N: improved estimator of <M^2> / N */
} lcqmc_sw_record;

#define LCQMC_SW_NOBS 4
typedef struct {
  int64_t n_updates;
  /* running sums and sums of squares since create of: energy, chi,
   * M^2 / N and |M| / N (M after each update) */
  double sum[LCQMC_SW_NOBS], sumsq[LCQMC_SW_NOBS];
} lcqmc_sw_obs;

/* New lattice, every sigma = +1, sweep 0.  L in [2, 46340] (L^2 < 2^31), K
 * >= 0 finite (LCQMC_E_INVAL otherwise).  cuda_stream: the stream all work of
 * the handle runs on (NULL: a stream of its own). */
int lcqmc_sw_create(int64_t L, double K, uint64_t seed, void *cuda_stream, lcqmc_sw_t *out);
/* Enqueues n updates (stream-ordered, no wait).  Each appends one record to a
 * ring of 4096 on the device. */
int lcqmc_sw_update(lcqmc_sw_t h, int64_t n);
/* Waits for the enqueued updates; LCQMC_E_DEVICE_TIMEOUT if a bounded
 * union-find walk ran out (the update stops and the spins are left as they
 * were before it). */
int lcqmc_sw_sync(lcqmc_sw_t h);
/* Waits, then copies up to max_n records not read before (oldest first) to
 * out (host, caller-owned); *n_out = their number.  Records older than the
 * last 4096 are lost. */
int lcqmc_sw_get_records(lcqmc_sw_t h, lcqmc_sw_record *out, int64_t max_n, int64_t *n_out);
/* Waits, then the running sums since create. */
int lcqmc_sw_measure(lcqmc_sw_t h, lcqmc_sw_obs *out);
/* Waits, then replaces the spins (host array of L^2 bytes, each 0 or 1, else
 * LCQMC_E_STATE) and sets the next update's sweep counter. */
int lcqmc_sw_set_spins(lcqmc_sw_t h, const uint8_t *spins, uint32_t sweep);
/* Waits, then copies the spins (L^2 bytes, row-major) to the host. */
int lcqmc_sw_get_spins(lcqmc_sw_t h, uint8_t *spins);
/* Waits, then the cluster name of every site (L^2 int32, host) in the last
 * update (LCQMC_E_STATE before the first). */
int lcqmc_sw_get_roots(lcqmc_sw_t h, int32_t *roots);
/* Per-phase device times (CUDA events, off by default; on: updates run
 * without the captured graph).  Phases: [0] bond draws and union-find inside
 * each 64 x 32 tile, [1] tile-boundary bonds in the global forest, [2] roots,
 * coins and flips, [3] open clusters' sizes and the record.  ms: summed
 * milliseconds since timing was switched on. */
#define LCQMC_SW_NPHASE 4
int lcqmc_sw_set_phase_timing(lcqmc_sw_t h, int enable);
int lcqmc_sw_get_phase_times(lcqmc_sw_t h, double *ms, int nphase);
/* The handle's CUDA stream (for events around updates). */
void *lcqmc_sw_stream(lcqmc_sw_t h);
/* Waits for the handle's work and frees everything it owns. */
int lcqmc_sw_destroy(lcqmc_sw_t h);

#ifdef __cplusplus
}
#endif
#endif
