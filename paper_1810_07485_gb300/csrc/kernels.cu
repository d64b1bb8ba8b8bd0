// Kernels of one continuous-time loop-cluster update (Sec. 2 MC step, Sec. 3.2
// union-find), batched over independent chains.  Work is cut into tiles of 128
// consecutive cells (bond x time window) of one chain; a tile is one block.
//
// Phase order per update (the Sec. 4.3 cost table's rows in brackets):
//   k_bond_parity    spin parity of every bond at each time-block start
//   k_insert         per cell: Poisson candidates, keep the antiparallel ones,
//                    merge with old operators, write vertices; offsets by
//                    decoupled look-back over the tiles          [1, 2]
//   k_cut            last leg per subsite, tau=0 subspin permutation
//   k_link           predecessor of each leg on both subsites; union of the two
//                    fragments below each vertex (lock-free, min root)    [2]
//   k_compress       root of every node, one coin per loop              [3]
//   k_est            new operator flags, loop lengths (tile-local loops in
//                    shared memory, others in global accumulators)      [4]
//   k_scan_ops       operator offsets per tile
//   k_compact        next operator list, squared lengths of open loops  [8]
//   k_sites          spins at tau = 0, vertex-free loops                [8]
//   k_final          per-chain record, running sums, buffer swap
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>

#include "dev.cuh"
#include "kernels.h"
#include "uf.cuh"

namespace lcq {

__constant__ uint64_t c_T_full[KMAX];
// exp(i 2 pi k / 2^16) in units of 2^-30, k = 0..2^16 (temporal moment)
__device__ int2 g_phase_tab[(1 << PHASE_BITS) + 1];

// ---- block-wide helpers (blockDim.x is a multiple of 32, <= 1024) ---------
template <typename T>
__device__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

template <typename T>
__device__ T block_excl_scan(T v, T *sm, T &total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T x = (lane < nw) ? sm[lane] : T(0);
    T xi = warp_incl_scan(x);
    if (lane < nw) sm[lane] = xi - x;
    if (lane == nw - 1) sm[32] = xi;
  }
  __syncthreads();
  T res = sm[wid] + inc - v;
  total = sm[32];
  __syncthreads();
  return res;
}

template <typename T>
__device__ T block_sum(T v, T *sm) {
  T tot;
  block_excl_scan(v, sm, tot);
  return tot;
}

// Exact block-wide sum of 128-bit values (warp shuffles of both halves).
__device__ u128 block_sum_u128(u128 v) {
  __shared__ u128 part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  u128 x = v;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long l = __shfl_down_sync(0xffffffffu, (unsigned long long)x, o);
    unsigned long long h = __shfl_down_sync(0xffffffffu, (unsigned long long)(x >> 64), o);
    x += ((u128)h << 64) | (u128)l;
  }
  if (lane == 0) part[wid] = x;
  __syncthreads();
  u128 t = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nw; ++i) t += part[i];
    part[0] = t;
  }
  __syncthreads();
  t = part[0];
  __syncthreads();
  return t;
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int o) {
  const unsigned long long l = __shfl_down_sync(0xffffffffu, (unsigned long long)v, o);
  const unsigned long long h = __shfl_down_sync(0xffffffffu, (unsigned long long)(v >> 64), o);
  return ((u128)h << 64) | (u128)l;
}

// Exact block-wide sums of one int64 and two (Z: three) 128-bit values with a
// single barrier; the totals are valid in thread 0.  Once per kernel.
template <bool Z>
__device__ void block_sums(long long &c, u128 &x, u128 &y, u128 &z) {
  __shared__ long long pc[32];
  __shared__ u128 px[32], py[32], pz[Z ? 32 : 1];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(0xffffffffu, c, o);
    x += shfl_down_u128(x, o);
    y += shfl_down_u128(y, o);
    if (Z) z += shfl_down_u128(z, o);
  }
  if (lane == 0) {
    pc[wid] = c;
    px[wid] = x;
    py[wid] = y;
    if (Z) pz[wid] = z;
  }
  __syncthreads();
  if (wid == 0) {
    c = lane < nw ? pc[lane] : 0;
    x = lane < nw ? px[lane] : (u128)0;
    y = lane < nw ? py[lane] : (u128)0;
    if (Z) z = lane < nw ? pz[lane] : (u128)0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      c += __shfl_down_sync(0xffffffffu, c, o);
      x += shfl_down_u128(x, o);
      y += shfl_down_u128(y, o);
      if (Z) z += shfl_down_u128(z, o);
    }
  }
}

__device__ __forceinline__ bool halted(const Scratch &s) { return __ldcg(s.status) != 0; }

// Tile blocks of the vertex-parallel kernels: TPB threads walk the tile's
// vertices in id order (coalesced); a vertex's cell comes from a binary search
// in the tile's cell offsets staged in shared memory.
constexpr int TPB = 256;

__device__ __forceinline__ int tile_cell_of(const int *cvp, int ncl, int w) {
  // largest i in [0, ncl) with cvp[i] <= w
  int lo = 0, hi = ncl - 1;
  while (lo < hi) {
    const int mid = lo + ((hi - lo + 1) >> 1);
    if (cvp[mid] <= w)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ---- bond parity at time-block starts ---------------------------------------
// bpar[(blk) * nbond + b] = parity of the operators of bond b in time blocks
// before blk; row nblk is the parity over the whole period.
__global__ void k_bond_parity(const DevChain *__restrict__ ch, const int2 *__restrict__ tab,
                              int64_t blk0, Scratch s) {
  if (halted(s)) return;
  const int2 t = tab[blk0 + blockIdx.x];
  const DevChain &C = ch[t.x];
  const int b = t.y * BOND_BLOCK + threadIdx.x;
  if (b >= C.nbond) return;
  const int32_t *op = C.op_ptr[C.cur];
  uint8_t *row = s.bpar + C.bpar_off;
  uint8_t p = 0;
  row[b] = 0;
  for (int blk = 0; blk < C.nblk; ++blk) {
    int j0 = blk * TW;
    int tw = min(TW, C.nwin - j0);
    int c0 = blk * C.nbond * TW + b * tw;
    p ^= (uint8_t)((op[c0 + tw] - op[c0]) & 1);
    row[(int64_t)(blk + 1) * C.nbond + b] = p;
  }
}

// ---- per-update scratch reset -------------------------------------------------
// The insertion's look-back words and tile tickets and the four per-vertex
// bitmaps (open marks, open roots, coin flips, crossing marks) start each
// update at zero: one grid-stride launch instead of one memset each (a small
// chain's update is a chain of short launches).
__global__ void k_clear(Scratch s, int64_t ntile, int64_t nw) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t step = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = i0; i < nw; i += step) {
    s.openmark[i] = 0u;
    s.openroot[i] = 0u;
    s.flipbits[i] = 0u;
    s.xmark[i] = 0u;
  }
  for (int64_t i = i0; i < ntile; i += step) s.tile_state[i] = 0ull;
  if (i0 < QMAX) s.tickets[i0] = 0u;
}

// ---- insertion (labeling, rules i-iii) --------------------------------------
// Imaginary times are handled as the int64 bit patterns of non-negative doubles
// (same order as the values); a candidate's time is the exact integer form of
// fma(t_end - t0, u, t0).  No fp64 instruction is issued.
template <int Q>
struct NbOps {
  static constexpr int N = 4 * Q - 2;
  int bond[N];
  int o0[N], o1[N];
};

// Single pass: every tile counts its cells' vertices, publishes the count, and
// gets the chain-local offset of its first vertex by decoupled look-back over
// the tiles before it (tile order = order in which blocks took their ticket,
// so every tile waited on has started and publishes its count without
// waiting).  Each wait is bounded; it also gives up when the update halts.
constexpr unsigned long long LB_AGG = 1ull, LB_INC = 2ull, LB_MASK = (1ull << 62) - 1;
constexpr int LB_MAX_SPINS = 1 << 24;

__device__ __forceinline__ void lb_publish(unsigned long long *st, int64_t g, unsigned long long flag,
                                           int64_t v) {
  atomicExch(st + g, (flag << 62) | ((unsigned long long)v & LB_MASK));
}

// Warp-cooperative look-back (run by warp 0): lane l inspects tile g-1-l of a
// window of 32 predecessors; the window moves down until it holds a tile with
// an inclusive prefix.  first = the chain's first tile, which publishes its
// inclusive prefix at once, so the walk never leaves the chain.
__device__ int64_t lb_lookback(unsigned long long *st, int64_t g, int64_t first, const Scratch &s) {
  const int lane = threadIdx.x & 31;
  int64_t excl = 0;
  int spins = 0;
  for (int64_t p = g - 1;;) {
    const int64_t idx = p - lane;
    unsigned long long x = (LB_INC << 62);  // below the chain: inclusive 0
    if (idx >= first) x = *((volatile unsigned long long *)(st + idx));
    const unsigned long long f = x >> 62;
    const unsigned inc = __ballot_sync(0xffffffffu, f == LB_INC);
    const unsigned none = __ballot_sync(0xffffffffu, f == 0);
    const int k = inc ? __ffs(inc) - 1 : 31;  // lanes 0..k are summed
    if (none & (k == 31 ? 0xffffffffu : ((2u << k) - 1u))) {  // a tile up to lane k not ready
      if (++spins > LB_MAX_SPINS) {
        if (lane == 0) atomicOr(s.status, ST_TIMEOUT);
        return 0;
      }
      if ((spins & 255) == 0 && halted(s)) return 0;
      __nanosleep(32);
      continue;
    }
    long long v = (lane <= k) ? (long long)(x & LB_MASK) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (inc) return excl;
    p -= 32;
  }
}

// Candidate-parallel insertion.  A tile's cells first set up in shared memory
// (count K of Poisson candidates, parity at the window start, neighbour
// operator ranges); then the tile's Philox calls are spread over all threads
// (call 0 of a cell gives K and candidate 0, call m >= 1 candidates 2m-1 and
// 2m), each candidate's time is formed and the antiparallel test taken; the
// kept candidates' places inside their cell follow from ranks: among the
// cell's kept candidates by (u53, draw index), and against its old operators
// by time (an old operator goes first on a tie).  Every vertex is then written
// by its own thread (time, flag, cell; the parent forest is set by the linking
// kernels).  Candidates are staged INS_CAP at a time: a tile whose candidates
// exceed that (the mean is 8 * TILE) runs its cells in groups, counting in a
// first pass and drawing again in the writing pass.
constexpr int INS_CAP = 1280;
// Threads of an insertion block: one per cell for the set-up and the scans
// (the upper half only joins the scans with zeros), all of them for the
// candidates' draws and the vertices' writes.
constexpr int INS_THREADS = 256;
constexpr int INS_SPAN = INS_CAP - KMAX;  // a group's cells start within INS_SPAN slots
constexpr int INS_UCAP = INS_CAP / 2 + TILE;
constexpr int INS_MIN_SPAN = 256;  // smallest group span a chain may ask for (tests)
constexpr int INS_MAXG = (TILE * (KMAX - 1)) / INS_MIN_SPAN + 2;
constexpr int INS_OPCAP = 2048;  // old operators of a group mapped to their cell
constexpr unsigned long long KEY_DROP = 1ull << 63;

// Old operator times a tile stages in shared memory: its own cells' and those
// of the cells up to 8 Q^2 cells away (the neighbour bonds of the same
// windows), when they fit (about 1230 for a thermalized S = 1 tile).
template <int Q>
struct InsStage {
  static constexpr int N = Q == 1 ? 1024 : (Q == 2 ? 1536 : 2048);
};

// Where an old operator's time is read: from the staged copy if its index is
// in [lo, hi), else from global memory.
struct OpView {
  const long long *g;   // op_tau of the chain
  const long long *sv;  // staged copy, indexed like g (valid in [lo, hi))
  int lo, hi;
  __device__ __forceinline__ const long long *range(int a, int b) const {
    return (a >= lo && b <= hi) ? sv : g;
  }
};

template <int Q>
struct InsSmem {
  long long sop[InsStage<Q>::N];    // staged old operator times (16-byte aligned: first member)
  unsigned long long key[INS_CAP];  // (u53 << 6) | draw, with bit 63 set if the candidate is not kept
  long long tau[INS_CAP];           // time bits; LLONG_MAX if not kept
  short klist[INS_CAP];             // kept candidates' slots (any order)
  uint8_t scell[INS_CAP];           // slot -> cell in tile
  uint8_t ucell[INS_UCAP];          // Philox call -> cell in tile
  uint8_t qcell[INS_OPCAP];         // old operator -> cell in tile
  NbOps<Q> X[TILE];
  unsigned long long T[2][KMAX];    // Poisson thresholds: full windows, last window
  int kpre[TILE + 1], upre[TILE + 1], q[TILE + 1];
  int K[TILE], nk[TILE], cex[TILE], b[TILE], j[TILE];
  uint8_t par0[TILE];
  int gfirst[INS_MAXG + 1];
  int G, nkept;
  int sm[33];
  int slo, shi;
  uint64_t bar;
  int64_t excl;
  int64_t gt;
};

// Number of operators of one neighbour bond (times tq[lo..hi), ascending)
// that act before a candidate at time tau on bond b: order (time, bond).
__device__ __forceinline__ int ops_before(const long long *__restrict__ tq, int lo, int hi,
                                          long long tau, int bb, int b) {
  const long long thr = tau + (bb < b ? 1 : 0);  // t < thr  <=>  (t, bb) < (tau, b)
  const int base = lo;
  while (lo < hi) {
    const int mid = lo + ((hi - lo) >> 1);  // no overflow near 2^31
    if (tq[mid] < thr)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo - base;
}

// Time of a candidate, tau = fma(d, u53 2^-53, t0) (one IEEE fused
// multiply-add), and whether it is kept: the bond's spins antiparallel at tau
// (parity at the window start flipped by the neighbour operators before tau).
template <int Q>
__device__ __forceinline__ bool ins_decide(const OpView &V, const NbOps<Q> &X, int b, int par0,
                                           uint64_t u53, double t0, double d, long long teb,
                                           long long &tau) {
  tau = __double_as_longlong(__fma_rn(d, __longlong_as_double((long long)unit_bits(u53)), t0));
  if (!(tau < teb)) return false;
  int p = par0;
#pragma unroll
  for (int k = 0; k < NbOps<Q>::N; ++k)
    p ^= ops_before(V.range(X.o0[k], X.o1[k]), X.o0[k], X.o1[k], tau, X.bond[k], b);
  return p & 1;
}

// Draw and decide the candidates of the cells of group g.
template <int Q>
__device__ void ins_draw(const DevChain &C, InsSmem<Q> &S, const OpView &V, int g, bool count) {
  const int c0 = S.gfirst[g], c1 = S.gfirst[g + 1];
  const int kb = S.kpre[c0], ub = S.upre[c0], nu = S.upre[c1] - ub;
  {
    const int c = threadIdx.x;
    if (c >= c0 && c < c1)
      for (int u = S.upre[c], e = S.upre[c + 1]; u < e; ++u) S.ucell[u - ub] = (uint8_t)c;
    if (threadIdx.x == 0) S.nkept = 0;
  }
  __syncthreads();
  const uint32_t k0 = (uint32_t)C.seed, k1 = (uint32_t)(C.seed >> 32);
  const int lane = threadIdx.x & 31;
  for (int u0 = 0; u0 < nu; u0 += INS_THREADS) {  // whole warps, reconverged per step
    const int u = u0 + threadIdx.x;
    bool kp[2] = {false, false};
    int sl[2] = {0, 0}, c = 0;
    if (u < nu) {
      c = S.ucell[u];
      const int m = u + ub - S.upre[c];
      const int j = S.j[c], K = S.K[c], ks = S.kpre[c] - kb, b = S.b[c], par0 = S.par0[c];
      const NbOps<Q> X = S.X[c];
      const double t0 = __longlong_as_double((long long)C.win[3 * j]);
      const long long teb = (long long)C.win[3 * j + 1];
      const double d = __longlong_as_double((long long)C.win[3 * j + 2]);
      const U4 o = philox((TAG_INSERT << 24) | (uint32_t)m, (uint32_t)b, (uint32_t)j, C.sweep, k0, k1);
      // words (x, y): candidate 2m-1 (for m = 0 the count); words (z, w): candidate 2m
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 2 * m - 1 + h;
        if (k < 0 || k >= K) continue;
        const uint64_t u53 = (h ? ((uint64_t)o.z | ((uint64_t)o.w << 32))
                                : ((uint64_t)o.x | ((uint64_t)o.y << 32))) >> 11;
        long long tau;
        const bool keep = ins_decide<Q>(V, X, b, par0, u53, t0, d, teb, tau);
        const int slot = ks + k;
        // (u53, draw) packed into one key, unique within the cell
        S.key[slot] = ((u53 << 6) | (uint64_t)k) | (keep ? 0ull : KEY_DROP);
        S.tau[slot] = keep ? tau : LLONG_MAX;
        S.scell[slot] = (uint8_t)c;
        kp[h] = keep;
        sl[h] = slot;
      }
    }
    // kept list: one shared atomic per warp and half
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned km = __ballot_sync(0xffffffffu, kp[h]);
      if (km) {
        const int leader = __ffs(km) - 1;
        int at = 0;
        if (lane == leader) at = atomicAdd(&S.nkept, __popc(km));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (kp[h]) {
          S.klist[at + __popc(km & ((1u << lane) - 1u))] = (short)sl[h];
          if (count) atomicAdd(&S.nk[c], 1);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
}

// Place and write the vertices of the cells of group g (kept candidates, then
// old operators); vertex ids are chain-local, base = the tile's first id.
template <int Q>
__device__ void ins_write(const DevChain &C, InsSmem<Q> &S, const OpView &V, int g,
                          int64_t base, const Scratch &s) {
  const int c0 = S.gfirst[g], c1 = S.gfirst[g + 1];
  const int kb = S.kpre[c0];
  const int64_t vb = C.vtx_base;
  long long *vt = (long long *)s.vtau + vb;
  uint8_t *vf = s.vflag + vb, *vc = s.vcell + vb;
  const int nkept = S.nkept;
  for (int i0 = 0; i0 < nkept; i0 += INS_THREADS) {
    const int i = i0 + threadIdx.x;
    if (i >= nkept) {
      __syncwarp();
      continue;
    }
    const int slot = S.klist[i];
    const long long tau = S.tau[slot];
    const int c = S.scell[slot];
    const int ks = S.kpre[c] - kb, K = S.K[c];
    const unsigned long long key = S.key[slot];
    int r = 0;
    for (int x = 0; x < K; ++x) r += S.key[ks + x] < key;  // kept keys ahead (a dropped one has bit 63)
    // old operators at or before tau (ascending times)
    int lo = S.q[c], hi = S.q[c + 1];
    const int q0 = lo;
    const long long *otau = V.range(lo, hi);
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);  // no overflow near 2^31
      if (otau[mid] <= tau)
        lo = mid + 1;
      else
        hi = mid;
    }
    r += lo - q0;
    const int64_t pos = base + S.cex[c] + r;
    vt[pos] = tau;
    vf[pos] = 0;
    vc[pos] = (uint8_t)c;
    __syncwarp();
  }
  const int qa = S.q[c0], qb = S.q[c1], qt = S.q[0];
  const bool mapped = qb - qt <= INS_OPCAP;
  for (int q0 = qa; q0 < qb; q0 += INS_THREADS) {
    const int q = q0 + threadIdx.x;
    if (q >= qb) {
      __syncwarp();
      continue;
    }
    int c;
    if (mapped) {
      c = S.qcell[q - qt];
    } else {
      int lo = c0, hi = c1 - 1;  // largest c in [c0, c1) with S.q[c] <= q
      while (lo < hi) {
        const int mid = lo + ((hi - lo + 1) >> 1);
        if (S.q[mid] <= q)
          lo = mid;
        else
          hi = mid - 1;
      }
      c = lo;
    }
    const long long ot = (q >= V.lo && q < V.hi) ? V.sv[q] : V.g[q];
    const int ks = S.kpre[c] - kb, K = S.K[c];
    int r = q - S.q[c];
    for (int x = 0; x < K; ++x) r += S.tau[ks + x] < ot;
    const int64_t pos = base + S.cex[c] + r;
    vt[pos] = ot;
    vf[pos] = VF_OLD;
    vc[pos] = (uint8_t)c;
    __syncwarp();
  }
}

template <int Q>
__device__ __forceinline__ void insert_tile(InsSmem<Q> &S, DevChain *__restrict__ ch,
                                            const int2 *__restrict__ tab, int64_t blk0, int group,
                                            Scratch s);

// The staging area is static shared memory for Q = 1 and dynamic shared
// memory (above the 48 KB static limit) for the larger neighbour tables and
// operator stages of Q = 2, 3, 4.
template <int Q>
__global__ void __launch_bounds__(INS_THREADS, Q == 1 ? 5 : 4) k_insert(DevChain *__restrict__ ch,
                                                 const int2 *__restrict__ tab, int64_t blk0,
                                                 int group, Scratch s) {
  if constexpr (Q == 1) {
    __shared__ __align__(16) InsSmem<Q> S;
    insert_tile<Q>(S, ch, tab, blk0, group, s);
  } else {
    extern __shared__ __align__(16) unsigned char ins_dyn[];
    insert_tile<Q>(*reinterpret_cast<InsSmem<Q> *>(ins_dyn), ch, tab, blk0, group, s);
  }
}

template <int Q>
__device__ __forceinline__ void insert_tile(InsSmem<Q> &S, DevChain *__restrict__ ch,
                                            const int2 *__restrict__ tab, int64_t blk0, int group,
                                            Scratch s) {
  if (halted(s)) return;
  if (threadIdx.x == 0) S.gt = blk0 + (int64_t)atomicAdd(s.tickets + group, 1u);
  __syncthreads();
  const int64_t gt = S.gt;
  const int2 t = tab[gt];
  DevChain &C = ch[t.x];
  const int c = threadIdx.x;
  const bool own = c < TILE;  // this thread's cell (the upper half has none)
  const int cell = t.y * TILE + c;
  const bool valid = own && cell < C.ncell;
  const int cur = C.cur;
  const int32_t *op = C.op_ptr[cur];
  const long long *otau = (const long long *)C.op_tau[cur];
  const uint8_t *s0 = C.s0[cur];
  int32_t *vp = s.vptr + C.cell_off;
  if (threadIdx.x == 0) {
    // Stage the old operator times around the tile with one bulk copy
    // (16-byte bounds: op_tau has room for one time past its capacity),
    // overlapped with the cells' set-up.
    const int R = 8 * Q * Q;
    const int ce = min(C.ncell, t.y * TILE + TILE);
    int lo = op[max(0, t.y * TILE - R)] & ~1, hi = (op[min(C.ncell, ce + R)] + 1) & ~1;
    if (hi - lo > InsStage<Q>::N) {
      lo = op[min(C.ncell, t.y * TILE)] & ~1;
      hi = (op[ce] + 1) & ~1;
      if (hi - lo > InsStage<Q>::N) hi = lo;
    }
    S.slo = lo;
    S.shi = hi;
    mbar_init(&S.bar);
    if (hi > lo) bulk_g2s(S.sop, otau + lo, (uint32_t)(hi - lo) * 8u, &S.bar);
  }
  if (threadIdx.x < KMAX) {
    S.T[0][threadIdx.x] = c_T_full[threadIdx.x];
    S.T[1][threadIdx.x] = C.T_last[threadIdx.x];
  }
  __syncthreads();

  // -- per-cell setup --------------------------------------------------------
  // The lower half of the block takes the cells' neighbour ranges and spin
  // parities, the upper half their candidate counts (Philox call 0), side by
  // side.
  int q0 = 0, q1 = 0;
  if (valid) {
    int b, j;
    cell_bj(C, cell, b, j);
    const int ul = left_sub<Q>(b), ur = right_sub<Q>(b, C.L);
    const int blk = j / TW, jb = blk * TW;
    const uint8_t *prow = s.bpar + C.bpar_off + (int64_t)blk * C.nbond;
    int par0 = (s0[ul] ^ s0[ur]) & 1;
    NbOps<Q> X;
    int k = 0;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int u = side ? ur : ul;
#pragma unroll
      for (int m = 0; m < 2 * Q; ++m) {
        const int bb = inc_bond<Q>(u, m, C.L);
        if (bb == b) continue;
        const int cj = cell_of(C, bb, j), cs = cell_of(C, bb, jb);
        X.bond[k] = bb;
        X.o0[k] = op[cj];
        X.o1[k] = op[cj + 1];
        par0 ^= (prow[bb] ^ (op[cj] - op[cs])) & 1;
        ++k;
      }
    }
    S.X[c] = X;
    S.par0[c] = (uint8_t)par0;
    S.b[c] = b;
    S.j[c] = j;
    q0 = op[cell];
    q1 = op[cell + 1];
  } else if (!own && t.y * TILE + (c - TILE) < C.ncell) {
    const int cc = c - TILE;  // the cell whose count this thread draws
    int b, j, K = 0;
    cell_bj(C, t.y * TILE + cc, b, j);
    const uint64_t db = C.win[3 * j + 2];
    const U4 o0 = philox(TAG_INSERT << 24, (uint32_t)b, (uint32_t)j, C.sweep, (uint32_t)C.seed,
                         (uint32_t)(C.seed >> 32));
    const uint64_t U = (uint64_t)o0.x | ((uint64_t)o0.y << 32);
    const unsigned long long *T = S.T[j == C.nwin - 1 ? 1 : 0];
    // K = number of thresholds T[0..KMAX-2] at or below U (they ascend)
#pragma unroll
    for (int step = 32; step > 0; step >>= 1)
      if (K + step <= KMAX - 1 && T[K + step - 1] <= U) K += step;
    if ((long long)db <= 0) K = 0;  // empty last window
    S.K[cc] = K;
  } else if (!own) {
    S.K[c - TILE] = 0;  // cells past the chain's end
  }
  if (!valid) q0 = q1 = op[C.ncell];  // cells past the chain's end: empty ranges
  if (own) {
    S.nk[c] = 0;
    S.q[c] = q0;
  }
  if (c == TILE - 1) S.q[TILE] = q1;
  __syncthreads();
  const int K = own ? S.K[c] : 0, P = K ? K / 2 + 1 : 0;
  int tot;
  const int ex = block_excl_scan<int>(K | (P << 16), S.sm, tot);
  if (own) {
    // old operator -> cell map (all of the tile's operators, if they fit)
    const int qa = S.q[0];
    for (int q = q0; q < q1 && q - qa < INS_OPCAP; ++q) S.qcell[q - qa] = (uint8_t)c;
    S.kpre[c] = ex & 0xffff;
    S.upre[c] = ex >> 16;
  }
  if (c == TILE - 1) {
    S.kpre[TILE] = tot & 0xffff;
    S.upre[TILE] = tot >> 16;
  }
  __syncthreads();
  if (own) {
    const int span =
        (C.ins_span >= INS_MIN_SPAN && C.ins_span < INS_SPAN) ? C.ins_span : INS_SPAN;
    const int gc = S.kpre[c] / span;
    if (c == 0 || gc != S.kpre[c - 1] / span) S.gfirst[gc] = c;
    if (c == TILE - 1) {
      S.G = gc + 1;
      S.gfirst[gc + 1] = TILE;
    }
  }
  __syncthreads();
  const int G = S.G;
  if (S.shi > S.slo) {
    const bool ok = mbar_wait(&S.bar, 0);
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) atomicOr(s.status, ST_TIMEOUT);
      return;
    }
  }
  const OpView V{otau, S.sop - S.slo, S.slo, S.shi};

  // -- draw, decide and count ------------------------------------------------
  for (int g = 0; g < G; ++g) ins_draw<Q>(C, S, V, g, true);
  const int cnt = valid ? (q1 - q0) + S.nk[c] : 0;
  int ctot;
  const int cex = block_excl_scan<int>(cnt, S.sm, ctot);
  if (own) S.cex[c] = cex;

  // -- chain-local offset of the tile: decoupled look-back --------------------
  if (threadIdx.x < 32) {
    int64_t excl = 0;
    if (t.y == 0) {
      if (threadIdx.x == 0) lb_publish(s.tile_state, gt, LB_INC, ctot);
    } else {
      if (threadIdx.x == 0) lb_publish(s.tile_state, gt, LB_AGG, ctot);
      __syncwarp();
      excl = lb_lookback(s.tile_state, gt, gt - t.y, s);
      if (threadIdx.x == 0) lb_publish(s.tile_state, gt, LB_INC, excl + ctot);
    }
    if (threadIdx.x == 0) {
      S.excl = excl;
      if (t.y == C.ntile - 1) {
        C.n = excl + ctot;
        if (excl + ctot > C.vcap) atomicOr(s.status, ST_VTX_OVERFLOW);
        // vertex ids are int32 and per-tile loops step past the last id by
        // up to a block: keep every id below 2^31 - 4096
        if (excl + ctot > (int64_t)VTX_ID_LIMIT) atomicOr(s.status, ST_ID_OVERFLOW);
      }
    }
  }
  __syncthreads();
  const int64_t base = S.excl;
  if (base + ctot > C.vcap) return;  // overflow: the host grows the chain and replays
  if (valid) {
    vp[cell] = (int32_t)(base + S.cex[c]);
    if (cell == C.ncell - 1) vp[C.ncell] = (int32_t)(base + S.cex[c] + cnt);
  }

  // -- write -----------------------------------------------------------------
  for (int g = 0; g < G; ++g) {
    if (G > 1) ins_draw<Q>(C, S, V, g, false);
    ins_write<Q>(C, S, V, g, base, s);
    __syncthreads();
  }
}

// ---- per-chain scan of the tiles' new-operator counts ------------------------------
__global__ void __launch_bounds__(1024) k_scan_ops(DevChain *__restrict__ ch, Scratch s) {
  // Chunks of 4 x 1024 tiles: each thread loads four consecutive counts
  // (coalesced across the warp), one block scan per chunk; the next chunk's
  // loads are issued before the current chunk's scan.
  __shared__ int64_t sm[33];
  if (halted(s)) return;
  DevChain &C = ch[blockIdx.x];
  const int nt = C.ntile;
  const int64_t *cnt = s.tile_sum2 + C.tile0;
  int64_t *pref = s.tile_pref2 + C.tile0;
  constexpr int V = 4;
  const int chunk = V * (int)blockDim.x;
  int64_t v[V], nx[V];
  auto load = [&](int base, int64_t *x) {
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int i = base + V * (int)threadIdx.x + k;
      x[k] = (i < nt) ? cnt[i] : 0;
    }
  };
  load(0, v);
  int64_t run = 0;
  for (int base = 0; base < nt; base += chunk) {
    if (base + chunk < nt) load(base + chunk, nx);
    int64_t mine = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) mine += v[k];
    int64_t total;
    int64_t ex = run + block_excl_scan<int64_t>(mine, sm, total);
#pragma unroll
    for (int k = 0; k < V; ++k) {
      const int i = base + V * (int)threadIdx.x + k;
      if (i < nt) pref[i] = ex;
      ex += v[k];
    }
    run += total;
#pragma unroll
    for (int k = 0; k < V; ++k) v[k] = nx[k];
  }
  if (threadIdx.x == 0) {
    C.n_off_new = run;
    if (run > C.op_cap) atomicOr(s.status, ST_OP_OVERFLOW);
  }
}

// ---- tau = 0: last leg per subsite, subspin permutation, cut predecessors -----
template <int Q>
__device__ void last_leg(const DevChain &C, const int32_t *vp, const long long *vtau, int64_t vb,
                         int bond, int &id, int &cellc, long long &tau) {
  id = -1;
  cellc = -1;
  tau = 0;
  for (int j = C.nwin - 1; j >= 0; --j) {
    const int c = cell_of(C, bond, j);
    const int a = vp[c], e = vp[c + 1];
    if (e > a) {
      id = e - 1;
      cellc = c;
      tau = vtau[vb + id];
      return;
    }
  }
}

template <int Q>
__global__ void __launch_bounds__(SITE_BLOCK) k_cut(const DevChain *__restrict__ ch,
                                                    const int2 *__restrict__ tab, int64_t blk0,
                                                    Scratch s) {
  if (halted(s)) return;
  const int2 t = tab[blk0 + blockIdx.x];
  const DevChain &C = ch[t.x];
  const int i = t.y * SITE_BLOCK + threadIdx.x;
  if (i >= C.L) return;
  const int32_t *vp = s.vptr + C.cell_off;
  const int64_t vb = C.vtx_base;
  const uint8_t *s0 = C.s0[C.cur];
  const uint8_t *ptot = s.bpar + C.bpar_off + (int64_t)C.nblk * C.nbond;
  int last[Q], lastc[Q], top[Q];
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    const int u = i * Q + a;
    int best = -1, bestc = -1;
    long long bt = 0;
    int par = 0;
#pragma unroll
    for (int m = 0; m < 2 * Q; ++m) {
      const int bb = inc_bond<Q>(u, m, C.L);
      par ^= ptot[bb];
      int id, cc;
      long long tt;
      last_leg<Q>(C, vp, (const long long *)s.vtau, vb, bb, id, cc, tt);
      if (id >= 0 && (best < 0 || tt > bt || (tt == bt && id > best))) {
        best = id;
        bt = tt;
        bestc = cc;
      }
    }
    last[a] = best;
    lastc[a] = bestc;
    top[a] = (s0[u] ^ par) & 1;
  }
  // perm[a]: the bottom subspin that the top of subspin a continues into.
  int perm[Q];
  if (Q == 1) {
    perm[0] = 0;
  } else if (Q > 2) {
    // Uniform among the permutations that join every top to a bottom of the
    // same spin (heat bath of the symmetrization, Sec. 5): tops and bottoms of
    // spin 1, then of spin 0, in subspin order; each bottom list shuffled by
    // Fisher-Yates from the last place down, place j drawn as
    // floor(w (j+1) / 2^32) with w the next word of
    // Philox(((TAG_PERM << 24) | 1, i, 0, sweep)); the m-th top of each spin
    // continues into the m-th shuffled bottom.
    int tops[2][Q], bots[2][Q], nt[2] = {0, 0}, nb[2] = {0, 0};
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int gt = top[a] ? 0 : 1, gb = (s0[i * Q + a] & 1) ? 0 : 1;
      tops[gt][nt[gt]++] = a;
      bots[gb][nb[gb]++] = a;
    }
#pragma unroll
    for (int a = 0; a < Q; ++a) perm[a] = a;
    if (nt[0] != nb[0]) {
      atomicOr(s.status, ST_BADSTATE);
    } else {
      const U4 o = philox((TAG_PERM << 24) | 1u, (uint32_t)i, 0u, C.sweep, (uint32_t)C.seed,
                          (uint32_t)(C.seed >> 32));
      const uint32_t w[4] = {o.x, o.y, o.z, o.w};
      int d = 0;
      for (int g = 0; g < 2; ++g) {
        for (int j = nb[g] - 1; j >= 1; --j) {
          const int r = (int)__umulhi(w[d++ & 3], (uint32_t)(j + 1));
          const int tmp = bots[g][j];
          bots[g][j] = bots[g][r];
          bots[g][r] = tmp;
        }
        for (int m = 0; m < nt[g]; ++m) perm[tops[g][m]] = bots[g][m];
      }
    }
  } else {
    const int b0 = s0[i * Q] & 1, b1 = s0[i * Q + (Q > 1 ? 1 : 0)] & 1;
    const bool ok_id = (top[0] == b0) && (top[1] == b1);
    const bool ok_sw = (top[0] == b1) && (top[1] == b0);
    int sw;
    if (ok_id && ok_sw)
      sw = coin(C, TAG_PERM, (uint32_t)i);
    else if (ok_sw)
      sw = 1;
    else if (ok_id)
      sw = 0;
    else {
      atomicOr(s.status, ST_BADSTATE);
      sw = 0;
    }
    perm[0] = sw ? 1 : 0;
    perm[1] = sw ? 0 : 1;
  }
#pragma unroll
  for (int a = 0; a < Q; ++a) {
    // Walk down through the cut: the bottom of subspin a is entered from the
    // top of pinv(a), then possibly through empty subspins.
    int x = a, cross = 0, node = -1, ncell = -1, mn = a, len = 0;
    for (int step = 0; step < Q; ++step) {
      int y = 0;
#pragma unroll
      for (int z = 0; z < Q; ++z)
        if (perm[z] == x) y = z;
      x = y;
      ++cross;
      if (last[x] >= 0) {
        node = last[x];
        ncell = lastc[x];
        break;
      }
      mn = min(mn, x);
      ++len;
      if (x == a) break;
    }
    const int64_t u = C.sub_off + i * Q + a;
    s.cut_node[u] = node;
    s.cut_cell[u] = ncell;
    s.cut_cross[u] = (int8_t)cross;
    s.free_min[u] = (node < 0) ? i * Q + mn : -1;
    s.free_len[u] = (int8_t)len;
  }
}

// ---- linking + union-find -----------------------------------------------------
__device__ __forceinline__ int before_window(const DevChain &C, const int32_t *vp, int bond, int j) {
  for (int jj = j - 1; jj >= 0; --jj) {
    const int c = cell_of(C, bond, jj);
    const int a = vp[c], e = vp[c + 1];
    if (e > a) return e - 1;
  }
  return -1;
}

// Per-cell linking context, staged in shared memory by one thread per cell.
template <int Q>
struct LinkCell {
  static constexpr int NO = 2 * Q - 1;  // other bonds touching each of the two subsites
  int wa[2][NO], we[2][NO], bj[2][NO];
  int own_bj, cut[2];
};

// Union-find of one tile's nodes in shared memory (local ids), with the same
// min-root rule as the global one: lp[x] <= x; a link is one CAS on the larger
// root.  Walks are bounded by the tile's node count.
__device__ __forceinline__ int suf_find(volatile int *lp, int x, int bound, int *status) {
  for (int it = 0; it <= bound; ++it) {
    const int p = lp[x];
    if (p == x) return x;
    const int g = lp[p];
    if (g != p) lp[x] = g;  // path halving (g is an ancestor of x)
    x = g;
  }
  atomicOr(status, ST_TIMEOUT);
  return x;
}

__device__ __forceinline__ void suf_union(int *lp, int a, int b, int bound, int *status) {
  for (int it = 0; it <= bound; ++it) {
    a = suf_find(lp, a, bound, status);
    b = suf_find(lp, b, bound, status);
    if (a == b) return;
    if (a > b) {
      const int t = a;
      a = b;
      b = t;
    }
    if (atomicCAS(lp + b, b, a) == b) return;
  }
  atomicOr(status, ST_TIMEOUT);
}

// First index q in [lo, hi) with vt[q] >= thr.  For a neighbour cell, whose
// ids are all below w or all above it, "key (tau, id) below (tw, w)" is
// vt[q] < tw + 1 or vt[q] < tw respectively.
__device__ __forceinline__ int time_lower_bound(const long long *vt, int lo, int hi, long long thr) {
  while (lo < hi) {
    const int mid = lo + ((hi - lo) >> 1);  // no overflow near 2^31
    if (vt[mid] < thr)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Linking, then the union of the two fragments below every vertex.  Edges
// with both nodes in the tile are united in shared memory, and the tile's
// forest is then stored flat: every node points at its tile component's
// root, its smallest node.  Edges
// that leave the tile are marked and united in the global forest by k_link_x,
// after every tile has stored its forest (a tile too large for shared memory
// leaves all of its edges to k_link_x, with every node its own root).
template <int Q>
__global__ void __launch_bounds__(TPB) k_link(const DevChain *__restrict__ ch,
                                              const int2 *__restrict__ tab, int64_t blk0,
                                              Scratch s) {
  __shared__ LinkCell<Q> lc[TILE];
  __shared__ int cvp[TILE + 1];
  __shared__ int lp[SMEM_CAP];
  if (halted(s)) return;
  const int2 t = tab[blk0 + blockIdx.x];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE), ncl = c1 - c0;
  const int32_t *vp = s.vptr + C.cell_off;
  for (int i = threadIdx.x; i <= ncl; i += blockDim.x) cvp[i] = vp[c0 + i];
  if (threadIdx.x < ncl) {
    LinkCell<Q> &L = lc[threadIdx.x];
    int b, j;
    cell_bj(C, c0 + threadIdx.x, b, j);
    const int sub[2] = {left_sub<Q>(b), right_sub<Q>(b, C.L)};
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      int k = 0;
#pragma unroll
      for (int m = 0; m < 2 * Q; ++m) {
        const int bb = inc_bond<Q>(sub[sd], m, C.L);
        if (bb == b) continue;
        const int cj = cell_of(C, bb, j);
        L.wa[sd][k] = vp[cj];
        L.we[sd][k] = vp[cj + 1];
        L.bj[sd][k] = before_window(C, vp, bb, j);
        ++k;
      }
      L.cut[sd] = s.cut_node[C.sub_off + sub[sd]];
    }
    L.own_bj = before_window(C, vp, b, j);
  }
  __syncthreads();
  const int a = cvp[0], e = cvp[ncl], nv = e - a;
  const bool local = nv <= local_cap(C);
  if (local)
    for (int i = threadIdx.x; i < nv; i += blockDim.x) lp[i] = i;
  __syncthreads();
  const int64_t vb = C.vtx_base, wb = vb >> 5;
  const long long *__restrict__ vt = (const long long *)s.vtau + vb;
  int32_t *par = s.parent + vb;
  // Whole warps walk the tile (trip count rounded up) and reconverge after
  // every vertex, so that the divergent union of one iteration does not split
  // the next one's predecessor search.
  for (int w0 = a; w0 < e; w0 += blockDim.x) {
    const int w = w0 + threadIdx.x;
    if (w >= e) {
      __syncwarp();
      continue;
    }
    const int ci = s.vcell[vb + w];
    const LinkCell<Q> &L = lc[ci];
    const int v0 = cvp[ci];
    const long long tw = vt[w];
    int P[2];
    uint8_t wrapbits = 0;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      int best = -1;
      long long bt = 0;
      if (w > v0) {
        best = w - 1;
        bt = vt[w - 1];
      } else if (L.own_bj >= 0) {
        best = L.own_bj;
        bt = vt[best];
      }
#pragma unroll
      for (int k = 0; k < LinkCell<Q>::NO; ++k) {
        const int q = time_lower_bound(vt, L.wa[sd][k], L.we[sd][k], tw + (L.wa[sd][k] < w ? 1 : 0));
        const int cand = (q > L.wa[sd][k]) ? q - 1 : L.bj[sd][k];
        if (cand >= 0) {
          const long long tc = vt[cand];
          if (best < 0 || tc > bt || (tc == bt && cand > best)) {
            best = cand;
            bt = tc;
          }
        }
      }
      if (best < 0) {
        best = L.cut[sd];
        wrapbits |= sd ? VF_WRAP_R : VF_WRAP_L;
        if (best < 0) {
          fail_check(s, 2, c0 + ci, w, sd, 0, 0);
          best = w;
        }
      }
      P[sd] = best;
    }
    s.pl[vb + w] = P[0];
    s.pr[vb + w] = P[1];
    if (wrapbits) s.vflag[vb + w] |= wrapbits;
    const bool inside = P[0] >= a && P[0] < e && P[1] >= a && P[1] < e;
    if (!inside) {
      set_bit(s.openmark, wb, P[0]);
      if (local && P[0] != P[1]) set_bit(s.xmark, wb, w);
    } else if (local && P[0] != P[1]) {
      suf_union(lp, P[0] - a, P[1] - a, nv, s.status);
    }
    __syncwarp();
  }
  __syncthreads();
  if (local) {
    // Every node walks to its root and stores it (in shared memory too, which
    // shortens the walks of the nodes below it).  Each store writes an
    // ancestor of the old word, so concurrent walks still end at the root;
    // the walks are bounded by the tile's node count.  One pass without
    // barriers (pointer jumping, one barrier per round: 0.83 -> 0.81 ms at
    // L=16384, beta=4096).
    volatile int *vlp = lp;
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
      int r = vlp[i];
      for (int it = 0; it < SMEM_CAP; ++it) {
        const int q = vlp[r];
        if (q == r) break;
        r = q;
      }
      vlp[i] = r;
      par[a + i] = a + r;
    }
  } else {
    for (int v = a + threadIdx.x; v < e; v += blockDim.x) par[v] = v;
  }
}

// Global unions of the edges that leave their tile (all edges of a tile too
// large for shared memory), on the forests the tiles stored.  One warp per
// tile, eight tiles per block: a tile has about 45 words of marks, and the
// unions are chains of dependent global loads, so many tiles are kept in
// flight.
constexpr int TPB_X = 256;
constexpr int XLIST = 256;  // crossing edges of a tile listed per warp

__global__ void __launch_bounds__(TPB_X) k_link_x(const DevChain *__restrict__ ch,
                                                const int2 *__restrict__ tab, int64_t ntiles,
                                                Scratch s) {
  __shared__ int xlist[TPB_X / 32][XLIST];
  if (halted(s)) return;
  const int lane = threadIdx.x & 31;
  const int64_t gt = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (gt >= ntiles) return;
  const int2 t = tab[gt];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE);
  const int32_t *vp = s.vptr + C.cell_off;
  const int a = vp[c0], e = vp[c1];
  const bool local = e - a <= local_cap(C);
  const int64_t vb = C.vtx_base;
  int32_t *par = s.parent + vb;
  if (!local) {
    for (int w = a + lane; w < e; w += 32) uf_union(par, s.pl[vb + w], s.pr[vb + w], s.status, s.uf_limit);
    return;
  }
  // The tile's crossing edges cluster at its first vertices (its first bond's
  // cells): they are listed first (a warp scan of the mark words' counts) and
  // then taken round-robin by the lanes, so that no lane walks most of them.
  int *list = xlist[threadIdx.x >> 5];
  const int64_t wfirst = (vb + a) >> 5, wlast = (vb + e - 1) >> 5;
  int nlist = 0;
  for (int64_t w0 = wfirst; e > a && w0 <= wlast; w0 += 32) {  // the same trip count on every lane
    const int64_t wd = w0 + lane;
    uint32_t bits = 0u;
    const int64_t v0 = (wd << 5) - vb;
    if (wd <= wlast) {
      bits = __ldcg(s.xmark + wd);
      if (v0 < a) bits &= ~0u << (a - v0);
      if (v0 + 32 > e) bits &= (e - v0 >= 32) ? ~0u : ((1u << (e - v0)) - 1u);
    }
    const int cnt = __popc(bits);
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    int at = nlist + inc - cnt;
    while (bits) {
      const int w = (int)v0 + __ffs(bits) - 1;
      bits &= bits - 1;
      if (at < XLIST)
        list[at] = w;
      else
        uf_union(par, s.pl[vb + w], s.pr[vb + w], s.status, s.uf_limit);  // past the list
      ++at;
    }
    nlist += __shfl_sync(0xffffffffu, inc, 31);
  }
  __syncwarp();
  for (int i = lane; i < min(nlist, XLIST); i += 32) {
    const int w = list[i];
    uf_union(par, s.pl[vb + w], s.pr[vb + w], s.status, s.uf_limit);
  }
}

// ---- compression + coins --------------------------------------------------------
__global__ void __launch_bounds__(TILE) k_compress(const DevChain *__restrict__ ch,
                                                   const int2 *__restrict__ tab, int64_t blk0,
                                                   Scratch s) {
  __shared__ U4 coins[MAX_COIN_GROUPS];
  __shared__ int64_t sm[33];
  __shared__ int spar[SMEM_CAP];  // the tile's parent words: walks stay here until they leave it
  if (halted(s)) return;
  const int64_t gt = blk0 + blockIdx.x;
  const int2 t = tab[gt];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE);
  const int32_t *vp = s.vptr + C.cell_off;
  const int a = vp[c0], e = vp[c1];
  const int64_t vb = C.vtx_base, wb = vb >> 5;
  int32_t *par = s.parent + vb;
  const bool oversized = (e - a) > local_cap(C);
  const int g0 = a >> 7;
  const int ng = (e > a) ? ((e - 1) >> 7) - g0 + 1 : 0;
  const uint32_t k0 = (uint32_t)C.seed, k1 = (uint32_t)(C.seed >> 32);
  for (int g = threadIdx.x; g < ng && g < MAX_COIN_GROUPS; g += blockDim.x)
    coins[g] = philox(TAG_FLIP << 24, (uint32_t)(g0 + g), 0u, C.sweep, k0, k1);
  // Only this block writes parent words of [a, e) in this kernel, and every
  // word it writes is an ancestor of the old one: the copy stays a valid forest.
  // Words that point out of the tile (parents are never larger than their
  // children, so outside means below a) are resolved first, each with one
  // global walk to its root, so that the nodes walking through them share
  // that walk; every other walk then stays in shared memory.  The shared copy
  // and the global words agree after that pass, and a node's word is stored
  // only if its root differs from it (linking left most words at their root:
  // 0.31 -> 0.28 ms at L=16384, beta=4096).
  if (!oversized) {
    for (int i = threadIdx.x; i < e - a; i += blockDim.x) {
      const int p = __ldcg(par + a + i);
      int q = p;
      if (p < a) {
        q = uf_root(par, p, s.status, s.uf_limit);
        if (q != p) par[a + i] = q;
      }
      spar[i] = q;
    }
  }
  __syncthreads();
  int64_t roots = 0;
  for (int v0 = a; v0 < e; v0 += blockDim.x) {  // whole warps, reconverged per step
    const int v = v0 + threadIdx.x;
    if (v >= e) {
      __syncwarp();
      continue;
    }
    int r;
    if (oversized) {
      r = uf_root(par, v, s.status, s.uf_limit);
    } else {
      // the walk ends at a root of the tile, or at a resolved outside root
      r = v;
      int p = spar[v - a];
      for (int it = 0; p != r && p >= a && it < SMEM_CAP; ++it) {
        r = p;
        p = spar[p - a];
      }
      if (p != r) r = (p < a) ? p : uf_root(par, p, s.status, s.uf_limit);
    }
    if (r != (oversized ? v : spar[v - a])) par[v] = r;  // only words that change
    if (r == v) {
      ++roots;
      const int g = (v >> 7) - g0;
      const int cf = (g < MAX_COIN_GROUPS) ? coin_from(coins[g], (uint32_t)v) : coin(C, TAG_FLIP, v);
      if (cf) set_bit(s.flipbits, wb, v);
      if (oversized) set_bit(s.openroot, wb, v);
    }
    if (get_bit(s.openmark, wb, v)) set_bit(s.openroot, wb, r);
    __syncwarp();
  }
  const int64_t tot = block_sum<int64_t>(roots, sm);
  if (threadIdx.x == 0) s.tile_roots[gt] = tot;
}

// ---- opt-in check of the loop forest after compression ----------------------------
// Every node's word is its loop's root, a root is its own parent and no parent
// is larger than its child (min-root rule).  The first violation is reported
// as consistency check 10 (chain, node, word, word of the word).
__global__ void __launch_bounds__(TILE) k_check_forest(const DevChain *__restrict__ ch,
                                                       const int2 *__restrict__ tab, Scratch s) {
  if (halted(s)) return;
  const int2 t = tab[blockIdx.x];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE);
  const int32_t *vp = s.vptr + C.cell_off;
  const int a = vp[c0], e = vp[c1];
  const int32_t *par = s.parent + C.vtx_base;
  for (int v = a + threadIdx.x; v < e; v += blockDim.x) {
    const int r = __ldcg(par + v);
    const int rr = (r >= 0 && r <= v) ? __ldcg(par + r) : -1;
    if (r < 0 || r > v || rr != r) fail_check(s, 10, t.x, v, r, rr, 0);
  }
}

// ---- loop properties, new flags ---------------------------------------------------
// Exact 64-bit two's-complement sums kept in shared memory as two 32-bit words
// and added with native 32-bit atomics (a 64-bit shared-memory add would be a
// compare-and-swap loop): the low word first, then the high word plus the
// carry out of the low word.
__device__ __forceinline__ void sadd64(unsigned *w, long long x) {
  const unsigned lo = (unsigned)x, hi = (unsigned)((unsigned long long)x >> 32);
  const unsigned old = atomicAdd(w, lo);
  const unsigned h = hi + ((old + lo < old) ? 1u : 0u);
  if (h) atomicAdd(w + 1, h);
}

__device__ __forceinline__ unsigned long long sget64(const unsigned *w) {
  return ((unsigned long long)w[1] << 32) | w[0];
}

// Per-tile table of loop sums keyed by root: a vertex of a loop of more than
// one node adds its (W, C, S, Zr, Zi) to its root's slot (linear probing,
// split sums).  If the table is full the sums go to the root's global record
// and the root is marked open, so that they are squared with the open loops.
constexpr int LOOP_SLOTS = 256;
constexpr int LOOP_SUMS = 5;  // W, C, S, Zr, Zi

struct LoopSums {
  long long v[LOOP_SUMS];
};

// Adds a loop's first NS sums to the global record of its root (vertex v):
// W, C, S, Zr in one 32-byte record, Zi beside it in its own array.
template <int NS>
__device__ __forceinline__ void acc_add(const Scratch &s, int64_t v, const long long *x) {
  unsigned long long *r = s.acc + ACC_WORDS * v;
#pragma unroll
  for (int i = 0; i < NS; ++i) atomicAdd(i < ACC_WORDS ? r + i : s.accz + v, (unsigned long long)x[i]);
}

// NS: how many of the sums are carried (3 without the temporal moment).
// mask = slots in use - 1 (LOOP_SLOTS - 1 unless a test shrinks the table).
template <int NS>
__device__ __forceinline__ void loop_add(int *keys, unsigned *vals, int key, const LoopSums &x,
                                         const Scratch &s, int64_t vb, unsigned mask) {
  unsigned h = (((unsigned)key * 2654435761u) >> 24) & mask;  // top 8 bits: LOOP_SLOTS = 256
  for (unsigned probe = 0; probe <= mask; ++probe) {
    int k = keys[h];
    if (k == -1) {
      k = atomicCAS(keys + h, -1, key);
      if (k == -1) k = key;
    }
    if (k == key) {
#pragma unroll
      for (int i = 0; i < NS; ++i) sadd64(vals + 2 * (NS * h + i), x.v[i]);
      return;
    }
    h = (h + 1) & mask;
  }
  acc_add<NS>(s, vb + key, x.v);
  set_bit(s.openroot, vb >> 5, key);
}

// Squares of one loop's sums: W^2 to w2, C^2 + S^2 to f2, (T) Zr^2 + Zi^2 to z2.
template <bool T>
__device__ __forceinline__ void loop_squares(const long long *v, u128 &w2, u128 &f2, u128 &z2) {
  w2 += sq_abs(v[0]);
  f2 += sq_abs(v[1]) + sq_abs(v[2]);
  if (T) z2 += sq_abs(v[3]) + sq_abs(v[4]);
}

constexpr int TPB_EST = 256;
// Vertices of a tile whose ticks (and phase factors) the loop-properties
// kernel stages in shared memory; ticks beyond it are computed where needed.
constexpr int EST_STAGE = 1536;

// T: also the temporal moment (phase factors, Zr and Zi); off by default.
template <int Q, bool T>
__global__ void __launch_bounds__(TPB_EST, T ? 6 : 8) k_est(const DevChain *__restrict__ ch,
                                             const int2 *__restrict__ tab, int64_t blk0,
                                             Scratch s) {
  __shared__ int lkeys[LOOP_SLOTS];
  constexpr int NS = T ? LOOP_SUMS : 3;  // sums carried per loop
  __shared__ unsigned lvals[2 * NS * LOOP_SLOTS];
  __shared__ int cvp[TILE + 1];
  __shared__ int cnew[TILE];
  __shared__ long long ccl[TILE], csl[TILE], ccr[TILE], csr[TILE], cxl[TILE], cxr[TILE];
  extern __shared__ long long est_dyn[];
  long long *qv = est_dyn;                   // ticks q(tau) of the tile's vertices
  int2 *ev = (int2 *)(est_dyn + EST_STAGE);  // their phase factors exp(i w1 tau)
  if (halted(s)) return;
  const int64_t gt = blk0 + blockIdx.x;
  const int2 t = tab[gt];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE), ncl = c1 - c0;
  const int32_t *vp = s.vptr + C.cell_off;
  const int a = vp[c0], e = vp[c1];
  const int64_t vb = C.vtx_base, wb = vb >> 5;
  const int32_t *par = s.parent + vb;
  const uint64_t *vt = (const uint64_t *)s.vtau + vb;
  const int F = C.F;
  // Ticks of every vertex of the tile, once: the fragments below a vertex
  // mostly start at vertices of the same tile.
  // Their phase factors too (temporal moment, w1 = 2 pi / beta).  They are
  // staged beside the cells' set-up, before the one barrier (behind a barrier
  // of their own the kernel took 0.866 ms instead of 0.854 at L=16384,
  // beta=4096).
  const uint64_t phR = C.phR;
  const int phS = C.phS;
  const int nq = min(min(e - a, local_cap(C)), EST_STAGE);
  const unsigned slot_mask =
      (C.loop_slots > 0 && C.loop_slots <= LOOP_SLOTS && !(C.loop_slots & (C.loop_slots - 1)))
          ? (unsigned)C.loop_slots - 1u
          : (unsigned)LOOP_SLOTS - 1u;
  for (int i = threadIdx.x; i < nq; i += blockDim.x) {
    const long long q = q_time(vt[a + i], F);
    qv[i] = q;
    if (T) ev[i] = phase_of((uint64_t)q, phR, phS, g_phase_tab);
  }
  for (int i = threadIdx.x; i <= ncl; i += blockDim.x) cvp[i] = vp[c0 + i];
  if (threadIdx.x < ncl) {
    // per cell: Fourier weights of its two sites, cut crossings (in ticks)
    int b, j;
    cell_bj(C, c0 + threadIdx.x, b, j);
    const int ul = left_sub<Q>(b), ur = right_sub<Q>(b, C.L);
    const int xl = ul / Q, xr = ur / Q;
    ccl[threadIdx.x] = C.cosq[xl];
    csl[threadIdx.x] = C.sinq[xl];
    ccr[threadIdx.x] = C.cosq[xr];
    csr[threadIdx.x] = C.sinq[xr];
    cxl[threadIdx.x] = (long long)s.cut_cross[C.sub_off + ul] * C.qbeta;
    cxr[threadIdx.x] = (long long)s.cut_cross[C.sub_off + ur] * C.qbeta;
    cnew[threadIdx.x] = 0;
  }
  for (int i = threadIdx.x; i < LOOP_SLOTS; i += blockDim.x) {
    lkeys[i] = -1;
#pragma unroll
    for (int k = 0; k < 2 * NS; ++k) lvals[2 * NS * i + k] = 0u;
  }
  __syncthreads();
  auto inq = [&](int v) { return v >= a && v < a + nq; };
  auto ticks = [&](int v) { return inq(v) ? qv[v - a] : q_time(vt[v], F); };
  auto phase = [&](int v) {
    return inq(v) ? ev[v - a] : phase_of((uint64_t)q_time(vt[v], F), phR, phS, g_phase_tab);
  };
  // Whole warps walk the tile (trip count rounded up), reconverging after
  // every vertex.
  u128 w2 = 0, f2 = 0, z2 = 0;  // this thread's share of the loops' squared sums
  for (int w0 = a; w0 < e; w0 += blockDim.x) {
    const int w = w0 + threadIdx.x;
    if (w < e) {
      const int ci = s.vcell[vb + w];
      const int P = s.pl[vb + w], R = s.pr[vb + w];
      const uint8_t f = s.vflag[vb + w];
      // a node whose two upper legs both end at w is a loop by itself: its
      // own root
      const int rb = (P == R) ? P : __ldcg(par + P), ra = __ldcg(par + w);
      const int nf = (f & VF_OLD) ^ get_bit(s.flipbits, wb, rb) ^ get_bit(s.flipbits, wb, ra);
      s.vflag[vb + w] = (uint8_t)(f | (nf ? VF_NEW : 0));
      if (nf) atomicAdd(cnew + ci, 1);
      // fragment lengths in ticks of 2^-F: q(tau_top) - q(tau_bottom) (+ crossings)
      const long long qw = ticks(w);
      const long long qP = ticks(P);
      long long dl = qw - qP;
      if (f & VF_WRAP_L) dl += cxl[ci];
      long long dr = qw - (R == P ? qP : ticks(R));
      if (f & VF_WRAP_R) dr += cxr[ci];
      LoopSums x;
      x.v[0] = dl + dr;
      x.v[1] = mul_q32(dl, ccl[ci]) + mul_q32(dr, ccr[ci]);
      x.v[2] = mul_q32(dl, csl[ci]) + mul_q32(dr, csr[ci]);
      // int over a fragment of e^{i w1 t} dt = (e(top) - e(bottom)) / (i w1),
      // across the cut too (e(t + beta) = e(t)): both fragments end at w
      x.v[3] = x.v[4] = 0;
      if (T) {
        const int2 ew = phase(w), eP = phase(P), eR = (R == P) ? eP : phase(R);
        x.v[3] = 2ll * ew.x - eP.x - eR.x;
        x.v[4] = 2ll * ew.y - eP.y - eR.y;
      }
      if (P == R) {
        // Both upper legs of node P end at w, so P is a loop by itself and its
        // two fragments are the two below w: the loop's sums are complete here.
        loop_squares<T>(x.v, w2, f2, z2);
      } else {
        loop_add<NS>(lkeys, lvals, rb, x, s, vb, slot_mask);
      }
    }
    __syncwarp();
  }
  __syncthreads();
  long long newcnt = 0;
  if (threadIdx.x < ncl) {
    newcnt = cnew[threadIdx.x];
    C.op_ptr[C.cur ^ 1][c0 + threadIdx.x] = (int32_t)newcnt;
  }
  // A loop closed in the tile is complete in its slot: square it here.  A loop
  // that leaves the tile adds its slot to the root's global record, squared
  // once every tile has added (next operator list kernel).
  for (int h = threadIdx.x; h < LOOP_SLOTS; h += blockDim.x) {
    const int kk = lkeys[h];
    if (kk < 0) continue;
    long long v[LOOP_SUMS] = {};
#pragma unroll
    for (int i = 0; i < NS; ++i) v[i] = (long long)sget64(lvals + 2 * (NS * h + i));
    if (get_bit(s.openroot, wb, kk)) {
      acc_add<NS>(s, vb + kk, v);
    } else {
      loop_squares<T>(v, w2, f2, z2);
    }
  }
  block_sums<T>(newcnt, w2, f2, z2);
  if (threadIdx.x == 0) {
    s.tile_sum2[gt] = newcnt;
    s.tile_sw2[2 * gt] = (unsigned long long)w2;
    s.tile_sw2[2 * gt + 1] = (unsigned long long)(w2 >> 64);
    s.tile_sf2[2 * gt] = (unsigned long long)f2;
    s.tile_sf2[2 * gt + 1] = (unsigned long long)(f2 >> 64);
    s.tile_sz2[2 * gt] = (unsigned long long)z2;
    s.tile_sz2[2 * gt + 1] = (unsigned long long)(z2 >> 64);
  }
}

// ---- next operator list + open loops -------------------------------------------------
// The tile's flags are read as aligned 32-bit words (four vertices each).
// Each warp takes a contiguous range of words: a first pass counts its new
// operators, one barrier exchanges the warp totals, and a second pass places
// them with warp shuffles (id order = order of the next operator list).  The
// cell offsets come from a block scan of the per-cell counts.
template <bool T>
__global__ void __launch_bounds__(TPB, T ? 4 : 8) k_compact(const DevChain *__restrict__ ch,
                                                 const int2 *__restrict__ tab, int64_t blk0,
                                                 Scratch s) {
  __shared__ int64_t sm[33];
  __shared__ int wtot[TPB / 32];
  if (halted(s)) return;
  const int64_t gt = blk0 + blockIdx.x;
  const int2 t = tab[gt];
  const DevChain &C = ch[t.x];
  const int c0 = t.y * TILE, c1 = min(C.ncell, c0 + TILE), ncl = c1 - c0;
  int32_t *nptr = C.op_ptr[C.cur ^ 1];
  double *ntau = C.op_tau[C.cur ^ 1];
  const int32_t *vp = s.vptr + C.cell_off;
  const int64_t vb = C.vtx_base;
  const int64_t base = s.tile_pref2[gt];
  const int a = vp[c0], e = vp[c1];
  const uint8_t *vf = s.vflag + vb;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = TPB / 32;
  // words [wa, we) of four flags; warp wid takes [wa + wid*per, ...)
  const int wa = a >> 2, we = (e + 3) >> 2;
  const int per = (we - wa + nw - 1) / nw;
  const int ww0 = min(we, wa + wid * per), ww1 = min(we, ww0 + per);
  auto newmask = [&](int wd) {  // bit i: vertex 4*wd + i is a new operator of this tile
    const uint32_t fl = *(const uint32_t *)(vf + 4 * wd);  // vb and 4*wd are multiples of 4
    int m = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int w = 4 * wd + i;
      if (w >= a && w < e && ((fl >> (8 * i)) & VF_NEW)) m |= 1 << i;
    }
    return m;
  };
  int cnt = 0;
  for (int wd = ww0 + lane; wd < ww1; wd += 32) cnt += __popc(newmask(wd));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) wtot[wid] = cnt;
  {
    const int cc = (threadIdx.x < ncl) ? nptr[c0 + threadIdx.x] : 0;
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t>((int64_t)cc, sm, tot);  // also publishes wtot
    if (threadIdx.x < ncl) {
      nptr[c0 + threadIdx.x] = (int32_t)(base + ex);
      if (c0 + (int)threadIdx.x == C.ncell - 1) nptr[C.ncell] = (int32_t)C.n_off_new;
    }
  }
  int64_t pos = base;
  for (int k = 0; k < wid; ++k) pos += wtot[k];
  for (int s0 = ww0; s0 < ww1; s0 += 32) {
    const int wd = s0 + lane;
    const int m = (wd < ww1) ? newmask(wd) : 0;
    const int c = __popc(m);
    int inc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    int64_t p = pos + inc - c;
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (m & (1 << i)) ntau[p++] = s.vtau[vb + 4 * wd + i];
    pos += __shfl_sync(0xffffffffu, inc, 31);
  }
  // Loops that left their tile: one 32-byte accumulator record per root (and
  // its Zi word), read and cleared; a thread takes one 32-vertex word of the
  // open-root bitmap.  With the Zi words, the next root's reads are issued
  // before the current root is cleared (two roots in flight per thread);
  // without them, the plain loop needs fewer registers and more resident
  // warps hide the latency better.
  u128 w2 = 0, f2 = 0, z2 = 0;
  const int64_t wfirst = (vb + a) >> 5, wlast = (vb + e - 1) >> 5;
  for (int64_t wd = wfirst + threadIdx.x; e > a && wd <= wlast; wd += blockDim.x) {
    uint32_t bits = __ldcg(s.openroot + wd);
    const int64_t v0 = (wd << 5) - vb;
    if (v0 < a) bits &= ~0u << (a - v0);
    if (v0 + 32 > e) bits &= (e - v0 >= 32) ? ~0u : ((1u << (e - v0)) - 1u);
    if (!T) {
      while (bits) {
        const int64_t v = vb + v0 + __ffs(bits) - 1;
        bits &= bits - 1;
        const ulonglong2 x = s.acc2[2 * v], y = s.acc2[2 * v + 1];
        s.acc2[2 * v] = make_ulonglong2(0ull, 0ull);
        s.acc2[2 * v + 1] = make_ulonglong2(0ull, 0ull);
        w2 += sq_abs((long long)x.x);
        f2 += sq_abs((long long)x.y) + sq_abs((long long)y.x);
      }
      continue;
    }
    if (!bits) continue;
    int64_t v = vb + v0 + __ffs(bits) - 1;
    bits &= bits - 1;
    ulonglong2 x = s.acc2[2 * v], y = s.acc2[2 * v + 1];
    unsigned long long zi = s.accz[v];
    for (;;) {
      const bool more = bits != 0;
      int64_t vn = 0;
      ulonglong2 xn, yn;
      unsigned long long zn = 0ull;
      if (more) {
        vn = vb + v0 + __ffs(bits) - 1;
        bits &= bits - 1;
        xn = s.acc2[2 * vn];
        yn = s.acc2[2 * vn + 1];
        zn = s.accz[vn];
      }
      s.acc2[2 * v] = make_ulonglong2(0ull, 0ull);
      s.acc2[2 * v + 1] = make_ulonglong2(0ull, 0ull);
      s.accz[v] = 0ull;
      w2 += sq_abs((long long)x.x);
      f2 += sq_abs((long long)x.y) + sq_abs((long long)y.x);
      z2 += sq_abs((long long)y.y) + sq_abs((long long)zi);
      if (!more) break;
      v = vn;
      x = xn;
      y = yn;
      zi = zn;
    }
  }
  long long none = 0;
  block_sums<T>(none, w2, f2, z2);
  if (threadIdx.x == 0) {
    auto add = [&](unsigned long long *t, u128 v) {
      u128 x = ((u128)t[2 * gt + 1] << 64) | t[2 * gt];
      x += v;
      t[2 * gt] = (unsigned long long)x;
      t[2 * gt + 1] = (unsigned long long)(x >> 64);
    };
    add(s.tile_sw2, w2);
    add(s.tile_sf2, f2);
    add(s.tile_sz2, z2);
  }
}

// ---- spins at tau = 0, vertex-free loops -------------------------------------------
template <int Q>
__global__ void __launch_bounds__(SITE_BLOCK) k_sites(const DevChain *__restrict__ ch,
                                                      const int2 *__restrict__ tab, int64_t blk0,
                                                      Scratch s) {
  __shared__ int64_t sm[33];
  if (halted(s)) return;
  const int64_t gb = blk0 + blockIdx.x;
  const int2 t = tab[gb];
  const DevChain &C = ch[t.x];
  const int i = t.y * SITE_BLOCK + threadIdx.x;
  const int64_t vb = C.vtx_base, wb = vb >> 5;
  int64_t nfree = 0;
  u128 w2 = 0, f2 = 0;
  if (i < C.L) {
    const uint8_t *s0 = C.s0[C.cur];
    uint8_t *s1 = C.s0[C.cur ^ 1];
#pragma unroll
    for (int a = 0; a < Q; ++a) {
      const int u = i * Q + a;
      const int node = s.cut_node[C.sub_off + u];
      int f;
      if (node >= 0) {
        f = get_bit(s.flipbits, wb, __ldcg(s.parent + vb + node));
      } else {
        const int mn = s.free_min[C.sub_off + u];
        f = coin(C, TAG_FREE, (uint32_t)mn);
        if (mn == u) {
          ++nfree;
          const long long len = (long long)s.free_len[C.sub_off + u] * C.qbeta;
          const int x = u / Q;
          w2 += sq_abs(len);
          f2 += sq_abs(mul_q32(len, C.cosq[x])) + sq_abs(mul_q32(len, C.sinq[x]));
        }
      }
      s1[u] = (uint8_t)(s0[u] ^ f);
    }
  }
  const int64_t tf = block_sum<int64_t>(nfree, sm);
  w2 = block_sum_u128(w2);
  f2 = block_sum_u128(f2);
  if (threadIdx.x == 0) {
    s.site_free[gb] = tf;
    s.site_sw2[2 * gb] = (unsigned long long)w2;
    s.site_sw2[2 * gb + 1] = (unsigned long long)(w2 >> 64);
    s.site_sf2[2 * gb] = (unsigned long long)f2;
    s.site_sf2[2 * gb + 1] = (unsigned long long)(f2 >> 64);
  }
}

// ---- per-chain record -----------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_final(DevChain *__restrict__ ch, Scratch s) {
  __shared__ int64_t sm[33];
  if (halted(s)) return;
  DevChain &C = ch[blockIdx.x];
  int64_t roots = 0, nfree = 0;
  u128 w2 = 0, f2 = 0, z2 = 0;
#pragma unroll 4
  for (int i = threadIdx.x; i < C.ntile; i += blockDim.x) {
    const int64_t g = C.tile0 + i;
    roots += s.tile_roots[g];
    w2 += ((u128)s.tile_sw2[2 * g + 1] << 64) | s.tile_sw2[2 * g];
    f2 += ((u128)s.tile_sf2[2 * g + 1] << 64) | s.tile_sf2[2 * g];
    z2 += ((u128)s.tile_sz2[2 * g + 1] << 64) | s.tile_sz2[2 * g];
  }
  for (int i = threadIdx.x; i < C.nsiteblk; i += blockDim.x) {
    const int64_t g = C.site0 + i;
    nfree += s.site_free[g];
    w2 += ((u128)s.site_sw2[2 * g + 1] << 64) | s.site_sw2[2 * g];
    f2 += ((u128)s.site_sf2[2 * g + 1] << 64) | s.site_sf2[2 * g];
  }
  roots = block_sum<int64_t>(roots, sm);
  nfree = block_sum<int64_t>(nfree, sm);
  w2 = block_sum_u128(w2);
  f2 = block_sum_u128(f2);
  z2 = block_sum_u128(z2);  // vertex-free loops are whole periods: no temporal term
  if (threadIdx.x != 0) return;
  lcqmc_record r;
  r.n = C.n;
  r.n_off_old = C.op_ptr[C.cur][C.ncell];
  r.n_off_new = C.n_off_new;
  r.n_free = nfree;
  r.n_clusters = roots + nfree;
  r.n_seg = 2 * C.n + nfree;
  r.F = C.F;
  r.pad = 0;
  r.sw2_lo = (unsigned long long)w2;
  r.sw2_hi = (unsigned long long)(w2 >> 64);
  r.sf2_lo = (unsigned long long)f2;
  r.sf2_hi = (unsigned long long)(f2 >> 64);
  r.sz2_lo = (unsigned long long)z2;
  r.sz2_hi = (unsigned long long)(z2 >> 64);
  const double two64 = 18446744073709551616.0;
  const double dsw = __dadd_rn(__dmul_rn((double)r.sw2_hi, two64), (double)r.sw2_lo);
  const double dsf = __dadd_rn(__dmul_rn((double)r.sf2_hi, two64), (double)r.sf2_lo);
  const double bl = __dmul_rn(__dmul_rn(4.0, C.beta), (double)C.L);
  r.energy = __dsub_rn(__dmul_rn(__dmul_rn((double)(C.Q * C.Q), C.J), 0.25),
                       __ddiv_rn((double)C.n, __dmul_rn(C.beta, (double)C.L)));
  r.chi_s = __ddiv_rn(ldexp(dsw, -2 * C.F), bl);
  r.chi_q = __ddiv_rn(ldexp(dsf, -2 * C.F), bl);
  // |int e^{i w1 t} dt|^2 = |Z|^2 2^-60 / w1^2 with w1 = 2 pi / beta:
  // chi_w = sz2 2^-60 beta / (16 pi^2 L)
  const double kPi = 3.14159265358979323846;
  const double dsz = __dadd_rn(__dmul_rn((double)r.sz2_hi, two64), (double)r.sz2_lo);
  r.chi_w = __ddiv_rn(__dmul_rn(ldexp(dsz, -60), C.beta),
                      __dmul_rn(__dmul_rn(__dmul_rn(16.0, kPi), kPi), (double)C.L));
  C.ring[C.n_rec % C.ring_cap] = r;
  C.n_rec += 1;
  const double v[NOBS] = {r.energy,
                          r.chi_s,
                          r.chi_q,
                          (double)r.n,
                          (double)r.n_off_new,
                          (double)r.n_seg,
                          (double)r.n_clusters,
                          (double)(r.n_seg + 2 * r.n),
                          r.chi_w};
  for (int k = 0; k < NOBS; ++k) {
    C.sum[k] += v[k];
    C.sumsq[k] += v[k] * v[k];
  }
  C.n_updates += 1;
  C.cur ^= 1;
  C.sweep += 1;
}

// ---- host-side launchers ----------------------------------------------------------------
void set_full_table(const uint64_t *T, cudaStream_t st) {
  cudaMemcpyToSymbolAsync(c_T_full, T, sizeof(uint64_t) * KMAX, 0, cudaMemcpyHostToDevice, st);
}

static inline dim3 g1(int64_t n) { return dim3((unsigned)n); }

// One launch per Q group (Q = 2S = 1 .. QMAX); the tile-wide kernels that do
// not depend on Q run over the tiles of every group at once.
#define FOR_EACH_Q(M) M(1) M(2) M(3) M(4)
static_assert(QMAX == 4, "FOR_EACH_Q lists every Q");

static int64_t all_tiles(const Launch &L) {
  int64_t n = 0;
  for (int q = 0; q < QMAX; ++q) n += L.ntile[q];
  return n;
}

void launch_bond_parity(const Launch &L, cudaStream_t st) {
  for (int q = 0; q < QMAX; ++q)
    if (L.nbondblk[q])
      k_bond_parity<<<g1(L.nbondblk[q]), BOND_BLOCK, 0, st>>>(L.ch, L.bond_tab, L.bond0[q], L.s);
}

void launch_clear(const Launch &L, int64_t ntile, int64_t nw, cudaStream_t st) {
  constexpr int T = 256;
  const int64_t n = std::max<int64_t>(std::max(ntile, nw), QMAX);
  const int64_t blocks = std::min<int64_t>((n + T - 1) / T, 152 * 8);
  k_clear<<<g1(blocks), T, 0, st>>>(L.s, ntile, nw);
}

void launch_insert(const Launch &L, cudaStream_t st) {
#define INSERT_Q(Q)                                                                                   \
  if (L.ntile[Q - 1])                                                                                 \
    k_insert<Q><<<g1(L.ntile[Q - 1]), INS_THREADS, Q == 1 ? 0 : sizeof(InsSmem<Q>), st>>>(L.ch,          \
                                                                                          L.tile_tab,    \
                                                                                          L.tile0[Q - 1], \
                                                                                          Q - 1, L.s);
  FOR_EACH_Q(INSERT_Q)
#undef INSERT_Q
}

void launch_scan_ops(const Launch &L, cudaStream_t st) {
  k_scan_ops<<<L.nchains, 1024, 0, st>>>(L.ch, L.s);
}

void launch_cut(const Launch &L, cudaStream_t st) {
#define CUT_Q(Q) \
  if (L.nsiteblk[Q - 1]) k_cut<Q><<<g1(L.nsiteblk[Q - 1]), SITE_BLOCK, 0, st>>>(L.ch, L.site_tab, L.site0[Q - 1], L.s);
  FOR_EACH_Q(CUT_Q)
#undef CUT_Q
}

void launch_link(const Launch &L, cudaStream_t st) {
#define LINK_Q(Q)     \
  if (L.ntile[Q - 1]) \
    k_link<Q><<<g1(L.ntile[Q - 1]), L.link_threads, 0, st>>>(L.ch, L.tile_tab, L.tile0[Q - 1], L.s);
  FOR_EACH_Q(LINK_Q)
#undef LINK_Q
  const int64_t n = all_tiles(L);
  const int wpb = L.link_x_warps;
  if (n) k_link_x<<<g1((n + wpb - 1) / wpb), 32 * wpb, 0, st>>>(L.ch, L.tile_tab, n, L.s);
}

void launch_compress(const Launch &L, cudaStream_t st) {
  const int64_t n = all_tiles(L);
  if (n) k_compress<<<g1(n), L.compress_threads, 0, st>>>(L.ch, L.tile_tab, 0, L.s);
}

void launch_check_forest(const Launch &L, cudaStream_t st) {
  const int64_t n = all_tiles(L);
  if (n) k_check_forest<<<g1(n), TILE, 0, st>>>(L.ch, L.tile_tab, L.s);
}

// Per-vertex staging of the loop-properties kernel: ticks and phase factors.
constexpr size_t EST_DYN_SMEM = EST_STAGE * (sizeof(long long) + sizeof(int2));

// Device tables and kernel attributes, set once per process and device: the
// phase factor table (cos and sin of 2 pi k / 2^16 rounded to 30 fractional
// bits) and the loop-properties kernel's shared memory size.
int init_kernel_attributes() {
  static std::mutex mu;
  static bool done[256];
  static int2 tab[(1 << PHASE_BITS) + 1];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return -1;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return 0;
  for (int k = 0; k <= (1 << PHASE_BITS); ++k) {
    const double ang = (2.0 * M_PI * (double)k) / (double)(1 << PHASE_BITS);
    tab[k] = make_int2((int)std::llrint(std::ldexp(std::cos(ang), 30)),
                       (int)std::llrint(std::ldexp(std::sin(ang), 30)));
  }
  if (cudaMemcpyToSymbol(g_phase_tab, tab, sizeof(tab)) != cudaSuccess) return -1;
#define EST_ATTR_Q(Q)                                                                 \
  if (cudaFuncSetAttribute(k_est<Q, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                           (int)EST_DYN_SMEM) != cudaSuccess)                           \
    return -1;
  FOR_EACH_Q(EST_ATTR_Q)
#undef EST_ATTR_Q
  if (cudaFuncSetAttribute(k_insert<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(InsSmem<2>)) != cudaSuccess ||
      cudaFuncSetAttribute(k_insert<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(InsSmem<3>)) != cudaSuccess ||
      cudaFuncSetAttribute(k_insert<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)sizeof(InsSmem<4>)) != cudaSuccess)
    return -1;
  done[dev] = true;
  return 0;
}

void launch_est(const Launch &L, cudaStream_t st) {
  // without the temporal moment only the ticks are staged
  const size_t dyn = L.temporal ? EST_DYN_SMEM : EST_STAGE * sizeof(long long);
#define EST_Q(Q)                                                                                       \
  if (L.ntile[Q - 1]) {                                                                                \
    if (L.temporal)                                                                                    \
      k_est<Q, true><<<g1(L.ntile[Q - 1]), TPB_EST, dyn, st>>>(L.ch, L.tile_tab, L.tile0[Q - 1], L.s);  \
    else                                                                                               \
      k_est<Q, false><<<g1(L.ntile[Q - 1]), TPB_EST, dyn, st>>>(L.ch, L.tile_tab, L.tile0[Q - 1], L.s); \
  }
  FOR_EACH_Q(EST_Q)
#undef EST_Q
}

void launch_compact(const Launch &L, cudaStream_t st) {
  const int64_t n = all_tiles(L);
  if (n) {
    if (L.temporal)
      k_compact<true><<<g1(n), TPB, 0, st>>>(L.ch, L.tile_tab, 0, L.s);
    else
      k_compact<false><<<g1(n), TPB, 0, st>>>(L.ch, L.tile_tab, 0, L.s);
  }
}

void launch_sites(const Launch &L, cudaStream_t st) {
#define SITES_Q(Q) \
  if (L.nsiteblk[Q - 1]) k_sites<Q><<<g1(L.nsiteblk[Q - 1]), SITE_BLOCK, 0, st>>>(L.ch, L.site_tab, L.site0[Q - 1], L.s);
  FOR_EACH_Q(SITES_Q)
#undef SITES_Q
}

void launch_final(const Launch &L, cudaStream_t st) {
  k_final<<<L.nchains, 1024, 0, st>>>(L.ch, L.s);
}

}  // namespace lcq
