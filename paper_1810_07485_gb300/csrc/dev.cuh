// Device-side definitions of the loop-cluster update: chain descriptor,
// batch scratch layout, Philox4x32-10, the canonical cell order and small
// bit / 128-bit helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lcqmc.h"

namespace lcq {

constexpr int KMAX = 48;          // Poisson count table length (K <= KMAX-1)
constexpr int QMAX = 4;           // largest 2S: subspins per site (S <= 2)
constexpr int TW = LCQMC_TW;      // windows per time block of the cell order
constexpr int64_t VTX_ID_LIMIT = 0x7ffff000;  // largest vertex count of one chain
constexpr int NOBS = 9;         // running averages per chain (lcqmc_obs.sum)
constexpr int ACC_WORDS = 4;    // 64-bit words of an open loop's record (32 bytes)
constexpr int PHASE_BITS = 16;  // phase factor table: 2^16 points of the period
constexpr int TILE = 128;         // cells per tile (one thread block)
constexpr int SMEM_CAP = 2048;    // vertices a tile can accumulate in shared memory
constexpr int MAX_COIN_GROUPS = 64;
constexpr int SITE_BLOCK = 128;   // original sites per block
constexpr int BOND_BLOCK = 128;   // bonds per block
constexpr double CELL_MEAN = 8.0; // mean candidate graphs per full window (w = 16/J)
constexpr uint32_t TAG_INSERT = 1u, TAG_FLIP = 2u, TAG_FREE = 3u, TAG_PERM = 4u;
constexpr int UF_MAX_ITERS = 1 << 22;  // bound of every union-find retry / find walk

// Status bits (device word; any set bit makes every later kernel of the update
// return at entry, so the persistent state is left untouched).
enum : int {
  ST_VTX_OVERFLOW = 1,
  ST_OP_OVERFLOW = 2,
  ST_TIMEOUT = 4,
  ST_INTERNAL = 8,
  ST_BADSTATE = 16,
  ST_ID_OVERFLOW = 32,
};

// Vertex flag bits.
enum : uint8_t { VF_OLD = 1, VF_WRAP_L = 2, VF_WRAP_R = 4, VF_NEW = 8 };

struct DevChain {
  // geometry
  int32_t L, Q, nsub, nbond, nwin, nblk, ncell, ntile, nsiteblk, F, ring_cap;
  int32_t ins_span;  // candidate slots per insertion group (0: the default)
  // test hooks that force the fallback paths (0: the defaults): vertices a
  // tile may hold in shared memory (1 .. SMEM_CAP), and slots of the per-tile
  // loop table (a power of 2, 1 .. 256)
  int32_t local_cap, loop_slots;
  double beta, J, w;
  uint64_t seed;
  // tables
  const uint64_t *T_last;      // Poisson thresholds of the last window
  const uint64_t *win;         // per window: bits of t0, t_end, t_end - t0
  const long long *cosq, *sinq;  // rint(2^32 cos(2 pi x / L)), rint(2^32 sin(...))
  long long qbeta;             // rint(beta 2^F)
  uint64_t phR;                // floor((2^(64+phS) - 1) / qbeta): period fraction of a tick count
  int32_t phS, pad1;           // floor(log2 qbeta)
  // persistent state, double-buffered (index cur is current)
  uint8_t *s0[2];
  int32_t *op_ptr[2];
  double *op_tau[2];
  int64_t op_cap;
  // offsets into batch scratch
  int64_t cell_off;  // vptr: ncell+1 entries
  int64_t tile0;     // first tile of the chain in the tile arrays
  int64_t site0;     // first site block
  int64_t bpar_off;  // bond parity table: (nblk+1) * nbond bytes
  int64_t sub_off;   // per-subsite arrays: nsub entries
  // dynamic, written by the kernels
  int32_t cur;
  uint32_t sweep;
  int64_t vtx_base;  // first vertex of the chain in the vertex arrays (multiple of 128)
  int64_t vcap;      // vertices reserved for the chain from vtx_base on
  int64_t n;         // graph vertices of the current update
  int64_t n_off_new; // off-diagonal operators after the current update
  // measurements
  lcqmc_record *ring;
  int64_t n_rec;
  int64_t n_updates;
  double sum[NOBS], sumsq[NOBS];
};

struct Scratch {
  int32_t *vptr;
  int64_t *tile_sum, *tile_pref, *tile_sum2, *tile_pref2, *tile_roots;
  unsigned long long *tile_sw2, *tile_sf2, *tile_sz2;  // 2 words (lo, hi) per tile
  int64_t *site_free;
  unsigned long long *site_sw2, *site_sf2;   // 2 words per site block
  uint8_t *bpar;
  int32_t *cut_node, *cut_cell, *free_min;
  int8_t *cut_cross, *free_len;
  double *vtau;
  uint8_t *vflag;
  uint8_t *vcell;  // per vertex: its cell's index inside the tile (0..127)
  int32_t *pl, *pr, *parent;
  union {
    unsigned long long *acc;  // per vertex: W, C, S, Zr (32-byte record), open loops only
    ulonglong2 *acc2;         // the same records as two 16-byte halves
  };
  unsigned long long *accz;  // per vertex: Zi, open loops only, temporal moment on
  uint32_t *openmark, *openroot, *flipbits, *xmark;
  int64_t vcap;
  unsigned long long *tile_state;  // per tile: insertion look-back word (flag << 62 | count)
  unsigned int *tickets;           // per Q group: next tile of the insertion launch
  int *status;
  int uf_limit;   // bound of the global union-find walks and retries (UF_MAX_ITERS)
  int64_t *need;  // [0] vertex capacity needed by the last update
  long long *dbg; // first failed consistency check: code, then 7 details
};

// Records the first failed consistency check (code > 0) and sets ST_INTERNAL.
__device__ __forceinline__ void fail_check(const Scratch &s, int code, long long a, long long b,
                                           long long c, long long d, long long e) {
  if (atomicCAS((unsigned long long *)s.dbg, 0ull, (unsigned long long)code) == 0ull) {
    s.dbg[1] = a;
    s.dbg[2] = b;
    s.dbg[3] = c;
    s.dbg[4] = d;
    s.dbg[5] = e;
  }
  atomicOr(s.status, ST_INTERNAL);
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) -----------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
    uint32_t lo0 = m0 * c0, hi0 = __umulhi(m0, c0);
    uint32_t lo1 = m1 * c2, hi1 = __umulhi(m1, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ int coin_from(const U4 &o, uint32_t idx) {
  uint32_t bit = idx & 127u;
  uint32_t word = (bit < 32) ? o.x : (bit < 64) ? o.y : (bit < 96) ? o.z : o.w;
  return (int)((word >> (bit & 31u)) & 1u);
}

// One fair coin per index, 128 indices per Philox block.
__device__ __forceinline__ int coin(const DevChain &C, uint32_t tag, uint32_t idx) {
  U4 o = philox(tag << 24, idx >> 7, 0u, C.sweep, (uint32_t)C.seed, (uint32_t)(C.seed >> 32));
  return coin_from(o, idx);
}

// Vertices of a tile that its kernels keep in shared memory: a tile with more
// takes the global-memory paths.
__device__ __forceinline__ int local_cap(const DevChain &C) {
  return (C.local_cap > 0 && C.local_cap < SMEM_CAP) ? C.local_cap : SMEM_CAP;
}

// ---- cell order ----------------------------------------------------------
__device__ __forceinline__ int cell_of(const DevChain &C, int b, int j) {
  int blk = j / TW, jj = j - blk * TW;
  int tw = min(TW, C.nwin - blk * TW);
  return blk * C.nbond * TW + b * tw + jj;
}

__device__ __forceinline__ void cell_bj(const DevChain &C, int c, int &b, int &j) {
  int per = C.nbond * TW;
  int blk = c / per;
  int r = c - blk * per;
  int tw = min(TW, C.nwin - blk * TW);
  b = r / tw;
  j = blk * TW + (r - b * tw);
}

// ---- lattice of subspins: bond b = i*Q*Q + a*Q + a2 joins (i,a) and (i+1,a2)
template <int Q>
__device__ __forceinline__ int left_sub(int b) {
  return (b / (Q * Q)) * Q + (b / Q) % Q;
}
template <int Q>
__device__ __forceinline__ int right_sub(int b, int L) {
  int i = b / (Q * Q) + 1;
  if (i == L) i = 0;
  return i * Q + b % Q;
}
// k-th bond touching subsite u: k < Q as its left end, k >= Q as its right end.
template <int Q>
__device__ __forceinline__ int inc_bond(int u, int k, int L) {
  int i = u / Q, a = u - (u / Q) * Q;
  if (k < Q) return i * Q * Q + a * Q + k;
  int im = (i == 0) ? L - 1 : i - 1;
  return im * Q * Q + (k - Q) * Q + a;
}

// ---- bulk copies global -> shared (TMA, no tensor map) ---------------------------
// One thread arms a shared-memory mbarrier with the byte count and starts the
// copy; every thread then waits on the barrier's phase.  Both addresses must
// be 16-byte aligned and the size a multiple of 16.  The wait is bounded: a
// copy that has not landed after STAGE_MAX_POLLS polls sets ST_TIMEOUT.
constexpr int STAGE_MAX_POLLS = 1 << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arms the barrier for `bytes` and starts one copy of `bytes` (thread-local call).
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Waits for phase `parity` of the barrier to complete; false if it did not
// within the bound.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  for (int i = 0; i < STAGE_MAX_POLLS; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// ---- bits ------------------------------------------------------------------
__device__ __forceinline__ int get_bit(const uint32_t *bits, int64_t word0, int32_t i) {
  return (int)((__ldcg(bits + word0 + (i >> 5)) >> (i & 31)) & 1u);
}
__device__ __forceinline__ void set_bit(uint32_t *bits, int64_t word0, int32_t i) {
  atomicOr(bits + word0 + (i >> 5), 1u << (i & 31));
}

typedef unsigned __int128 u128;

__device__ __forceinline__ u128 sq_abs(long long v) {
  unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
  return (u128)a * (u128)a;
}

// ---- times as bit patterns ------------------------------------------------------
// GB300 executes fp64 instructions on a handful of lanes per SM, so the hot
// loops keep imaginary times as the bit patterns of non-negative doubles
// (ordered like the doubles themselves when read as int64).  The only fp64
// instruction left is one fused multiply-add per insertion candidate; the
// conversion of times to integer ticks is done with integer arithmetic,
// exactly as IEEE 754 defines it (round to nearest, ties to even).

constexpr uint64_t M52 = (1ull << 52) - 1;

// Bits of the double u53 * 2^-53 for u53 < 2^53 (exact).
__host__ __device__ __forceinline__ uint64_t unit_bits(uint64_t u53) {
  if (u53 == 0) return 0;
#ifdef __CUDA_ARCH__
  const int s = __clzll((long long)u53) - 11;
#else
  const int s = __builtin_clzll(u53) - 11;
#endif
  // u53 in [2^(52-s), 2^(53-s)): value 1.f * 2^(-1-s)
  return ((uint64_t)(1022 - s) << 52) | ((u53 << s) & M52);
}

// llrint(ldexp(x, F)) for a non-negative double x given as bits (x 2^F < 2^62).
__host__ __device__ __forceinline__ long long q_time(uint64_t x_bits, int F) {
  if (x_bits == 0) return 0;
  const int ex = (int)((x_bits >> 52) & 0x7ff);
  const uint64_t m = (x_bits & M52) | (ex ? (1ull << 52) : 0);
  const int sh = (ex ? ex : 1) - 1075 + F;  // x 2^F = m 2^sh
  if (sh >= 0) return (long long)(m << sh);
  const int r = -sh;
  if (r > 63) return 0;  // m < 2^53 <= 2^(r-1): below one half
  uint64_t q = m >> r;
  const uint64_t rem = m & ((1ull << r) - 1), half = 1ull << (r - 1);
  if (rem > half || (rem == half && (q & 1))) ++q;
  return (long long)q;
}

// exp(i 2 pi q / qbeta) in units of 2^-30 (.x cos, .y sin) for a tick count
// q: the period fraction X = (q R) >> sh modulo 2^64 (R, sh per chain), the
// table at 2^16 points (tab[k] for angle 2 pi k / 2^16, one extra entry at the
// end) and linear interpolation with the 2^-32-scaled correction floored.
__device__ __forceinline__ int2 phase_of(uint64_t q, uint64_t R, int sh, const int2 *tab) {
  const uint64_t lo = q * R, hi = __umul64hi(q, R);
  const uint64_t X = (sh == 0) ? lo : ((lo >> sh) | (hi << (64 - sh)));
  const int k = (int)(X >> (64 - PHASE_BITS));
  const long long t = (long long)((X >> (32 - PHASE_BITS)) & 0xffffffffull);
  const int2 a = tab[k], b = tab[k + 1];
  const long long dc = (long long)(b.x - a.x) * t, ds = (long long)(b.y - a.y) * t;
  return make_int2(a.x + (int)(dc >> 32), a.y + (int)(ds >> 32));  // arithmetic shift: floor
}

// round(v * c / 2^32) with ties upward: floor((v c + 2^31) / 2^32), 128-bit exact.
__host__ __device__ __forceinline__ long long mul_q32(long long v, long long c) {
  const __int128 p = (__int128)v * (__int128)c + ((__int128)1 << 31);
  return (long long)(p >> 32);
}

}  // namespace lcq
