// Swendsen-Wang update of the two-dimensional Ising model: the benchmark on
// which the paper measures its union-find (Sec. 4.1).  Kernels, a small
// engine and the lcqmc_sw_* entry points of include/lcqmc.h.
//
// One update (L x L periodic lattice, site i = y L + x, spin s in {0, 1}):
//   bonds R(i) = (i, right) and D(i) = (i, below); the draws of site i are
//   Philox(ctr = (TAG_SWBOND << 24, i, 0, sweep), key = seed), word 0 for
//   R(i), word 1 for D(i); a bond is active iff its spins are equal and its
//   draw is below T = round(2^32 (1 - e^{-2K}));
//   clusters of active bonds, each named by its smallest site index r;
//   every cluster flips with the coin bit (r mod 128) of
//   Philox(ctr = (TAG_SWFLIP << 24, r / 128, 0, sweep)).
//
// GPU layout: 64 x 32 site tiles, one 256-thread block each.
//   k_sw_local  bond draws, union-find of the tile's bonds in shared memory
//               (min-root hooking, one CAS), flattened; par[i] = the tile-local
//               root (its smallest site); tile-boundary bonds kept as bit masks
//   k_sw_merge  boundary bonds united in the global forest (same min-root rule,
//               path halving), one warp per tile: the paper's two-step
//               local/global union-find (Sec. 3.2) inside one GPU
//   k_sw_flip   root of every local root (path halving), one coin per local
//               root, spins flipped; sizes of clusters closed in the tile
//               squared here, sizes of open ones added at their global root
//   k_sw_sizes  open clusters' sizes squared, cleared for the next update
//   k_sw_final  the update's record and running sums
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dev.cuh"
#include "engine.h"
#include "uf.cuh"

namespace lcq {
namespace {

constexpr int SW_TX = 64, SW_TY = 32, SW_TS = SW_TX * SW_TY;  // tile of 64 x 32 sites
constexpr int SW_TPB = 256;
constexpr int SW_PER = SW_TS / SW_TPB;  // sites per thread
constexpr int SW_WORDS = SW_TS / 32;    // bitmap words per tile
constexpr int SW_SIZE_BLOCKS = 1216;    // blocks of the open-cluster pass: 8 per SM
// An open cluster's root is the smallest site of a tile component that holds
// a site on the tile's border: at most 2 (64 + 32) of them per tile.
constexpr int SW_OPEN_PER_TILE = 2 * (SW_TX + SW_TY);
constexpr int SW_RING = 4096;
constexpr uint32_t TAG_SWBOND = 5u, TAG_SWFLIP = 6u;
constexpr int64_t SW_MAX_SITES = 2147483647;  // site ids are int32

struct SwDev {
  int32_t L, ntx, nty, ntile;
  int64_t N;
  uint64_t T;  // a bond is active iff its draw is below T
  uint64_t seed;
  uint32_t sweep, ring_cap;
  int64_t n_updates;
  double sum[LCQMC_SW_NOBS], sumsq[LCQMC_SW_NOBS];
};

struct SwScratch {
  SwDev *dev;
  int *status;
  uint8_t *spin;                // N
  int32_t *par;                 // N: local root (non-roots), global forest (local roots)
  uint32_t *lroot, *openb;      // per tile, SW_WORDS words: local roots; roots of open components
  uint32_t *edge_r;             // per tile: right-edge bond of row j active (bit j)
  unsigned long long *edge_d;   // per tile: bottom-edge bond of column j active (bit j)
  int32_t *csize;               // N: size of an open cluster at its root; 0 between updates
  int32_t *olist;               // roots of open clusters (at most SW_OPEN_PER_TILE per tile)
  int *ocount;                  // their number; 0 between updates
  long long *tile_part;         // per tile: n_eq, n_act, closed clusters, mag, largest closed
  unsigned long long *tile_c2;  // per tile: sum of the closed clusters' size^2
  long long *size_part;         // per size block: open clusters, largest open
  unsigned long long *size_c2;  // per size block: sum of the open clusters' size^2
  lcqmc_sw_record *ring;
  int32_t *roots;               // lcqmc_sw_get_roots output (N), allocated on demand
};

__device__ __forceinline__ void sw_tile(const SwDev &D, int t, int &x0, int &y0, int &w, int &h) {
  const int ty = t / D.ntx, tx = t - ty * D.ntx;
  x0 = tx * SW_TX;
  y0 = ty * SW_TY;
  w = min(SW_TX, D.L - x0);
  h = min(SW_TY, D.L - y0);
}

// Shared-memory union-find of one tile (local ids, lp[x] <= x, one CAS on the
// larger root).  Walks are bounded by the tile size.
__device__ __forceinline__ int sw_find(volatile int *lp, int x, int *status) {
  for (int it = 0; it <= SW_TS; ++it) {
    const int p = lp[x];
    if (p == x) return x;
    const int g = lp[p];
    if (g != p) lp[x] = g;  // path halving
    x = g;
  }
  atomicOr(status, ST_TIMEOUT);
  return x;
}

__device__ __forceinline__ void sw_union(int *lp, int a, int b, int *status) {
  for (int it = 0; it <= SW_TS; ++it) {
    a = sw_find(lp, a, status);
    b = sw_find(lp, b, status);
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

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, (long long)__shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sums of NS int64 values, the max of one more, and one uint64 sum;
// valid in thread 0.  One barrier pair per call.
template <int NS>
__device__ void block_reduce(long long (&v)[NS], long long &mx, unsigned long long &u) {
  __shared__ long long ps[NS][32], pm[32];
  __shared__ unsigned long long pu[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k) v[k] = warp_sum_ll(v[k]);
  mx = warp_max_ll(mx);
  u = warp_sum_ull(u);
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) ps[k][wid] = v[k];
    pm[wid] = mx;
    pu[wid] = u;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) v[k] = warp_sum_ll(lane < nw ? ps[k][lane] : 0);
    mx = warp_max_ll(lane < nw ? pm[lane] : 0);
    u = warp_sum_ull(lane < nw ? pu[lane] : 0ull);
  }
  __syncthreads();
}

// ---- bonds and tile union-find --------------------------------------------------
// Bond bits are kept per tile in shared memory, one ballot per warp and step.
// Inside a row the active right bonds form runs of consecutive sites; a site's
// run starts at the highest "run start" bit at or below it (bit arithmetic on
// the row's 64-bit mask), which seeds the forest.  Only the vertical bonds
// then need unions, and a vertical bond whose left neighbour is also active,
// with both right bonds between them active, joins runs already joined.
__global__ void __launch_bounds__(SW_TPB) k_sw_local(SwScratch s) {
  __shared__ uint8_t sp[SW_TY + 2][SW_TX + 2];  // spins with a one-site periodic halo
  __shared__ int lp[SW_TS];
  __shared__ uint32_t bR[SW_WORDS], bD[SW_WORDS], bO[SW_WORDS];  // inner right / down bonds, open sites
  __shared__ uint32_t ob[SW_WORDS];                              // local roots of open components
  __shared__ uint32_t er_s;
  __shared__ unsigned long long ed_s;
  if (__ldcg(s.status)) return;
  const SwDev &D = *s.dev;
  const int t = blockIdx.x, L = D.L;
  int x0, y0, w, h;
  sw_tile(D, t, x0, y0, w, h);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int r = wid; r < h + 2; r += SW_TPB / 32) {  // a warp per row, no division
    int gy = y0 - 1 + r;
    gy += (gy < 0) ? L : 0;
    gy -= (gy >= L) ? L : 0;
    const uint8_t *row = s.spin + (int64_t)gy * L;
    for (int c = lane; c < w + 2; c += 32) {
      int gx = x0 - 1 + c;
      gx += (gx < 0) ? L : 0;
      gx -= (gx >= L) ? L : 0;
      sp[r][c] = row[gx];
    }
  }
  if (threadIdx.x < SW_WORDS) ob[threadIdx.x] = 0u;
  if (threadIdx.x == 0) {
    er_s = 0u;
    ed_s = 0ull;
  }
  __syncthreads();
  const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32), sweep = D.sweep;
  const uint64_t T = D.T;
  long long cnt[2] = {0, 0};  // equal bonds, active bonds
#pragma unroll 2
  for (int k = 0; k < SW_PER; ++k) {
    const int l = threadIdx.x + k * SW_TPB, lx = l & (SW_TX - 1), ly = l / SW_TX;
    bool ar = false, ad = false;
    if (lx < w && ly < h) {
      const uint32_t g = (uint32_t)((int64_t)(y0 + ly) * L + x0 + lx);
      const U4 o = philox(TAG_SWBOND << 24, g, 0u, sweep, k0, k1);
      const uint8_t sc = sp[ly + 1][lx + 1];
      const bool eqr = sc == sp[ly + 1][lx + 2], eqd = sc == sp[ly + 2][lx + 1];
      ar = eqr && (uint64_t)o.x < T;
      ad = eqd && (uint64_t)o.y < T;
      cnt[0] += (int)eqr + (int)eqd;
      cnt[1] += (int)ar + (int)ad;
    }
    const bool edge_r = ar && lx + 1 == w, edge_d = ad && ly + 1 == h;
    const uint32_t mr = __ballot_sync(0xffffffffu, ar && !edge_r);
    const uint32_t md = __ballot_sync(0xffffffffu, ad && !edge_d);
    const uint32_t mo = __ballot_sync(0xffffffffu, edge_r || edge_d);
    if (lane == 0) {
      bR[k * (SW_TPB / 32) + wid] = mr;
      bD[k * (SW_TPB / 32) + wid] = md;
      bO[k * (SW_TPB / 32) + wid] = mo;
    }
    if (edge_r) atomicOr(&er_s, 1u << ly);
    if (edge_d) atomicOr(&ed_s, 1ull << lx);
  }
  __syncthreads();
  // bonds of the neighbouring tiles that end in this one: R of the column to
  // the left (threads 0..h-1), D of the row above (threads 64..64+w-1)
  if (threadIdx.x < h) {
    const int j = threadIdx.x;
    const uint32_t gl = (uint32_t)((int64_t)(y0 + j) * L + (x0 == 0 ? L - 1 : x0 - 1));
    if (sp[j + 1][0] == sp[j + 1][1] && (uint64_t)philox(TAG_SWBOND << 24, gl, 0u, sweep, k0, k1).x < T)
      atomicOr(&bO[(j * SW_TX) >> 5], 1u);
  } else if (threadIdx.x >= 64 && threadIdx.x < 64 + w) {
    const int c = threadIdx.x - 64;
    const uint32_t gu = (uint32_t)((int64_t)(y0 == 0 ? L - 1 : y0 - 1) * L + x0 + c);
    if (sp[0][c + 1] == sp[1][c + 1] && (uint64_t)philox(TAG_SWBOND << 24, gu, 0u, sweep, k0, k1).y < T)
      atomicOr(&bO[c >> 5], 1u << (c & 31));
  }
  // forest seeded with the row runs
  for (int l = threadIdx.x; l < SW_TS; l += SW_TPB) {
    const int lx = l & (SW_TX - 1), ly = l / SW_TX;
    const unsigned long long m = ((unsigned long long)bR[2 * ly + 1] << 32) | bR[2 * ly];
    const unsigned long long starts = ~(m << 1);  // bit x: R(x-1) inactive
    const unsigned long long upto = (lx == SW_TX - 1) ? ~0ull : ((2ull << lx) - 1ull);
    lp[l] = ly * SW_TX + (63 - __clzll(starts & upto));
  }
  __syncthreads();
  // vertical bonds, skipping those implied by the left neighbour's
#pragma unroll 2
  for (int k = 0; k < SW_PER; ++k) {
    const int l = threadIdx.x + k * SW_TPB, lx = l & (SW_TX - 1), ly = l / SW_TX;
    if (ly + 1 >= SW_TY) continue;
    const unsigned long long d = ((unsigned long long)bD[2 * ly + 1] << 32) | bD[2 * ly];
    if (!((d >> lx) & 1ull)) continue;
    if (lx > 0) {
      const unsigned long long r0 = ((unsigned long long)bR[2 * ly + 1] << 32) | bR[2 * ly];
      const unsigned long long r1 = ((unsigned long long)bR[2 * ly + 3] << 32) | bR[2 * ly + 2];
      if ((d & r0 & r1) >> (lx - 1) & 1ull) continue;  // D(x-1), R(x-1) above and below: joined
    }
    sw_union(lp, l, l + SW_TX, s.status);
  }
  __syncthreads();
  // every site's local root (read-only walks: no union is running any more)
#pragma unroll 2
  for (int k = 0; k < SW_PER; ++k) {
    const int l = threadIdx.x + k * SW_TPB, lx = l & (SW_TX - 1), ly = l / SW_TX;
    const bool valid = lx < w && ly < h;
    int r = l;
    if (valid) {
      r = lp[l];
      for (int it = 0; it <= SW_TS && lp[r] != r; ++it) r = lp[r];
      s.par[(int64_t)(y0 + ly) * L + x0 + lx] = (int32_t)((int64_t)(y0 + r / SW_TX) * L + x0 + (r & (SW_TX - 1)));
      if ((bO[l >> 5] >> (l & 31)) & 1u) atomicOr(&ob[r >> 5], 1u << (r & 31));
    }
    const uint32_t m = __ballot_sync(0xffffffffu, valid && r == l);
    if (lane == 0) s.lroot[(int64_t)t * SW_WORDS + k * (SW_TPB / 32) + wid] = m;
  }
  long long mx = 0;
  unsigned long long none = 0;
  block_reduce<2>(cnt, mx, none);  // its barrier also completes the open marks
  if (threadIdx.x < SW_WORDS) s.openb[(int64_t)t * SW_WORDS + threadIdx.x] = ob[threadIdx.x];
  if (threadIdx.x == 0) {
    s.edge_r[t] = er_s;
    s.edge_d[t] = ed_s;
    s.tile_part[5 * (int64_t)t] = cnt[0];
    s.tile_part[5 * (int64_t)t + 1] = cnt[1];
  }
}

// ---- tile-boundary bonds in the global forest ------------------------------------
__global__ void __launch_bounds__(256) k_sw_merge(SwScratch s) {
  if (__ldcg(s.status)) return;
  const SwDev &D = *s.dev;
  const int t = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= D.ntile) return;
  const int L = D.L;
  int x0, y0, w, h;
  sw_tile(D, t, x0, y0, w, h);
  const uint32_t er = s.edge_r[t];
  const unsigned long long ed = s.edge_d[t];
  const int xr = (x0 + w == L) ? 0 : x0 + w, yd = (y0 + h == L) ? 0 : y0 + h;
  for (int j = lane; j < SW_TY + SW_TX; j += 32) {
    int64_t a, b;
    if (j < SW_TY) {
      if (!((er >> j) & 1u)) continue;
      a = (int64_t)(y0 + j) * L + x0 + w - 1;
      b = (int64_t)(y0 + j) * L + xr;
    } else {
      const int c = j - SW_TY;
      if (!((ed >> c) & 1ull)) continue;
      a = (int64_t)(y0 + h - 1) * L + x0 + c;
      b = (int64_t)yd * L + x0 + c;
    }
    // start from the two local roots: only local roots' words change here
    uf_union(s.par, __ldcg(s.par + a), __ldcg(s.par + b), s.status);
  }
}

// ---- roots, coins, flips, cluster sizes ---------------------------------------------
__global__ void __launch_bounds__(SW_TPB, 6) k_sw_flip(SwScratch s) {
  __shared__ int cnt[SW_TS];
  __shared__ uint8_t coin_s[SW_TS];
  if (__ldcg(s.status)) return;
  const SwDev &D = *s.dev;
  const int t = blockIdx.x, L = D.L;
  int x0, y0, w, h;
  sw_tile(D, t, x0, y0, w, h);
  for (int l = threadIdx.x; l < SW_TS; l += SW_TPB) cnt[l] = 0;
  __syncthreads();
  const uint32_t k0 = (uint32_t)D.seed, k1 = (uint32_t)(D.seed >> 32), sweep = D.sweep;
  const uint32_t *lrw = s.lroot + (int64_t)t * SW_WORDS;
  const float invL = 1.0f / (float)L;
  int lr[SW_PER], gr[SW_PER];
  uint32_t isroot = 0u;
#pragma unroll
  for (int k = 0; k < SW_PER; ++k) {
    const int l = threadIdx.x + k * SW_TPB, lx = l & (SW_TX - 1), ly = l / SW_TX;
    lr[k] = -1;
    gr[k] = 0;
    if (lx >= w || ly >= h) continue;
    const int64_t g = (int64_t)(y0 + ly) * L + x0 + lx;
    if ((lrw[l >> 5] >> (l & 31)) & 1u) {
      isroot |= 1u << k;
      lr[k] = l;
      // path halving on the way and the root stored at the start: every
      // entry still points to an ancestor, and only local roots' entries
      // change (non-roots keep pointing at their local root)
      gr[k] = uf_find(s.par, (int)g, s.status);
      if (gr[k] != (int)g) s.par[g] = gr[k];
      coin_s[l] = (uint8_t)coin_from(philox(TAG_SWFLIP << 24, (uint32_t)gr[k] >> 7, 0u, sweep, k0, k1),
                                     (uint32_t)gr[k]);
    } else {
      const int p = __ldcg(s.par + g);  // the site's local root, in this tile
      int py = __float2int_rz((float)p * invL), px = p - py * L;  // quotient within 1, corrected
      if (px < 0) {
        --py;
        px += L;
      } else if (px >= L) {
        ++py;
        px -= L;
      }
      if (py < y0 || py >= y0 + h || px < x0 || px >= x0 + w) {  // cannot happen: merges
        atomicOr(s.status, ST_INTERNAL);                         // write local roots only
        lr[k] = -1;
        continue;
      }
      lr[k] = (py - y0) * SW_TX + (px - x0);
    }
    atomicAdd(&cnt[lr[k]], 1);
  }
  __syncthreads();
  long long v[2] = {0, 0};  // closed clusters, magnetization
  long long mx = 0;
  unsigned long long c2 = 0;
#pragma unroll
  for (int k = 0; k < SW_PER; ++k) {
    if (lr[k] < 0) continue;
    const int l = threadIdx.x + k * SW_TPB, lx = l & (SW_TX - 1), ly = l / SW_TX;
    const int64_t g = (int64_t)(y0 + ly) * L + x0 + lx;
    const uint8_t ns = (uint8_t)(s.spin[g] ^ coin_s[lr[k]]);
    s.spin[g] = ns;
    v[1] += ns ? -1 : 1;
    if ((isroot >> k) & 1u) {
      const int c = cnt[l];
      if ((__ldcg(s.openb + (int64_t)t * SW_WORDS + (l >> 5)) >> (l & 31)) & 1u) {
        atomicAdd(s.csize + gr[k], c);
        if (gr[k] == (int)g) {  // the cluster's root: listed once
          const int i = atomicAdd(s.ocount, 1);
          if (i < SW_OPEN_PER_TILE * D.ntile)
            s.olist[i] = gr[k];
          else
            atomicOr(s.status, ST_INTERNAL);
        }
      } else {
        v[0] += 1;
        c2 += (unsigned long long)c * (unsigned long long)c;
        mx = max(mx, (long long)c);
      }
    }
  }
  block_reduce<2>(v, mx, c2);
  if (threadIdx.x == 0) {
    s.tile_part[5 * (int64_t)t + 2] = v[0];
    s.tile_part[5 * (int64_t)t + 3] = v[1];
    s.tile_part[5 * (int64_t)t + 4] = mx;
    s.tile_c2[t] = c2;
  }
}

// ---- open clusters: sizes squared and cleared -----------------------------------------
__global__ void __launch_bounds__(256) k_sw_sizes(SwScratch s) {
  if (__ldcg(s.status)) return;
  const int n = __ldcg(s.ocount);
  long long v[1] = {0};
  long long mx = 0;
  unsigned long long c2 = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int r = __ldcg(s.olist + i);
    const long long c = __ldcg(s.csize + r);
    s.csize[r] = 0;
    v[0] += 1;
    c2 += (unsigned long long)c * (unsigned long long)c;
    mx = max(mx, c);
  }
  block_reduce<1>(v, mx, c2);
  if (threadIdx.x == 0) {
    s.size_part[2 * blockIdx.x] = v[0];
    s.size_part[2 * blockIdx.x + 1] = mx;
    s.size_c2[blockIdx.x] = c2;
  }
}

// ---- record --------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_sw_final(SwScratch s, int nsize) {
  if (__ldcg(s.status)) return;
  SwDev &D = *s.dev;
  long long v[4] = {0, 0, 0, 0};  // n_eq, n_act, clusters, magnetization
  long long mx = 0;
  unsigned long long c2 = 0;
  for (int t = threadIdx.x; t < D.ntile; t += blockDim.x) {
    const long long *p = s.tile_part + 5 * (int64_t)t;
    v[0] += p[0];
    v[1] += p[1];
    v[2] += p[2];
    v[3] += p[3];
    mx = max(mx, p[4]);
    c2 += s.tile_c2[t];
  }
  for (int b = threadIdx.x; b < nsize; b += blockDim.x) {
    v[2] += s.size_part[2 * b];
    mx = max(mx, s.size_part[2 * b + 1]);
    c2 += s.size_c2[b];
  }
  block_reduce<4>(v, mx, c2);
  if (threadIdx.x == 0) {
    const int64_t N = D.N;
    lcqmc_sw_record r;
    r.sweep = D.sweep;
    r.n_eq = v[0];
    r.n_act = v[1];
    r.n_clusters = v[2];
    r.max_cluster = mx;
    r.sum_c2 = c2;
    r.mag = v[3];
    r.energy = (double)(2 * N - 2 * v[0]) / (double)N;  // -(1/N) sum_bonds sigma sigma
    r.chi = (double)c2 / (double)N;                      // sum_c |c|^2 / N
    s.ring[D.n_updates % D.ring_cap] = r;
    const double m = (double)v[3];
    const double x[LCQMC_SW_NOBS] = {r.energy, r.chi, m * m / (double)N, fabs(m) / (double)N};
    for (int k = 0; k < LCQMC_SW_NOBS; ++k) {
      D.sum[k] += x[k];
      D.sumsq[k] += x[k] * x[k];
    }
    D.n_updates += 1;
    D.sweep += 1u;
    *s.ocount = 0;
  }
}

__global__ void k_sw_roots(SwScratch s) {
  if (__ldcg(s.status)) return;
  const SwDev &D = *s.dev;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < D.N; g += (int64_t)gridDim.x * blockDim.x)
    s.roots[g] = uf_root(s.par, (int)g, s.status);
}

#define SWCK(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " #call); \
      return LCQMC_E_CUDA;                                                           \
    }                                                                                \
  } while (0)

uint64_t sw_threshold(double K) {
  const double x = std::floor(std::ldexp(-std::expm1(-2.0 * K), 32) + 0.5);
  if (x <= 0.0) return 0;
  if (x >= 4294967296.0) return (uint64_t)1 << 32;
  return (uint64_t)x;
}

}  // namespace

class SwEngine {
 public:
  ~SwEngine() { release(); }

  int init(int64_t L, double K, uint64_t seed, void *stream) {
    if (L < 2 || L > 46340 || L * L > SW_MAX_SITES) {
      set_error("L must be >= 2 with L^2 < 2^31");
      return LCQMC_E_INVAL;
    }
    if (!(K >= 0.0) || !std::isfinite(K)) {
      set_error("K must be finite and >= 0");
      return LCQMC_E_INVAL;
    }
    if (stream) {
      st_ = (cudaStream_t)stream;
    } else {
      SWCK(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
      own_stream_ = true;
    }
    h_ = SwDev{};
    h_.L = (int32_t)L;
    h_.N = L * L;
    h_.ntx = (int32_t)((L + SW_TX - 1) / SW_TX);
    h_.nty = (int32_t)((L + SW_TY - 1) / SW_TY);
    h_.ntile = h_.ntx * h_.nty;
    h_.T = sw_threshold(K);
    h_.seed = seed;
    h_.ring_cap = SW_RING;
    const int64_t N = h_.N, nt = h_.ntile;
    int rc = 0;
    rc |= dalloc((void **)&s_.dev, sizeof(SwDev));
    rc |= dalloc((void **)&s_.status, sizeof(int));
    rc |= dalloc((void **)&s_.spin, (size_t)N);
    rc |= dalloc((void **)&s_.par, 4 * (size_t)N);
    rc |= dalloc((void **)&s_.lroot, 4 * (size_t)nt * SW_WORDS);
    rc |= dalloc((void **)&s_.openb, 4 * (size_t)nt * SW_WORDS);
    rc |= dalloc((void **)&s_.edge_r, 4 * (size_t)nt);
    rc |= dalloc((void **)&s_.edge_d, 8 * (size_t)nt);
    rc |= dalloc((void **)&s_.csize, 4 * (size_t)N);
    rc |= dalloc((void **)&s_.olist, 4 * (size_t)nt * SW_OPEN_PER_TILE);
    rc |= dalloc((void **)&s_.ocount, sizeof(int));
    rc |= dalloc((void **)&s_.tile_part, 5 * 8 * (size_t)nt);
    rc |= dalloc((void **)&s_.tile_c2, 8 * (size_t)nt);
    rc |= dalloc((void **)&s_.size_part, 2 * 8 * (size_t)SW_SIZE_BLOCKS);
    rc |= dalloc((void **)&s_.size_c2, 8 * (size_t)SW_SIZE_BLOCKS);
    rc |= dalloc((void **)&s_.ring, sizeof(lcqmc_sw_record) * SW_RING);
    if (rc) return LCQMC_E_NOMEM;
    SWCK(cudaMemsetAsync(s_.status, 0, sizeof(int), st_));
    SWCK(cudaMemsetAsync(s_.spin, 0, (size_t)N, st_));  // ordered start: every sigma = +1
    SWCK(cudaMemsetAsync(s_.csize, 0, 4 * (size_t)N, st_));
    SWCK(cudaMemsetAsync(s_.ocount, 0, sizeof(int), st_));
    SWCK(cudaMemcpyAsync(s_.dev, &h_, sizeof(SwDev), cudaMemcpyHostToDevice, st_));
    for (int i = 0; i <= 4; ++i) SWCK(cudaEventCreate(&ev_[i]));
    SWCK(cudaStreamSynchronize(st_));
    return LCQMC_OK;
  }

  int update(int64_t n) {
    if (n < 0) {
      set_error("n must be >= 0");
      return LCQMC_E_INVAL;
    }
    nvtxRangePushA("lcqmc_sw_update");  // profiler range (no-op without a tool)
    const int rc = update_n(n);
    nvtxRangePop();
    return rc;
  }

  int update_n(int64_t n) {
    for (int64_t i = 0; i < n; ++i) {
      if (timing_) {
        int rc = enqueue(true);
        if (rc) return rc;
      } else {
        if (!gexec_) {
          cudaGraph_t g;
          SWCK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
          int rc = enqueue(false);
          cudaGraph_t gg = nullptr;
          cudaError_t e = cudaStreamEndCapture(st_, &gg);
          if (rc) return rc;
          SWCK(e);
          g = gg;
          e = cudaGraphInstantiate(&gexec_, g, 0);
          cudaGraphDestroy(g);
          SWCK(e);
        }
        SWCK(cudaGraphLaunch(gexec_, st_));
      }
      ++enq_;
    }
    return LCQMC_OK;
  }

  int sync() {
    SWCK(cudaStreamSynchronize(st_));
    int st = 0;
    SWCK(cudaMemcpy(&st, s_.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st) {
      set_error("a bounded union-find walk ran out (status " + std::to_string(st) + ")");
      return LCQMC_E_DEVICE_TIMEOUT;
    }
    return LCQMC_OK;
  }

  int records(lcqmc_sw_record *out, int64_t max_n, int64_t *n_out) {
    if (!n_out || (max_n > 0 && !out)) {
      set_error("null output");
      return LCQMC_E_INVAL;
    }
    int rc = sync();
    if (rc) return rc;
    if (enq_ - read_ > SW_RING) read_ = enq_ - SW_RING;  // older records were overwritten
    const int64_t n = std::min<int64_t>(max_n, enq_ - read_);
    for (int64_t k = 0; k < n;) {
      const int64_t pos = (read_ + k) % SW_RING;
      const int64_t run = std::min<int64_t>(n - k, SW_RING - pos);
      SWCK(cudaMemcpy(out + k, s_.ring + pos, sizeof(lcqmc_sw_record) * run, cudaMemcpyDeviceToHost));
      k += run;
    }
    read_ += n;
    *n_out = n;
    return LCQMC_OK;
  }

  int measure(lcqmc_sw_obs *out) {
    if (!out) {
      set_error("null output");
      return LCQMC_E_INVAL;
    }
    int rc = sync();
    if (rc) return rc;
    SwDev d;
    SWCK(cudaMemcpy(&d, s_.dev, sizeof(SwDev), cudaMemcpyDeviceToHost));
    std::memset(out, 0, sizeof(*out));
    out->n_updates = d.n_updates;
    for (int k = 0; k < LCQMC_SW_NOBS; ++k) {
      out->sum[k] = d.sum[k];
      out->sumsq[k] = d.sumsq[k];
    }
    return LCQMC_OK;
  }

  int set_spins(const uint8_t *spins, uint32_t sweep) {
    if (!spins) {
      set_error("null spins");
      return LCQMC_E_INVAL;
    }
    for (int64_t i = 0; i < h_.N; ++i)
      if (spins[i] > 1) {
        set_error("spins must be 0 or 1");
        return LCQMC_E_STATE;
      }
    int rc = sync();
    if (rc) return rc;
    SWCK(cudaMemcpy(s_.spin, spins, (size_t)h_.N, cudaMemcpyHostToDevice));
    SWCK(cudaMemcpy((char *)s_.dev + offsetof(SwDev, sweep), &sweep, sizeof(uint32_t),
                    cudaMemcpyHostToDevice));
    return LCQMC_OK;
  }

  int get_spins(uint8_t *spins) {
    if (!spins) {
      set_error("null spins");
      return LCQMC_E_INVAL;
    }
    int rc = sync();
    if (rc) return rc;
    SWCK(cudaMemcpy(spins, s_.spin, (size_t)h_.N, cudaMemcpyDeviceToHost));
    return LCQMC_OK;
  }

  int get_roots(int32_t *roots) {
    if (!roots) {
      set_error("null roots");
      return LCQMC_E_INVAL;
    }
    if (enq_ == 0) {
      set_error("no update has run yet");
      return LCQMC_E_STATE;
    }
    int rc = sync();
    if (rc) return rc;
    if (!s_.roots && dalloc((void **)&s_.roots, 4 * (size_t)h_.N)) return LCQMC_E_NOMEM;
    const int64_t blocks = std::min<int64_t>((h_.N + 255) / 256, 4096);
    k_sw_roots<<<(int)blocks, 256, 0, st_>>>(s_);
    SWCK(cudaGetLastError());
    rc = sync();
    if (rc) return rc;
    SWCK(cudaMemcpy(roots, s_.roots, 4 * (size_t)h_.N, cudaMemcpyDeviceToHost));
    return LCQMC_OK;
  }

  int set_phase_timing(int on) {
    int rc = sync();
    if (rc) return rc;
    timing_ = on != 0;
    for (double &x : ph_) x = 0.0;
    return LCQMC_OK;
  }

  int phase_times(double *ms, int nphase) {
    if (!ms || nphase < 0) {
      set_error("null output");
      return LCQMC_E_INVAL;
    }
    int rc = sync();
    if (rc) return rc;
    if (pending_) {
      accumulate();
      pending_ = false;
    }
    for (int k = 0; k < nphase; ++k) ms[k] = k < LCQMC_SW_NPHASE ? ph_[k] : 0.0;
    return LCQMC_OK;
  }

  cudaStream_t stream() const { return st_; }
  int64_t sites() const { return h_.N; }

 private:
  int dalloc(void **p, size_t bytes) {
    if (cudaMalloc(p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      (void)cudaGetLastError();
      set_error("device allocation of " + std::to_string(bytes) + " bytes failed");
      *p = nullptr;
      return 1;
    }
    allocs_.push_back(*p);
    return 0;
  }

  void release() {
    if (st_) cudaStreamSynchronize(st_);
    if (gexec_) cudaGraphExecDestroy(gexec_);
    gexec_ = nullptr;
    for (cudaEvent_t &e : ev_)
      if (e) cudaEventDestroy(e);
    for (void *p : allocs_) cudaFree(p);
    allocs_.clear();
    if (own_stream_ && st_) cudaStreamDestroy(st_);
    st_ = nullptr;
  }

  void accumulate() {
    for (int k = 0; k < LCQMC_SW_NPHASE; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev_[k], ev_[k + 1]) == cudaSuccess) ph_[k] += t;
    }
  }

  int enqueue(bool timed) {
    if (timed && pending_) {  // the previous timed update's events are complete once it is
      SWCK(cudaEventSynchronize(ev_[LCQMC_SW_NPHASE]));
      accumulate();
      pending_ = false;
    }
    auto mark = [&](int k) -> cudaError_t { return timed ? cudaEventRecord(ev_[k], st_) : cudaSuccess; };
    const int nt = h_.ntile;
    const int nsize = (int)std::min<int64_t>(SW_SIZE_BLOCKS, ((int64_t)nt * SW_OPEN_PER_TILE + 255) / 256);
    SWCK(mark(0));  // [0] bond draws, tile union-find
    k_sw_local<<<nt, SW_TPB, 0, st_>>>(s_);
    SWCK(mark(1));  // [1] tile-boundary bonds, global union-find
    k_sw_merge<<<(nt * 32 + 255) / 256, 256, 0, st_>>>(s_);
    SWCK(mark(2));  // [2] roots, coins, flips
    k_sw_flip<<<nt, SW_TPB, 0, st_>>>(s_);
    SWCK(mark(3));  // [3] open clusters' sizes, record
    k_sw_sizes<<<nsize, 256, 0, st_>>>(s_);
    k_sw_final<<<1, 1024, 0, st_>>>(s_, nsize);
    SWCK(mark(4));
    SWCK(cudaGetLastError());
    if (timed) pending_ = true;
    return LCQMC_OK;
  }

  SwDev h_{};
  SwScratch s_{};
  cudaStream_t st_ = nullptr;
  bool own_stream_ = false;
  cudaGraphExec_t gexec_ = nullptr;
  cudaEvent_t ev_[LCQMC_SW_NPHASE + 1] = {};
  bool timing_ = false, pending_ = false;
  double ph_[LCQMC_SW_NPHASE] = {};
  std::vector<void *> allocs_;
  int64_t enq_ = 0, read_ = 0;
};

}  // namespace lcq

struct lcqmc_sw {
  lcq::SwEngine eng;
};

#define SWNEED(h)                         \
  do {                                    \
    if (!(h)) {                           \
      lcq::set_error("null handle");      \
      return LCQMC_E_INVAL;               \
    }                                     \
  } while (0)

extern "C" {

int lcqmc_sw_create(int64_t L, double K, uint64_t seed, void *cuda_stream, lcqmc_sw_t *out) {
  if (!out) {
    lcq::set_error("null output handle");
    return LCQMC_E_INVAL;
  }
  *out = nullptr;
  auto *h = new (std::nothrow) lcqmc_sw;
  if (!h) {
    lcq::set_error("host allocation failed");
    return LCQMC_E_NOMEM;
  }
  int rc = h->eng.init(L, K, seed, cuda_stream);
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return LCQMC_OK;
}

int lcqmc_sw_update(lcqmc_sw_t h, int64_t n) {
  SWNEED(h);
  return h->eng.update(n);
}

int lcqmc_sw_sync(lcqmc_sw_t h) {
  SWNEED(h);
  return h->eng.sync();
}

int lcqmc_sw_get_records(lcqmc_sw_t h, lcqmc_sw_record *out, int64_t max_n, int64_t *n_out) {
  SWNEED(h);
  return h->eng.records(out, max_n, n_out);
}

int lcqmc_sw_measure(lcqmc_sw_t h, lcqmc_sw_obs *out) {
  SWNEED(h);
  return h->eng.measure(out);
}

int lcqmc_sw_set_spins(lcqmc_sw_t h, const uint8_t *spins, uint32_t sweep) {
  SWNEED(h);
  return h->eng.set_spins(spins, sweep);
}

int lcqmc_sw_get_spins(lcqmc_sw_t h, uint8_t *spins) {
  SWNEED(h);
  return h->eng.get_spins(spins);
}

int lcqmc_sw_get_roots(lcqmc_sw_t h, int32_t *roots) {
  SWNEED(h);
  return h->eng.get_roots(roots);
}

int lcqmc_sw_set_phase_timing(lcqmc_sw_t h, int enable) {
  SWNEED(h);
  return h->eng.set_phase_timing(enable);
}

int lcqmc_sw_get_phase_times(lcqmc_sw_t h, double *ms, int nphase) {
  SWNEED(h);
  return h->eng.phase_times(ms, nphase);
}

void *lcqmc_sw_stream(lcqmc_sw_t h) { return h ? (void *)h->eng.stream() : nullptr; }

int lcqmc_sw_destroy(lcqmc_sw_t h) {
  delete h;
  return LCQMC_OK;
}

}  // extern "C"
