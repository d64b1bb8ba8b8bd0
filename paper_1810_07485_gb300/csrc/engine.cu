// Host engine of the loop-cluster update: per-chain state, batch scratch, the
// per-update launch sequence (captured once as a CUDA graph), capacity growth
// with replay, and state import / export.
#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "engine.h"

#include <nvtx3/nvToolsExt.h>

namespace lcq {

// NVTX range for profilers (no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }
const char *last_error() { return g_err.c_str(); }

#define CK(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      set_error(std::string("CUDA error: ") + cudaGetErrorString(e_) + " at " #call); \
      return LCQMC_E_CUDA;                                                           \
    }                                                                                \
  } while (0)

// ---- method tables (host) ------------------------------------------------------
// Poisson(mu) thresholds T[k] = floor(2^64 P(K <= k)), from the recurrence
// P(0) = e^{-mu}, P(k) = P(k-1) mu / k; saturated at 2^64 - 1.
static void poisson_table(double mu, uint64_t *T) {
  double pk = std::exp(-mu), cdf = 0.0;
  for (int k = 0; k < KMAX; ++k) {
    if (k > 0) pk = pk * mu / (double)k;
    cdf += pk;
    const double x = std::ldexp(cdf, 64);
    T[k] = (x >= 18446744073709551616.0) ? UINT64_MAX : (uint64_t)x;
  }
}

static int fixed_exponent(const ChainSpec &c) {
  const double total = (double)c.Q * (double)c.L * c.beta;
  int e;
  const double m = std::frexp(total, &e);
  const int cl = (m == 0.5) ? e - 1 : e;
  return std::min(62, std::max(0, 60 - cl));
}

int validate_spec(int64_t L, double S, double J, double beta, ChainSpec &out) {
  const double twoS = 2.0 * S;
  if (!(L >= 2) || (L & 1)) {
    set_error("L must be even and >= 2 (odd L frustrates the periodic antiferromagnet)");
    return LCQMC_E_INVAL;
  }
  if (!(twoS == 1.0 || twoS == 2.0 || twoS == 3.0 || twoS == 4.0)) {
    set_error("2S must be 1, 2, 3 or 4");
    return LCQMC_E_INVAL;
  }
  if (!(J > 0.0) || !std::isfinite(J) || !(beta > 0.0) || !std::isfinite(beta)) {
    set_error("J and beta must be positive and finite");
    return LCQMC_E_INVAL;
  }
  out.L = L;
  out.Q = (int)twoS;
  out.J = J;
  out.beta = beta;
  const double w = 16.0 / J;
  const double nw = std::ceil(beta / w);
  const double ncell = nw * (double)L * out.Q * out.Q;
  if (!(ncell < 2147483000.0) || (double)L * out.Q > 1.0e9) {
    set_error("too many cells (bond x time window) for 32-bit indices");
    return LCQMC_E_ID_OVERFLOW;
  }
  return LCQMC_OK;
}

static int64_t vertex_estimate(const ChainSpec &c) {
  const double m = 0.8 * c.Q * c.Q * c.J * c.beta * (double)c.L;
  return (int64_t)(m + 16.0 * std::sqrt(m) + 256.0);
}
static int64_t op_estimate(const ChainSpec &c) {
  const double m = 0.45 * c.Q * c.Q * c.J * c.beta * (double)c.L;
  return (int64_t)(m + 16.0 * std::sqrt(m) + 256.0);
}

struct Geo {
  int64_t nsub, nbond, nwin, nblk, ncell, ntile, nsiteblk, nbondblk;
  double w;
};
static Geo geo_of(const ChainSpec &c) {
  Geo g;
  g.nsub = c.L * c.Q;
  g.nbond = c.L * c.Q * c.Q;
  g.w = 16.0 / c.J;
  g.nwin = std::max<int64_t>(1, (int64_t)std::ceil(c.beta / g.w));
  g.nblk = (g.nwin + TW - 1) / TW;
  g.ncell = g.nbond * g.nwin;
  g.ntile = (g.ncell + TILE - 1) / TILE;
  g.nsiteblk = (c.L + SITE_BLOCK - 1) / SITE_BLOCK;
  g.nbondblk = (g.nbond + BOND_BLOCK - 1) / BOND_BLOCK;
  return g;
}

size_t Engine::estimate_footprint(const std::vector<ChainSpec> &specs, int ring_cap) {
  size_t bytes = 0;
  int64_t vc = 4096;
  for (const auto &c : specs) {
    Geo g = geo_of(c);
    bytes += 2 * (g.nsub + 2 * 4 * (g.ncell + 1) + 8 * op_estimate(c));
    bytes += 8 * KMAX + 16 * c.L + 24 * g.nwin + sizeof(lcqmc_record) * ring_cap;
    bytes += 4 * (g.ncell + 1) + 64 * g.ntile + 48 * g.nsiteblk + (g.nblk + 1) * g.nbond +
             14 * g.nsub + sizeof(DevChain) + 8 * (g.ntile + g.nsiteblk + g.nbondblk);
    vc += (vertex_estimate(c) + 127) / 128 * 128;
  }
  bytes += (size_t)vc * (8 + 2 + 12 + 8 * ACC_WORDS + 8) + 4 * (size_t)(vc / 32 + 1) * 4;
  return bytes;
}

// ---- allocation ------------------------------------------------------------------------
void *Engine::dalloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (has_alloc_) {
    p = alloc_.alloc(bytes, alloc_.ctx);
  } else if (pool_) {
    if (cudaMallocFromPoolAsync(&p, bytes, pool_, st_) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}
void Engine::dfree(void *p) {
  if (!p) return;
  if (has_alloc_)
    alloc_.free(p, alloc_.ctx);
  else if (pool_)
    cudaFreeAsync(p, st_);
  else
    cudaFree(p);
}


#define DALLOC(ptr, type, count)                                                    \
  do {                                                                              \
    ptr = (type *)dalloc(sizeof(type) * (size_t)(count));                           \
    if (!ptr) {                                                                     \
      set_error("device allocation of " + std::to_string(sizeof(type) * (size_t)(count)) + \
                " bytes failed");                                                   \
      return LCQMC_E_NOMEM;                                                         \
    }                                                                               \
  } while (0)

void Engine::free_vertex() {
  dfree(s_.vtau);
  dfree(s_.vflag);
  dfree(s_.vcell);
  dfree(s_.pl);
  dfree(s_.pr);
  dfree(s_.parent);
  dfree(s_.acc);
  dfree(s_.accz);
  dfree(s_.openmark);
  dfree(s_.openroot);
  dfree(s_.flipbits);
  dfree(s_.xmark);
  s_.vtau = nullptr;
  s_.vflag = nullptr;
  s_.vcell = nullptr;
  s_.pl = s_.pr = s_.parent = nullptr;
  s_.acc = nullptr;
  s_.accz = nullptr;
  s_.openmark = s_.openroot = s_.flipbits = s_.xmark = nullptr;
  vertex_bytes_ = 0;
}

int Engine::alloc_vertex(int64_t vcap) {
  free_vertex();
  vcap = (vcap + 127) / 128 * 128;
  DALLOC(s_.vtau, double, vcap);
  DALLOC(s_.vflag, uint8_t, vcap);
  DALLOC(s_.vcell, uint8_t, vcap);
  DALLOC(s_.pl, int32_t, vcap);
  DALLOC(s_.pr, int32_t, vcap);
  DALLOC(s_.parent, int32_t, vcap);
  DALLOC(s_.acc, unsigned long long, ACC_WORDS * vcap);
  DALLOC(s_.accz, unsigned long long, vcap);
  const int64_t nw = vcap / 32 + 1;
  DALLOC(s_.openmark, uint32_t, nw);
  DALLOC(s_.openroot, uint32_t, nw);
  DALLOC(s_.flipbits, uint32_t, nw);
  DALLOC(s_.xmark, uint32_t, nw);
  CK(cudaMemsetAsync(s_.acc, 0, ACC_WORDS * sizeof(unsigned long long) * vcap, st_));
  CK(cudaMemsetAsync(s_.accz, 0, sizeof(unsigned long long) * vcap, st_));
  s_.vcap = vcap;
  vcap_ = vcap;
  vertex_bytes_ = (size_t)vcap * (8 + 2 + 12 + 8 * ACC_WORDS + 8) + 4 * (size_t)nw * 4;
  L_.s = s_;
  drop_graphs();
  return LCQMC_OK;
}

void Engine::destroy_state(ChainState *c) {
  if (!c) return;
  ChainBuf &b = c->buf;
  for (int k = 0; k < 2; ++k) {
    dfree(b.s0[k]);
    dfree(b.op_ptr[k]);
    dfree(b.op_tau[k]);
  }
  dfree(b.T_last);
  dfree(b.cosq);
  dfree(b.sinq);
  dfree(b.win);
  dfree(b.ring);
  b = ChainBuf{};
}

Engine::~Engine() {
  if (st_) cudaStreamSynchronize(st_);
  drop_graphs();
  for (auto e : ev_) cudaEventDestroy(e);
  free_vertex();
  for (auto &c : owned_) destroy_state(c.get());
  dfree(dch_);
  dfree(tile_tab_);
  dfree(site_tab_);
  dfree(bond_tab_);
  dfree(s_.vptr);
  dfree(s_.tile_sum);
  dfree(s_.tile_pref);
  dfree(s_.tile_sum2);
  dfree(s_.tile_pref2);
  dfree(s_.tile_roots);
  dfree(s_.tile_sw2);
  dfree(s_.tile_sf2);
  dfree(s_.tile_sz2);
  dfree(s_.site_free);
  dfree(s_.site_sw2);
  dfree(s_.site_sf2);
  dfree(s_.bpar);
  dfree(s_.cut_node);
  dfree(s_.cut_cell);
  dfree(s_.free_min);
  dfree(s_.cut_cross);
  dfree(s_.free_len);
  dfree(s_.status);
  dfree(s_.tickets);
  dfree(s_.tile_state);
  dfree(s_.need);
  dfree(s_.dbg);
  if (st_) cudaStreamSynchronize(st_);  // stream-ordered frees done
  if (pool_) cudaMemPoolDestroy(pool_);
  if (own_stream_ && st_) cudaStreamDestroy(st_);
}

int Engine::open(void *stream, const lcqmc_allocator *alloc, int ring_cap, bool serving) {
  CK(cudaGetDevice(&device_));
  if (init_kernel_attributes() != 0) {
    set_error("device table initialization failed");
    return LCQMC_E_CUDA;
  }
  // Debug: verify the loop forest after every compression.
  if (const char *e = std::getenv("LCQMC_CHECK_FOREST")) L_.check_forest = std::atoi(e) != 0;
  if (alloc && alloc->alloc && alloc->free) {
    alloc_ = *alloc;
    has_alloc_ = true;
  }
  if (stream) {
    st_ = (cudaStream_t)stream;
  } else {
    CK(cudaStreamCreateWithFlags(&st_, cudaStreamNonBlocking));
    own_stream_ = true;
  }
  if (serving) {
    serving_ = true;
    if (!has_alloc_) {
      cudaMemPoolProps props{};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device_;
      CK(cudaMemPoolCreate(&pool_, &props));
      // keep freed memory in the pool for the next request's state
      uint64_t keep = UINT64_MAX;
      CK(cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &keep));
    }
  }
  ring_cap_ = ring_cap;
  std::vector<uint64_t> T(KMAX);
  poisson_table(CELL_MEAN, T.data());
  set_full_table(T.data(), st_);
  DALLOC(s_.status, int, 1);
  s_.uf_limit = UF_MAX_ITERS;
  // Tests: the most steps a global union-find walk or retry loop of this
  // engine may take (1 .. 2^22; lcqmc_set_wait_limit sets it for a chain).
  if (const char *e = std::getenv("LCQMC_WAIT_LIMIT")) {
    const long long v = std::atoll(e);
    if (v >= 1 && v <= UF_MAX_ITERS) s_.uf_limit = (int)v;
  }
  DALLOC(s_.tickets, unsigned int, QMAX);
  DALLOC(s_.need, int64_t, 4);
  DALLOC(s_.dbg, long long, 8);
  CK(cudaMemsetAsync(s_.status, 0, sizeof(int), st_));
  CK(cudaMemsetAsync(s_.dbg, 0, 8 * sizeof(long long), st_));
  CK(cudaStreamSynchronize(st_));
  return LCQMC_OK;
}

// Persistent state of one chain: Neel start, no operators, sweep 0.
int Engine::create_state(const ChainSpec &spec, ChainState *out) {
  out->spec = spec;
  out->rec_read = 0;
  const Geo g = geo_of(spec);
  DevChain &d = out->dev;
  d = DevChain{};
  d.L = (int32_t)spec.L;
  d.Q = spec.Q;
  d.nsub = (int32_t)g.nsub;
  d.nbond = (int32_t)g.nbond;
  d.nwin = (int32_t)g.nwin;
  d.nblk = (int32_t)g.nblk;
  d.ncell = (int32_t)g.ncell;
  d.ntile = (int32_t)g.ntile;
  d.nsiteblk = (int32_t)g.nsiteblk;
  d.F = fixed_exponent(spec);
  d.ring_cap = ring_cap_;
  d.beta = spec.beta;
  d.J = spec.J;
  d.w = g.w;
  d.seed = spec.seed;
  d.op_cap = op_estimate(spec);
  ChainBuf &b = out->buf;
  for (int k = 0; k < 2; ++k) {
    DALLOC(b.s0[k], uint8_t, d.nsub);
    DALLOC(b.op_ptr[k], int32_t, (int64_t)d.ncell + 1);
    DALLOC(b.op_tau[k], double, d.op_cap + 2);  // +2: bulk copies end on a 16-byte bound
    d.s0[k] = b.s0[k];
    d.op_ptr[k] = b.op_ptr[k];
    d.op_tau[k] = b.op_tau[k];
  }
  std::vector<uint8_t> s0(d.nsub);
  for (int u = 0; u < d.nsub; ++u) s0[u] = (uint8_t)((u / d.Q) & 1);
  CK(cudaMemcpyAsync(b.s0[0], s0.data(), d.nsub, cudaMemcpyHostToDevice, st_));
  CK(cudaMemsetAsync(b.op_ptr[0], 0, sizeof(int32_t) * ((size_t)d.ncell + 1), st_));
  std::vector<uint64_t> T(KMAX);
  const double t0 = (double)(d.nwin - 1) * d.w;
  const double dl = d.beta - t0;
  poisson_table(dl > 0.0 ? d.J * dl * 0.5 : 0.0, T.data());
  DALLOC(b.T_last, uint64_t, KMAX);
  CK(cudaMemcpyAsync(b.T_last, T.data(), 8 * KMAX, cudaMemcpyHostToDevice, st_));
  // 2^32 cos(k x), 2^32 sin(k x), k = 2 pi / L, rounded to integers.
  std::vector<long long> cs(d.L), sn(d.L);
  for (int x = 0; x < d.L; ++x) {
    const double ang = (2.0 * M_PI * (double)x) / (double)d.L;
    cs[x] = std::llrint(std::ldexp(std::cos(ang), 32));
    sn[x] = std::llrint(std::ldexp(std::sin(ang), 32));
  }
  DALLOC(b.cosq, long long, d.L);
  DALLOC(b.sinq, long long, d.L);
  CK(cudaMemcpyAsync(b.cosq, cs.data(), 8 * (size_t)d.L, cudaMemcpyHostToDevice, st_));
  CK(cudaMemcpyAsync(b.sinq, sn.data(), 8 * (size_t)d.L, cudaMemcpyHostToDevice, st_));
  // Window j covers [t0, t_end): t0 = j w, t_end = (j+1) w or beta for the last.
  std::vector<uint64_t> win(3 * (size_t)d.nwin);
  for (int j = 0; j < d.nwin; ++j) {
    const double a = (double)j * d.w;
    const double te = (j == d.nwin - 1) ? d.beta : (double)(j + 1) * d.w;
    const double dd = te - a;
    std::memcpy(&win[3 * (size_t)j], &a, 8);
    std::memcpy(&win[3 * (size_t)j + 1], &te, 8);
    std::memcpy(&win[3 * (size_t)j + 2], &dd, 8);
  }
  DALLOC(b.win, uint64_t, 3 * (size_t)d.nwin);
  CK(cudaMemcpyAsync(b.win, win.data(), 8 * win.size(), cudaMemcpyHostToDevice, st_));
  DALLOC(b.ring, lcqmc_record, ring_cap_);
  d.T_last = b.T_last;
  d.cosq = b.cosq;
  d.sinq = b.sinq;
  d.win = b.win;
  d.ring = b.ring;
  d.qbeta = std::llrint(std::ldexp(d.beta, d.F));
  {
    // period fraction of a tick count: X = (q phR) >> phS, phS = floor(log2 qbeta)
    int k = 63;
    while (k > 0 && !(((uint64_t)d.qbeta >> k) & 1u)) --k;
    d.phS = k;
    d.phR = (uint64_t)((((unsigned __int128)1 << (64 + k)) - 1) / (unsigned __int128)(uint64_t)d.qbeta);
  }
  CK(cudaStreamSynchronize(st_));  // host staging vectors go out of scope
  return LCQMC_OK;
}

size_t Engine::state_bytes(const ChainSpec &c, int ring_cap) {
  const Geo g = geo_of(c);
  return 2 * ((size_t)g.nsub + 4 * ((size_t)g.ncell + 1) + 8 * (size_t)op_estimate(c)) + 8 * KMAX +
         16 * (size_t)c.L + 24 * (size_t)g.nwin + sizeof(lcqmc_record) * (size_t)ring_cap;
}

size_t Engine::scratch_bytes(const ChainSpec &c) {
  const Geo g = geo_of(c);
  const size_t v = (size_t)((vertex_estimate(c) + 127) / 128 * 128);
  return v * 45 + 4 * (size_t)(g.ncell + 1) + 96 * (size_t)g.ntile + 48 * (size_t)g.nsiteblk +
         (size_t)(g.nblk + 1) * g.nbond + 14 * (size_t)g.nsub + sizeof(DevChain);
}

int Engine::grow_array(void **p, int64_t *cap, int64_t need, size_t elem) {
  if (need <= *cap && *p) return LCQMC_OK;
  const int64_t nc = std::max<int64_t>(need, 1);
  void *q = dalloc(elem * (size_t)nc);
  if (!q) {
    set_error("device allocation of scratch failed");
    return LCQMC_E_NOMEM;
  }
  dfree(*p);
  *p = q;
  *cap = nc;
  return LCQMC_OK;
}

// Makes `chains` the resident set: per-chain offsets into the batch scratch,
// block tables (Q=1 chains' blocks before Q=2 chains'), scratch sized to the
// set (grown, never shrunk).  The chains' persistent state is untouched.
int Engine::set_chains(const std::vector<ChainState *> &chains) {
  if (!cs_.empty()) {
    int rc = sync();
    if (rc) return rc;
  }
  cs_ = chains;
  return layout();
}

// Offsets of the resident chains in the batch scratch.  Each chain owns a fixed
// vertex region [vtx_base, vtx_base + vcap) (128-aligned), so the single-pass
// insertion of one chain never waits for another chain's vertex count.
int Engine::layout() {
  const int nc = (int)cs_.size();
  hch.assign(nc, DevChain{});
  std::vector<int2> ttab, stab, btab;
  int64_t cell_off = 0, bpar_off = 0, sub_off = 0, vest = 0;
  for (int q = 0; q < QMAX; ++q) {
    L_.tile0[q] = (int64_t)ttab.size();
    L_.site0[q] = (int64_t)stab.size();
    L_.bond0[q] = (int64_t)btab.size();
    for (int c = 0; c < nc; ++c) {
      if (cs_[c]->spec.Q != q + 1) continue;
      const Geo g = geo_of(cs_[c]->spec);
      DevChain &d = hch[c];
      d = cs_[c]->dev;
      d.cell_off = cell_off;
      d.tile0 = (int64_t)ttab.size();
      d.site0 = (int64_t)stab.size();
      d.bpar_off = bpar_off;
      d.sub_off = sub_off;
      if (cs_[c]->vcap <= 0) cs_[c]->vcap = (vertex_estimate(cs_[c]->spec) + 127) / 128 * 128;
      d.vcap = cs_[c]->vcap;
      // Test hook: a smaller candidate staging group, so that every tile of
      // insertion takes the multi-group path (count, then draw again to write).
      d.ins_span = 0;
      if (const char *e = std::getenv("LCQMC_INSERT_GROUP_SLOTS")) d.ins_span = std::atoi(e);
      // Test hooks: fewer vertices per tile in shared memory (tiles above it
      // take the global-memory paths of linking, union-find, compression and
      // loop sums), and a smaller per-tile loop table (loops that do not fit
      // spill to their global records).
      d.local_cap = 0;
      if (const char *e = std::getenv("LCQMC_LOCAL_CAP")) d.local_cap = std::atoi(e);
      d.loop_slots = 0;
      if (const char *e = std::getenv("LCQMC_LOOP_SLOTS")) d.loop_slots = std::atoi(e);
      cell_off += g.ncell + 1;
      bpar_off += (g.nblk + 1) * g.nbond;
      sub_off += g.nsub;
      for (int64_t t = 0; t < g.ntile; ++t) ttab.push_back(make_int2(c, (int)t));
      for (int64_t t = 0; t < g.nsiteblk; ++t) stab.push_back(make_int2(c, (int)t));
      for (int64_t t = 0; t < g.nbondblk; ++t) btab.push_back(make_int2(c, (int)t));
    }
    L_.ntile[q] = (int64_t)ttab.size() - L_.tile0[q];
    L_.nsiteblk[q] = (int64_t)stab.size() - L_.site0[q];
    L_.nbondblk[q] = (int64_t)btab.size() - L_.bond0[q];
  }
  for (int c = 0; c < nc; ++c) {  // vertex regions in chain order
    hch[c].vtx_base = vest;
    vest += (hch[c].vcap + 127) / 128 * 128;
  }
  const int64_t nt = std::max<int64_t>(1, (int64_t)ttab.size());
  const int64_t ns = std::max<int64_t>(1, (int64_t)stab.size());
  const int64_t nb = std::max<int64_t>(1, (int64_t)btab.size());
  int rc = 0;
#define GROW(ptr, cap, need, T)                                                     \
  if ((rc = grow_array((void **)&(ptr), &(cap), (need), sizeof(T))) != 0) return rc
  GROW(dch_, cap_chains_, std::max(nc, 1), DevChain);
  GROW(tile_tab_, cap_tt_, nt, int2);
  GROW(site_tab_, cap_st_, ns, int2);
  GROW(bond_tab_, cap_bt_, nb, int2);
  GROW(s_.vptr, cap_cells_, std::max<int64_t>(1, cell_off), int32_t);
  int64_t c1 = cap_tiles_, c2 = cap_tiles_, c3 = cap_tiles_, c4 = cap_tiles_, c5 = cap_tiles_,
          c6 = cap_tiles_, c7 = cap_tiles_, c9 = cap_tiles_;
  if (nt > cap_tiles_) {
    GROW(s_.tile_sum, c1, nt, int64_t);
    GROW(s_.tile_pref, c2, nt, int64_t);
    GROW(s_.tile_sum2, c3, nt, int64_t);
    GROW(s_.tile_pref2, c4, nt, int64_t);
    GROW(s_.tile_roots, c5, nt, int64_t);
    GROW(s_.tile_sw2, c6, 2 * nt, unsigned long long);
    GROW(s_.tile_sf2, c7, 2 * nt, unsigned long long);
    GROW(s_.tile_sz2, c9, 2 * nt, unsigned long long);
    int64_t c8 = cap_tiles_;
    GROW(s_.tile_state, c8, nt, unsigned long long);
    cap_tiles_ = nt;
  }
  if (ns > cap_sites_) {
    int64_t a1 = cap_sites_, a2 = cap_sites_, a3 = cap_sites_;
    GROW(s_.site_free, a1, ns, int64_t);
    GROW(s_.site_sw2, a2, 2 * ns, unsigned long long);
    GROW(s_.site_sf2, a3, 2 * ns, unsigned long long);
    cap_sites_ = ns;
  }
  GROW(s_.bpar, cap_bpar_, std::max<int64_t>(1, bpar_off), uint8_t);
  if (sub_off > cap_subs_ || !s_.cut_node) {
    int64_t a1 = cap_subs_, a2 = cap_subs_, a3 = cap_subs_, a4 = cap_subs_, a5 = cap_subs_;
    const int64_t need = std::max<int64_t>(1, sub_off);
    GROW(s_.cut_node, a1, need, int32_t);
    GROW(s_.cut_cell, a2, need, int32_t);
    GROW(s_.free_min, a3, need, int32_t);
    GROW(s_.cut_cross, a4, need, int8_t);
    GROW(s_.free_len, a5, need, int8_t);
    cap_subs_ = need;
  }
#undef GROW
  if (nc > 0) {
    CK(cudaMemcpyAsync(dch_, hch.data(), sizeof(DevChain) * nc, cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(tile_tab_, ttab.data(), sizeof(int2) * ttab.size(), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(site_tab_, stab.data(), sizeof(int2) * stab.size(), cudaMemcpyHostToDevice, st_));
    CK(cudaMemcpyAsync(bond_tab_, btab.data(), sizeof(int2) * btab.size(), cudaMemcpyHostToDevice, st_));
  }
  fixed_bytes_ = 4 * (size_t)cap_cells_ + 112 * (size_t)cap_tiles_ + 48 * (size_t)cap_sites_ +
                 (size_t)cap_bpar_ + 14 * (size_t)cap_subs_ + sizeof(DevChain) * (size_t)cap_chains_;
  L_.ch = dch_;
  L_.nchains = nc;
  L_.tile_tab = tile_tab_;
  L_.site_tab = site_tab_;
  L_.bond_tab = bond_tab_;
  L_.s = s_;
  drop_graphs();
  if (vest > vcap_) {
    rc = alloc_vertex(vest);
    if (rc) return rc;
  } else {
    L_.s = s_;
  }
  L_.s = s_;
  CK(cudaStreamSynchronize(st_));
  return LCQMC_OK;
}

int Engine::init(const std::vector<ChainSpec> &specs, void *stream, const lcqmc_allocator *alloc,
                 int ring_cap) {
  if (specs.empty()) {
    set_error("empty batch");
    return LCQMC_E_INVAL;
  }
  int rc = open(stream, alloc, ring_cap);
  if (rc) return rc;
  std::vector<ChainState *> v;
  for (const auto &sp : specs) {
    owned_.push_back(std::make_unique<ChainState>());
    rc = create_state(sp, owned_.back().get());
    if (rc) return rc;
    v.push_back(owned_.back().get());
  }
  return set_chains(v);
}

// ---- update sequence ---------------------------------------------------------------------
int Engine::enqueue_one(bool timed, int slot) {
  const int64_t nw = vcap_ / 32 + 1;
  // phases as in the paper's Table 3 rows: event pairs and NVTX ranges
  static const char *const kPhase[LCQMC_NPHASE] = {"lcqmc.insert",    "lcqmc.cut",
                                                   "lcqmc.link_union", "lcqmc.loop_ids",
                                                   "lcqmc.loop_props", "lcqmc.op_offsets",
                                                   "lcqmc.op_rewrite", "lcqmc.spin_rewrite"};
  auto mark = [&](int k) {
    if (!timed) return;
    cudaEventRecord(ev_[slot * (LCQMC_NPHASE + 1) + k], st_);
    if (k > 0) nvtxRangePop();
    if (k < LCQMC_NPHASE) nvtxRangePushA(kPhase[k]);
  };
  mark(0);  // [0] labeling: random numbers, insertion, vertex offsets (one pass)
  launch_bond_parity(L_, st_);
  launch_clear(L_, cap_tiles_, nw, st_);
  launch_insert(L_, st_);
  mark(1);  // [1] tau = 0 cut
  launch_cut(L_, st_);
  mark(2);  // [2] linking + union-find
  launch_link(L_, st_);
  mark(3);  // [3] loop ids (compression, coins)
  launch_compress(L_, st_);
  if (L_.check_forest) launch_check_forest(L_, st_);
  mark(4);  // [4] loop properties, new flags
  launch_est(L_, st_);
  mark(5);  // [5] operator offsets
  launch_scan_ops(L_, st_);
  mark(6);  // [6] operator rewrite
  launch_compact(L_, st_);
  mark(7);  // [7] spin rewrite + record
  launch_sites(L_, st_);
  launch_final(L_, st_);
  mark(8);
  CK(cudaGetLastError());
  return LCQMC_OK;
}

void Engine::drop_graphs() {
  if (gexec_) cudaGraphExecDestroy(gexec_);
  if (gexec_blk_) cudaGraphExecDestroy(gexec_blk_);
  gexec_ = gexec_blk_ = nullptr;
}

// Captures `count` consecutive updates as one graph (the launches carry the
// current buffers, block sizes and temporal switch: drop_graphs() whenever
// one of those changes).
int Engine::capture(int count, cudaGraphExec_t *out) {
  if (*out) return LCQMC_OK;
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(st_, cudaStreamCaptureModeThreadLocal));
  int rc = LCQMC_OK;
  for (int i = 0; i < count && !rc; ++i) rc = enqueue_one(false, 0);
  cudaError_t e = cudaStreamEndCapture(st_, &g);
  if (rc) {
    if (e == cudaSuccess) cudaGraphDestroy(g);
    return rc;
  }
  CK(e);
  e = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return LCQMC_OK;
}

int Engine::update(int64_t n) {
  if (n < 0) {
    set_error("negative update count");
    return LCQMC_E_INVAL;
  }
  if (n == 0) return LCQMC_OK;
  NvtxRange range("lcqmc_update");
  if (pending_ == 0) pending_sweep0_ = hch[0].sweep;
  if (timing_) {
    const int per = LCQMC_NPHASE + 1;
    while ((int)ev_.size() < (ev_used_ + (int)n) * per) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ev_.push_back(e);
    }
    for (int64_t i = 0; i < n; ++i) {
      int rc = enqueue_one(true, ev_used_++);
      if (rc) return rc;
    }
  } else if (serving_) {
    for (int64_t i = 0; i < n; ++i) {
      int rc = enqueue_one(false, 0);
      if (rc) return rc;
    }
  } else {
    const int64_t nblk = n / kGraphBlock, rest = n % kGraphBlock;
    int rc = nblk ? capture(kGraphBlock, &gexec_blk_) : LCQMC_OK;
    if (!rc && rest) rc = capture(1, &gexec_);
    if (rc) return rc;
    for (int64_t i = 0; i < nblk; ++i) CK(cudaGraphLaunch(gexec_blk_, st_));
    for (int64_t i = 0; i < rest; ++i) CK(cudaGraphLaunch(gexec_, st_));
  }
  pending_ += n;
  return LCQMC_OK;
}

int Engine::pull_chains() {
  if (hch.empty()) return LCQMC_OK;
  CK(cudaMemcpyAsync(hch.data(), dch_, sizeof(DevChain) * hch.size(), cudaMemcpyDeviceToHost, st_));
  CK(cudaStreamSynchronize(st_));
  for (size_t c = 0; c < hch.size(); ++c) cs_[c]->dev = hch[c];
  return LCQMC_OK;
}

int Engine::push_chains() {
  if (hch.empty()) return LCQMC_OK;
  CK(cudaMemcpyAsync(dch_, hch.data(), sizeof(DevChain) * hch.size(), cudaMemcpyHostToDevice, st_));
  CK(cudaStreamSynchronize(st_));
  for (size_t c = 0; c < hch.size(); ++c) cs_[c]->dev = hch[c];
  return LCQMC_OK;
}

int Engine::grow_ops(int64_t c, int64_t need) {
  DevChain &d = hch[c];
  ChainBuf &b = cs_[c]->buf;
  const int64_t cap = need + need / 4 + 1024;
  const int64_t nold = 0;
  (void)nold;
  for (int k = 0; k < 2; ++k) {
    double *p;
    DALLOC(p, double, cap + 2);  // +2: bulk copies end on a 16-byte bound
    if (k == d.cur) {
      int32_t n_off = 0;
      CK(cudaMemcpyAsync(&n_off, b.op_ptr[k] + d.ncell, 4, cudaMemcpyDeviceToHost, st_));
      CK(cudaStreamSynchronize(st_));
      if (n_off > 0)
        CK(cudaMemcpyAsync(p, b.op_tau[k], 8 * (size_t)n_off, cudaMemcpyDeviceToDevice, st_));
    }
    CK(cudaStreamSynchronize(st_));
    dfree(b.op_tau[k]);
    b.op_tau[k] = p;
    d.op_tau[k] = p;
  }
  op_bytes_ += 2 * 8 * (size_t)(cap - d.op_cap);
  d.op_cap = cap;
  return LCQMC_OK;
}

int Engine::sync() {
  for (int guard = 0; guard < 64; ++guard) {
    CK(cudaStreamSynchronize(st_));
    int status = 0;
    CK(cudaMemcpy(&status, s_.status, sizeof(int), cudaMemcpyDeviceToHost));
    int rc = pull_chains();
    if (rc) return rc;
    if (timing_ && ev_used_ > 0) {
      for (int u = 0; u < ev_used_; ++u)
        for (int k = 0; k < LCQMC_NPHASE; ++k) {
          float ms = 0.f;
          if (cudaEventElapsedTime(&ms, ev_[u * (LCQMC_NPHASE + 1) + k],
                                   ev_[u * (LCQMC_NPHASE + 1) + k + 1]) == cudaSuccess)
            phase_ms_[k] += ms;
        }
      ev_used_ = 0;
    }
    if (status == 0) {
      pending_ = 0;
      return LCQMC_OK;
    }
    const int64_t done = (int64_t)(uint32_t)(hch[0].sweep - pending_sweep0_);
    const int64_t remaining = pending_ - done;
    if (status & (ST_TIMEOUT | ST_INTERNAL | ST_BADSTATE | ST_ID_OVERFLOW)) {
      CK(cudaMemsetAsync(s_.status, 0, sizeof(int), st_));
      pending_ = 0;
      if (status & ST_TIMEOUT) {
        set_error("a bounded union-find wait ran out on the device");
        return LCQMC_E_DEVICE_TIMEOUT;
      }
      if (status & ST_ID_OVERFLOW) {
        set_error("more than 2^31 - 4096 graph vertices in one chain");
        return LCQMC_E_ID_OVERFLOW;
      }
      if (status & ST_BADSTATE) {
        set_error("configuration violates the world-line constraint at tau=0");
        return LCQMC_E_STATE;
      }
      long long dbg[8] = {0};
      cudaMemcpy(dbg, s_.dbg, sizeof(dbg), cudaMemcpyDeviceToHost);
      cudaMemset(s_.dbg, 0, sizeof(dbg));
      char msg[256];
      std::snprintf(msg, sizeof msg,
                    "internal consistency check %lld failed on the device (%lld %lld %lld %lld %lld)",
                    dbg[0], dbg[1], dbg[2], dbg[3], dbg[4], dbg[5]);
      set_error(msg);
      return LCQMC_E_CUDA;
    }
    if (status & ST_VTX_OVERFLOW) {
      for (size_t c = 0; c < cs_.size(); ++c)
        if (hch[c].n > cs_[c]->vcap) cs_[c]->vcap = (hch[c].n + hch[c].n / 8 + 4096 + 127) / 128 * 128;
      rc = layout();
      if (rc) return rc;
    }
    if (status & ST_OP_OVERFLOW) {
      for (int64_t c = 0; c < (int64_t)hch.size(); ++c)
        if (hch[c].n_off_new > hch[c].op_cap) {
          rc = grow_ops(c, hch[c].n_off_new);
          if (rc) return rc;
        }
      rc = push_chains();
      if (rc) return rc;
      drop_graphs();
    }
    CK(cudaMemsetAsync(s_.status, 0, sizeof(int), st_));
    pending_ = 0;
    if (remaining > 0) {
      replays_ += remaining;
      rc = update(remaining);
      if (rc) return rc;
    }
  }
  set_error("capacity growth did not converge");
  return LCQMC_E_NOMEM;
}

// ---- measurements ------------------------------------------------------------------------
int Engine::measure(int64_t c, lcqmc_obs *out) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  std::memset(out, 0, sizeof(*out));
  out->n_updates = d.n_updates;
  for (int k = 0; k < NOBS; ++k) {
    out->sum[k] = d.sum[k];
    out->sumsq[k] = d.sumsq[k];
  }
  if (d.n_updates > 0 && d.sum[2] > 0) {
    const double r = d.sum[1] / d.sum[2] - 1.0;
    out->xi = r > 0 ? (double)d.L / (2.0 * M_PI) * std::sqrt(r) : 0.0;
  }
  // second moment in imaginary time: xi_tau = (beta/2pi) sqrt(chi(pi,0)/chi(pi,w1) - 1),
  // gap = 1/xi_tau (Sec. 5)
  if (d.n_updates > 0 && d.sum[8] > 0) {
    const double r = d.sum[1] / d.sum[8] - 1.0;
    out->xi_tau = r > 0 ? d.beta / (2.0 * M_PI) * std::sqrt(r) : 0.0;
    out->gap = out->xi_tau > 0 ? 1.0 / out->xi_tau : 0.0;
  }
  return LCQMC_OK;
}

int Engine::reset_obs(int64_t c) {
  int rc = sync();
  if (rc) return rc;
  DevChain &d = hch[c];
  d.n_updates = 0;
  for (int k = 0; k < NOBS; ++k) d.sum[k] = d.sumsq[k] = 0.0;
  return push_chains();
}

int Engine::records(int64_t c, lcqmc_record *out, int64_t max, int64_t *count) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  int64_t &rd = cs_[c]->rec_read;
  if (d.n_rec - rd > d.ring_cap) rd = d.n_rec - d.ring_cap;
  int64_t avail = d.n_rec - rd;
  const int64_t m = std::min<int64_t>(avail, std::max<int64_t>(0, max));
  for (int64_t i = 0; i < m; ++i) {
    const int64_t slot = (rd + i) % d.ring_cap;
    CK(cudaMemcpyAsync(out + i, cs_[c]->buf.ring + slot, sizeof(lcqmc_record), cudaMemcpyDeviceToHost, st_));
  }
  CK(cudaStreamSynchronize(st_));
  rd += m;
  *count = m;
  return LCQMC_OK;
}

int Engine::geometry(int64_t c, lcqmc_geometry *out) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  out->L = d.L;
  out->nsub = d.nsub;
  out->nbond = d.nbond;
  out->nwin = d.nwin;
  out->ncell = d.ncell;
  out->Q = d.Q;
  out->F = d.F;
  out->J = d.J;
  out->beta = d.beta;
  out->w = d.w;
  out->seed = d.seed;
  out->sweep = d.sweep;
  out->replays = (uint32_t)std::min<int64_t>(replays_, 0xffffffffll);
  return LCQMC_OK;
}

int Engine::export_config(int64_t c, uint8_t *s0, int32_t *op_ptr, double *op_tau, int64_t op_cap,
                          int64_t *n_off) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  const ChainBuf &b = cs_[c]->buf;
  int32_t n = 0;
  CK(cudaMemcpy(&n, b.op_ptr[d.cur] + d.ncell, 4, cudaMemcpyDeviceToHost));
  if (n_off) *n_off = n;
  if (s0) CK(cudaMemcpy(s0, b.s0[d.cur], d.nsub, cudaMemcpyDeviceToHost));
  if (op_ptr) CK(cudaMemcpy(op_ptr, b.op_ptr[d.cur], 4 * ((size_t)d.ncell + 1), cudaMemcpyDeviceToHost));
  if (op_tau) {
    if (op_cap < n) {
      set_error("op_tau buffer too small");
      return LCQMC_E_CAPACITY;
    }
    if (n > 0) CK(cudaMemcpy(op_tau, b.op_tau[d.cur], 8 * (size_t)n, cudaMemcpyDeviceToHost));
  }
  return LCQMC_OK;
}

// World-line validity of an imported state (Sec. 2): every operator in its
// cell's window, ascending within the cell, acting on antiparallel spins; the
// spins at tau = beta equal those at tau = 0 (up to a subspin permutation of
// each site for S = 1).
static int check_state(const DevChain &d, const uint8_t *s0, const int32_t *op_ptr,
                       const double *op_tau, int64_t n_off) {
  if (op_ptr[0] != 0 || op_ptr[d.ncell] != n_off) return LCQMC_E_STATE;
  for (int u = 0; u < d.nsub; ++u)
    if (s0[u] > 1) return LCQMC_E_STATE;
  struct Ev {
    double tau;
    int bond;
  };
  std::vector<Ev> ev;
  ev.reserve(n_off);
  for (int b = 0; b < d.nbond; ++b)
    for (int j = 0; j < d.nwin; ++j) {
      const int blk = j / TW, jj = j - blk * TW, tw = std::min(TW, d.nwin - blk * TW);
      const int c = blk * d.nbond * TW + b * tw + jj;
      if (op_ptr[c + 1] < op_ptr[c]) return LCQMC_E_STATE;
      const double t0 = (double)j * d.w;
      const double t_end = (j == d.nwin - 1) ? d.beta : (double)(j + 1) * d.w;
      for (int q = op_ptr[c]; q < op_ptr[c + 1]; ++q) {
        if (!(op_tau[q] >= t0 && op_tau[q] < t_end)) return LCQMC_E_STATE;
        if (q > op_ptr[c] && op_tau[q] < op_tau[q - 1]) return LCQMC_E_STATE;
        ev.push_back(Ev{op_tau[q], b});
      }
    }
  std::sort(ev.begin(), ev.end(), [](const Ev &a, const Ev &b) {
    return a.tau < b.tau || (a.tau == b.tau && a.bond < b.bond);
  });
  std::vector<uint8_t> s(s0, s0 + d.nsub);
  const int Q = d.Q;
  for (const Ev &e : ev) {
    const int i = e.bond / (Q * Q), a = (e.bond / Q) % Q, a2 = e.bond % Q;
    const int ul = i * Q + a, ur = ((i + 1) % d.L) * Q + a2;
    if (s[ul] == s[ur]) return LCQMC_E_STATE;
    s[ul] ^= 1;
    s[ur] ^= 1;
  }
  for (int i = 0; i < d.L; ++i) {
    int top = 0, bot = 0;
    for (int a = 0; a < Q; ++a) {
      top += s[i * Q + a];
      bot += s0[i * Q + a];
    }
    if (top != bot) return LCQMC_E_STATE;
  }
  return LCQMC_OK;
}

int Engine::import_config(int64_t c, const uint8_t *s0, const int32_t *op_ptr, const double *op_tau,
                          int64_t n_off, uint32_t sweep) {
  int rc = sync();
  if (rc) return rc;
  DevChain &d = hch[c];
  if (n_off < 0 || (n_off > 0 && !op_tau) || !s0 || !op_ptr) {
    set_error("bad arguments to import_config");
    return LCQMC_E_INVAL;
  }
  rc = check_state(d, s0, op_ptr, op_tau, n_off);
  if (rc) {
    set_error("imported configuration is not a valid world-line state");
    return rc;
  }
  if (n_off > d.op_cap) {
    rc = grow_ops(c, n_off);
    if (rc) return rc;
    drop_graphs();
  }
  const ChainBuf &b = cs_[c]->buf;
  CK(cudaMemcpy(b.s0[d.cur], s0, d.nsub, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b.op_ptr[d.cur], op_ptr, 4 * ((size_t)d.ncell + 1), cudaMemcpyHostToDevice));
  if (n_off > 0) CK(cudaMemcpy(b.op_tau[d.cur], op_tau, 8 * (size_t)n_off, cudaMemcpyHostToDevice));
  d.sweep = sweep;
  return push_chains();
}

int Engine::export_graph(int64_t c, double *tau, uint8_t *flag, int32_t *pl, int32_t *pr,
                         int32_t *root, int64_t n_cap, int64_t *n) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  const int64_t nv = d.n;
  if (n) *n = nv;
  if (!tau && !flag && !pl && !pr && !root) return LCQMC_OK;
  if (n_cap < nv) {
    set_error("graph buffers too small");
    return LCQMC_E_CAPACITY;
  }
  const int64_t vb = d.vtx_base;
  if (tau) CK(cudaMemcpy(tau, s_.vtau + vb, 8 * nv, cudaMemcpyDeviceToHost));
  if (flag) {
    CK(cudaMemcpy(flag, s_.vflag + vb, nv, cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < nv; ++i) flag[i] &= VF_OLD;
  }
  if (pl) CK(cudaMemcpy(pl, s_.pl + vb, 4 * nv, cudaMemcpyDeviceToHost));
  if (pr) CK(cudaMemcpy(pr, s_.pr + vb, 4 * nv, cudaMemcpyDeviceToHost));
  if (root) CK(cudaMemcpy(root, s_.parent + vb, 4 * nv, cudaMemcpyDeviceToHost));
  return LCQMC_OK;
}

int Engine::export_cells(int64_t c, int32_t *vptr, int64_t cap) {
  int rc = sync();
  if (rc) return rc;
  const DevChain &d = hch[c];
  if (!vptr || cap < (int64_t)d.ncell + 1) {
    set_error("cell offset buffer too small");
    return LCQMC_E_CAPACITY;
  }
  CK(cudaMemcpy(vptr, s_.vptr + d.cell_off, 4 * ((size_t)d.ncell + 1), cudaMemcpyDeviceToHost));
  return LCQMC_OK;
}

int Engine::set_phase_timing(int enable) {
  int rc = sync();
  if (rc) return rc;
  timing_ = enable != 0;
  for (double &x : phase_ms_) x = 0.0;
  return LCQMC_OK;
}

int Engine::set_wait_limit(int64_t limit) {
  if (limit < 0 || limit > UF_MAX_ITERS) {
    set_error("wait limit out of range: 1 .. 2^22, or 0 for the default");
    return LCQMC_E_INVAL;
  }
  int rc = sync();
  if (rc) return rc;
  s_.uf_limit = limit ? (int)limit : UF_MAX_ITERS;
  L_.s = s_;
  drop_graphs();  // the captured launches carry the scratch descriptor
  return LCQMC_OK;
}

int Engine::set_temporal(int enable) {
  int rc = sync();
  if (rc) return rc;
  if ((L_.temporal != 0) != (enable != 0)) {
    L_.temporal = enable != 0;
    drop_graphs();  // the captured launches carry the choice
  }
  return LCQMC_OK;
}

void Engine::get_tuning(lcqmc_tuning *out) const {
  out->link_threads = L_.link_threads;
  out->link_x_warps = L_.link_x_warps;
  out->compress_threads = L_.compress_threads;
  out->pad = 0;
}

int Engine::set_tuning(const lcqmc_tuning &t) {
  if (!(t.link_threads == 128 || t.link_threads == 256) || t.link_x_warps < 1 || t.link_x_warps > 8 ||
      t.compress_threads < 32 || t.compress_threads > 128 || t.compress_threads % 32 != 0) {
    set_error("tuning out of range: link_threads 128 or 256, link_x_warps 1..8, "
              "compress_threads 32..128 in steps of 32");
    return LCQMC_E_INVAL;
  }
  int rc = sync();
  if (rc) return rc;
  L_.link_threads = t.link_threads;
  L_.link_x_warps = t.link_x_warps;
  L_.compress_threads = t.compress_threads;
  drop_graphs();  // the captured launches carry the block sizes
  return LCQMC_OK;
}

// Coordinate search over the block sizes of the union-find phases, each
// candidate timed by the phase events over n updates: linking + global unions
// (phase 2) over link_threads x link_x_warps, then compression (phase 3) over
// compress_threads.  The trial updates are ordinary updates of every chain;
// the block sizes do not change any result.
int Engine::autotune(int64_t n, lcqmc_tuning *out) {
  if (n < 1) {
    set_error("autotune needs at least one update per trial");
    return LCQMC_E_INVAL;
  }
  const bool was_timing = timing_;
  lcqmc_tuning best;
  get_tuning(&best);
  auto trial = [&](const lcqmc_tuning &t, int phase, double *ms) -> int {
    int rc = set_tuning(t);
    if (!rc) rc = set_phase_timing(1);
    if (!rc) rc = update(n);
    if (!rc) rc = sync();
    if (!rc) *ms = phase_ms_[phase];
    return rc;
  };
  double best_ms = 1e300;
  static const int link_threads[] = {128, 256}, link_x_warps[] = {2, 4, 8}, compress_threads[] = {64, 128};
  lcqmc_tuning cur = best;
  for (int lt : link_threads)
    for (int xw : link_x_warps) {
      cur.link_threads = lt;
      cur.link_x_warps = xw;
      double ms = 0.0;
      int rc = trial(cur, 2, &ms);
      if (rc) return rc;
      if (ms < best_ms) {
        best_ms = ms;
        best = cur;
      }
    }
  best_ms = 1e300;
  cur = best;
  for (int ct : compress_threads) {
    cur.compress_threads = ct;
    double ms = 0.0;
    int rc = trial(cur, 3, &ms);
    if (rc) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best.compress_threads = ct;
    }
  }
  int rc = set_tuning(best);
  if (!rc) rc = set_phase_timing(was_timing ? 1 : 0);
  if (rc) return rc;
  if (out) *out = best;
  return LCQMC_OK;
}

int Engine::phase_times(double *ms, int nphase) {
  int rc = sync();
  if (rc) return rc;
  for (int k = 0; k < nphase && k < LCQMC_NPHASE; ++k) ms[k] = phase_ms_[k];
  return LCQMC_OK;
}

size_t Engine::footprint() const { return fixed_bytes_ + vertex_bytes_ + op_bytes_; }

}  // namespace lcq
