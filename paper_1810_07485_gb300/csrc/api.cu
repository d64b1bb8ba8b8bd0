// extern "C" entry points of include/lcqmc.h: single chains and batches.
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <vector>

#include "engine.h"

namespace lcq {
const char *last_error();
}
using lcq::Engine;

struct lcqmc_chain {
  Engine eng;
};
struct lcqmc_batch {
  Engine eng;
};

namespace {

constexpr int kChainRing = 4096;
constexpr int kBatchRing = 256;
constexpr char kMagic[8] = {'L', 'C', 'Q', 'M', 'C', 'C', 'K', '1'};

struct CkptHeader {
  char magic[8];
  int64_t L;
  int32_t Q, pad;
  double J, beta;
  uint64_t seed;
  uint32_t sweep, pad2;
  int64_t nsub, ncell, n_off;
};

int make_chain(int64_t L, double S, double J, double beta, uint64_t seed, void *stream,
               const lcqmc_allocator *alloc, lcqmc_handle *out) {
  if (!out) {
    lcq::set_error("null output handle");
    return LCQMC_E_INVAL;
  }
  *out = nullptr;
  lcq::ChainSpec sp;
  int rc = lcq::validate_spec(L, S, J, beta, sp);
  if (rc) return rc;
  sp.seed = seed;
  auto *h = new (std::nothrow) lcqmc_chain;
  if (!h) {
    lcq::set_error("host allocation failed");
    return LCQMC_E_NOMEM;
  }
  rc = h->eng.init({sp}, stream, alloc, kChainRing);
  if (rc) {
    delete h;
    return rc;
  }
  *out = h;
  return LCQMC_OK;
}

}  // namespace

extern "C" {

const char *lcqmc_last_error(void) { return lcq::last_error(); }

// Host-side check of the integer forms of the method's rounding steps (the
// same functions the kernels run) against the C library's fma / llrint.
int lcqmc_selftest(int which, int64_t n, uint64_t seed, int64_t *mismatches) {
  if (!mismatches || n < 0) return LCQMC_E_INVAL;
  uint64_t x = seed * 0x9E3779B97F4A7C15ull + 1;
  auto next = [&x]() {  // splitmix64
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto unif = [&]() { return (double)(next() >> 11) * 0x1p-53; };
  int64_t bad = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (which == 0) {
      // the unit factor u53 * 2^-53 of a candidate time, over all magnitudes
      uint64_t u53 = next() >> 11;
      u53 >>= next() % 54;
      const double ref = std::ldexp((double)u53, -53);
      uint64_t rbits;
      std::memcpy(&rbits, &ref, 8);
      if (lcq::unit_bits(u53) != rbits) ++bad;
    } else if (which == 1) {
      const int F = (int)(next() % 63);
      const double v = std::ldexp(unif() + 0.5, (int)(next() % 60) - 40);
      if (!(std::ldexp(v, F) < 0x1p62)) continue;
      uint64_t vb;
      std::memcpy(&vb, &v, 8);
      if (lcq::q_time(vb, F) != std::llrint(std::ldexp(v, F))) ++bad;
    } else {
      return LCQMC_E_INVAL;
    }
  }
  *mismatches = bad;
  return LCQMC_OK;
}

int lcqmc_create(int64_t L, double S, double J, double beta, uint64_t seed, lcqmc_handle *out) {
  return make_chain(L, S, J, beta, seed, nullptr, nullptr, out);
}

int lcqmc_create_ex(int64_t L, double S, double J, double beta, uint64_t seed, void *cuda_stream,
                    const lcqmc_allocator *alloc, lcqmc_handle *out) {
  return make_chain(L, S, J, beta, seed, cuda_stream, alloc, out);
}

#define NEED(h)                                   \
  do {                                            \
    if (!(h)) {                                   \
      lcq::set_error("null handle");              \
      return LCQMC_E_INVAL;                       \
    }                                             \
  } while (0)

int lcqmc_update(lcqmc_handle h, int64_t n) {
  NEED(h);
  return h->eng.update(n);
}
int lcqmc_sync(lcqmc_handle h) {
  NEED(h);
  return h->eng.sync();
}
int lcqmc_measure(lcqmc_handle h, lcqmc_obs *out) {
  NEED(h);
  if (!out) return LCQMC_E_INVAL;
  return h->eng.measure(0, out);
}
int lcqmc_reset_obs(lcqmc_handle h) {
  NEED(h);
  return h->eng.reset_obs(0);
}
int lcqmc_get_records(lcqmc_handle h, lcqmc_record *out, int64_t max, int64_t *count) {
  NEED(h);
  if (!count || (max > 0 && !out)) return LCQMC_E_INVAL;
  return h->eng.records(0, out, max, count);
}
int lcqmc_get_geometry(lcqmc_handle h, lcqmc_geometry *out) {
  NEED(h);
  if (!out) return LCQMC_E_INVAL;
  return h->eng.geometry(0, out);
}
int lcqmc_export_config(lcqmc_handle h, uint8_t *s0, int32_t *op_ptr, double *op_tau,
                        int64_t op_cap, int64_t *n_off) {
  NEED(h);
  return h->eng.export_config(0, s0, op_ptr, op_tau, op_cap, n_off);
}
int lcqmc_import_config(lcqmc_handle h, const uint8_t *s0, const int32_t *op_ptr,
                        const double *op_tau, int64_t n_off, uint32_t sweep) {
  NEED(h);
  return h->eng.import_config(0, s0, op_ptr, op_tau, n_off, sweep);
}
int lcqmc_set_keep_graph(lcqmc_handle h, int keep) {
  NEED(h);
  (void)keep;  // the vertex arrays of the last update stay until the next one
  return LCQMC_OK;
}
int lcqmc_export_graph(lcqmc_handle h, double *tau, uint8_t *flag, int32_t *pl, int32_t *pr,
                       int32_t *root, int64_t n_cap, int64_t *n) {
  NEED(h);
  return h->eng.export_graph(0, tau, flag, pl, pr, root, n_cap, n);
}

int lcqmc_export_cells(lcqmc_handle h, int32_t *vptr, int64_t cap) {
  NEED(h);
  return h->eng.export_cells(0, vptr, cap);
}

int lcqmc_checkpoint(lcqmc_handle h, void *buf, size_t *len) {
  NEED(h);
  if (!len) return LCQMC_E_INVAL;
  lcqmc_geometry g;
  int rc = h->eng.geometry(0, &g);
  if (rc) return rc;
  int64_t n_off = 0;
  rc = h->eng.export_config(0, nullptr, nullptr, nullptr, 0, &n_off);
  if (rc) return rc;
  const size_t need = sizeof(CkptHeader) + (size_t)g.nsub + 4 * ((size_t)g.ncell + 1) + 8 * (size_t)n_off;
  if (!buf) {
    *len = need;
    return LCQMC_OK;
  }
  if (*len < need) {
    *len = need;
    lcq::set_error("checkpoint buffer too small");
    return LCQMC_E_CAPACITY;
  }
  CkptHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kMagic, 8);
  hd.L = g.L;
  hd.Q = g.Q;
  hd.J = g.J;
  hd.beta = g.beta;
  hd.seed = g.seed;
  hd.sweep = g.sweep;
  hd.nsub = g.nsub;
  hd.ncell = g.ncell;
  hd.n_off = n_off;
  char *p = (char *)buf;
  std::memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  uint8_t *s0 = (uint8_t *)p;
  int32_t *ptr = (int32_t *)(p + g.nsub);
  double *tau = (double *)(p + g.nsub + 4 * (g.ncell + 1));
  // Unaligned host buffers: copy through aligned temporaries.
  std::vector<uint8_t> vs(g.nsub);
  std::vector<int32_t> vp(g.ncell + 1);
  std::vector<double> vt(n_off > 0 ? n_off : 1);
  rc = h->eng.export_config(0, vs.data(), vp.data(), vt.data(), n_off, &n_off);
  if (rc) return rc;
  std::memcpy(s0, vs.data(), g.nsub);
  std::memcpy(ptr, vp.data(), 4 * (g.ncell + 1));
  std::memcpy(tau, vt.data(), 8 * n_off);
  *len = need;
  return LCQMC_OK;
}

int lcqmc_restore(lcqmc_handle h, const void *buf, size_t len) {
  NEED(h);
  if (!buf || len < sizeof(CkptHeader)) return LCQMC_E_INVAL;
  CkptHeader hd;
  std::memcpy(&hd, buf, sizeof(hd));
  lcqmc_geometry g;
  int rc = h->eng.geometry(0, &g);
  if (rc) return rc;
  if (std::memcmp(hd.magic, kMagic, 8) != 0 || hd.L != g.L || hd.Q != g.Q || hd.J != g.J ||
      hd.beta != g.beta || hd.seed != g.seed || hd.nsub != g.nsub || hd.ncell != g.ncell ||
      hd.n_off < 0) {
    lcq::set_error("checkpoint does not match this chain");
    return LCQMC_E_STATE;
  }
  const size_t need = sizeof(CkptHeader) + (size_t)g.nsub + 4 * ((size_t)g.ncell + 1) + 8 * (size_t)hd.n_off;
  if (len < need) return LCQMC_E_INVAL;
  const char *p = (const char *)buf + sizeof(hd);
  std::vector<uint8_t> vs(p, p + g.nsub);
  std::vector<int32_t> vp(g.ncell + 1);
  std::vector<double> vt(hd.n_off > 0 ? hd.n_off : 1);
  std::memcpy(vp.data(), p + g.nsub, 4 * (g.ncell + 1));
  std::memcpy(vt.data(), p + g.nsub + 4 * (g.ncell + 1), 8 * hd.n_off);
  return h->eng.import_config(0, vs.data(), vp.data(), vt.data(), hd.n_off, hd.sweep);
}

int lcqmc_set_phase_timing(lcqmc_handle h, int enable) {
  NEED(h);
  return h->eng.set_phase_timing(enable);
}
int lcqmc_set_temporal(lcqmc_handle h, int enable) {
  NEED(h);
  return h->eng.set_temporal(enable);
}
int lcqmc_set_wait_limit(lcqmc_handle h, int64_t limit) {
  NEED(h);
  return h->eng.set_wait_limit(limit);
}
int lcqmc_get_tuning(lcqmc_handle h, lcqmc_tuning *out) {
  NEED(h);
  if (!out) {
    lcq::set_error("null output");
    return LCQMC_E_INVAL;
  }
  h->eng.get_tuning(out);
  return LCQMC_OK;
}
int lcqmc_set_tuning(lcqmc_handle h, const lcqmc_tuning *cfg) {
  NEED(h);
  if (!cfg) {
    lcq::set_error("null tuning");
    return LCQMC_E_INVAL;
  }
  return h->eng.set_tuning(*cfg);
}
int lcqmc_autotune(lcqmc_handle h, int64_t updates_per_trial, lcqmc_tuning *out) {
  NEED(h);
  return h->eng.autotune(updates_per_trial, out);
}
int lcqmc_get_phase_times(lcqmc_handle h, double *ms, int nphase) {
  NEED(h);
  if (!ms) return LCQMC_E_INVAL;
  return h->eng.phase_times(ms, nphase);
}
void *lcqmc_stream(lcqmc_handle h) { return h ? (void *)h->eng.stream() : nullptr; }

int lcqmc_destroy(lcqmc_handle h) {
  delete h;
  return LCQMC_OK;
}

// ---- batches ----------------------------------------------------------------------------
int lcqmc_batch_create(int64_t nchains, const lcqmc_chain_spec *specs, void *cuda_stream,
                       lcqmc_batch_t *out) {
  if (!out || !specs || nchains <= 0 || nchains > (1 << 20)) {
    lcq::set_error("bad batch arguments");
    return LCQMC_E_INVAL;
  }
  *out = nullptr;
  std::vector<lcq::ChainSpec> v(nchains);
  for (int64_t i = 0; i < nchains; ++i) {
    int rc = lcq::validate_spec(specs[i].L, specs[i].S, specs[i].J, specs[i].beta, v[i]);
    if (rc) return rc;
    v[i].seed = specs[i].seed;
  }
  auto *b = new (std::nothrow) lcqmc_batch;
  if (!b) return LCQMC_E_NOMEM;
  int rc = b->eng.init(v, cuda_stream, nullptr, kBatchRing);
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return LCQMC_OK;
}
int lcqmc_batch_update(lcqmc_batch_t b, int64_t n) {
  NEED(b);
  return b->eng.update(n);
}
int lcqmc_batch_sync(lcqmc_batch_t b) {
  NEED(b);
  return b->eng.sync();
}
int lcqmc_batch_measure(lcqmc_batch_t b, int64_t chain, lcqmc_obs *out) {
  NEED(b);
  if (chain < 0 || chain >= b->eng.nchains() || !out) return LCQMC_E_INVAL;
  return b->eng.measure(chain, out);
}
int lcqmc_batch_get_records(lcqmc_batch_t b, int64_t chain, lcqmc_record *out, int64_t max,
                            int64_t *count) {
  NEED(b);
  if (chain < 0 || chain >= b->eng.nchains() || !count) return LCQMC_E_INVAL;
  return b->eng.records(chain, out, max, count);
}
int lcqmc_batch_set_temporal(lcqmc_batch_t b, int enable) {
  if (!b) return LCQMC_E_INVAL;
  return b->eng.set_temporal(enable);
}
int lcqmc_batch_get_tuning(lcqmc_batch_t b, lcqmc_tuning *out) {
  if (!b || !out) return LCQMC_E_INVAL;
  b->eng.get_tuning(out);
  return LCQMC_OK;
}
int lcqmc_batch_set_tuning(lcqmc_batch_t b, const lcqmc_tuning *cfg) {
  if (!b || !cfg) return LCQMC_E_INVAL;
  return b->eng.set_tuning(*cfg);
}
int lcqmc_batch_autotune(lcqmc_batch_t b, int64_t updates_per_trial, lcqmc_tuning *out) {
  if (!b) return LCQMC_E_INVAL;
  return b->eng.autotune(updates_per_trial, out);
}
int lcqmc_batch_destroy(lcqmc_batch_t b) {
  delete b;
  return LCQMC_OK;
}

}  // extern "C"
