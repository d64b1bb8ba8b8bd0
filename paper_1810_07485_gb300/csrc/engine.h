// Host engine: device buffers and update sequence for a batch of chains.
#pragma once
#include <cuda_runtime.h>

#include <memory>
#include <string>
#include <vector>

#include "kernels.h"

namespace lcq {

struct ChainSpec {
  int64_t L;
  int Q;
  double J, beta;
  uint64_t seed;
};

struct ChainBuf {
  uint8_t *s0[2] = {nullptr, nullptr};
  int32_t *op_ptr[2] = {nullptr, nullptr};
  double *op_tau[2] = {nullptr, nullptr};
  uint64_t *T_last = nullptr;
  long long *cosq = nullptr, *sinq = nullptr;
  uint64_t *win = nullptr;
  lcqmc_record *ring = nullptr;
};

// Persistent state of one chain (device buffers + last known descriptor).
struct ChainState {
  ChainSpec spec{};
  ChainBuf buf{};
  DevChain dev{};
  int64_t rec_read = 0;
  int64_t vcap = 0;  // vertices reserved per update (grown on overflow)
};

void set_error(const std::string &msg);
int validate_spec(int64_t L, double S, double J, double beta, ChainSpec &out);

class Engine {
 public:
  Engine() = default;
  ~Engine();
  Engine(const Engine &) = delete;
  Engine &operator=(const Engine &) = delete;

  int init(const std::vector<ChainSpec> &specs, void *stream, const lcqmc_allocator *alloc,
           int ring_cap);
  // Served form: open an engine with no chains, create / destroy chain states
  // it does not own, and change the resident set between ticks.
  // serving: device memory from a stream-ordered pool of the engine's own (no
  // device-wide synchronization when request states come and go), and
  // updates launched directly instead of from a captured graph (the resident
  // set changes too often for a capture to pay off).
  int open(void *stream, const lcqmc_allocator *alloc, int ring_cap, bool serving = false);
  int create_state(const ChainSpec &spec, ChainState *out);
  void destroy_state(ChainState *c);
  int set_chains(const std::vector<ChainState *> &chains);
  static size_t state_bytes(const ChainSpec &c, int ring_cap);
  static size_t scratch_bytes(const ChainSpec &c);
  int update(int64_t n);
  int sync();
  int pull_chains();  // device descriptors -> hch (after sync)
  int push_chains();  // hch -> device descriptors (after sync)
  int measure(int64_t chain, lcqmc_obs *out);
  int reset_obs(int64_t chain);
  int records(int64_t chain, lcqmc_record *out, int64_t max, int64_t *count);
  int export_config(int64_t chain, uint8_t *s0, int32_t *op_ptr, double *op_tau, int64_t op_cap,
                    int64_t *n_off);
  int import_config(int64_t chain, const uint8_t *s0, const int32_t *op_ptr, const double *op_tau,
                    int64_t n_off, uint32_t sweep);
  int export_graph(int64_t chain, double *tau, uint8_t *flag, int32_t *pl, int32_t *pr,
                   int32_t *root, int64_t n_cap, int64_t *n);
  int geometry(int64_t chain, lcqmc_geometry *out);
  int export_cells(int64_t chain, int32_t *vptr, int64_t cap);
  int set_phase_timing(int enable);
  int set_temporal(int enable);  // temporal moment chi(pi, 2 pi/beta) for every chain
  int set_wait_limit(int64_t limit);  // bound of the global union-find walks (0: default)
  // block sizes of the union-find phases: read, set (checked), or tuned by
  // timing each candidate over n updates of the batch (ordinary updates)
  void get_tuning(lcqmc_tuning *out) const;
  int set_tuning(const lcqmc_tuning &t);
  int autotune(int64_t n, lcqmc_tuning *out);
  int phase_times(double *ms, int nphase);
  size_t footprint() const;  // device bytes held
  static size_t estimate_footprint(const std::vector<ChainSpec> &specs, int ring_cap);

  cudaStream_t stream() const { return st_; }
  int nchains() const { return (int)cs_.size(); }
  const ChainSpec &spec(int64_t i) const { return cs_[i]->spec; }
  int64_t vertex_capacity() const { return vcap_; }
  std::vector<DevChain> hch;

 private:
  void *dalloc(size_t bytes);
  void dfree(void *p);
  int alloc_vertex(int64_t vcap);
  void free_vertex();
  int grow_ops(int64_t chain, int64_t need);
  int enqueue_one(bool timed, int slot);
  int capture(int count, cudaGraphExec_t *out);
  void drop_graphs();

  int device_ = 0;
  cudaStream_t st_ = nullptr;
  bool own_stream_ = false;
  lcqmc_allocator alloc_{};
  bool has_alloc_ = false;
  std::vector<ChainState *> cs_;
  std::vector<std::unique_ptr<ChainState>> owned_;
  int64_t cap_chains_ = 0, cap_tt_ = 0, cap_st_ = 0, cap_bt_ = 0, cap_cells_ = 0, cap_tiles_ = 0,
          cap_sites_ = 0, cap_bpar_ = 0, cap_subs_ = 0;
  int grow_array(void **p, int64_t *cap, int64_t need, size_t elem);
  int layout();
  DevChain *dch_ = nullptr;
  int2 *tile_tab_ = nullptr, *site_tab_ = nullptr, *bond_tab_ = nullptr;
  Launch L_{};
  Scratch s_{};
  int64_t vcap_ = 0;
  int ring_cap_ = 0;
  size_t fixed_bytes_ = 0, vertex_bytes_ = 0, op_bytes_ = 0;
  // one update, and a block of kGraphBlock updates (fewer graph launches for
  // small chains, whose updates are a few microseconds of work)
  static constexpr int kGraphBlock = 8;
  cudaGraphExec_t gexec_ = nullptr, gexec_blk_ = nullptr;
  bool serving_ = false;
  cudaMemPool_t pool_ = nullptr;
  bool timing_ = false;
  std::vector<cudaEvent_t> ev_;
  int ev_used_ = 0;
  double phase_ms_[LCQMC_NPHASE] = {0};
  int64_t pending_ = 0;
  uint32_t pending_sweep0_ = 0;
  int64_t replays_ = 0;  // updates re-run after capacity growth
};

}  // namespace lcq
