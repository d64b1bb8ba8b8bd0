// Host engine: device buffers and update sequence for a batch of chains.
#pragma once
#include <cuda_runtime.h>

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
  int phase_times(double *ms, int nphase);
  size_t footprint() const;  // device bytes held
  static size_t estimate_footprint(const std::vector<ChainSpec> &specs, int ring_cap);

  cudaStream_t stream() const { return st_; }
  int nchains() const { return (int)spec_.size(); }
  const ChainSpec &spec(int64_t i) const { return spec_[i]; }
  std::vector<DevChain> hch;

 private:
  void *dalloc(size_t bytes);
  void dfree(void *p);
  int alloc_vertex(int64_t vcap);
  void free_vertex();
  int grow_ops(int64_t chain, int64_t need);
  int enqueue_one(bool timed, int slot);
  int capture();

  int device_ = 0;
  cudaStream_t st_ = nullptr;
  bool own_stream_ = false;
  lcqmc_allocator alloc_{};
  bool has_alloc_ = false;
  std::vector<ChainSpec> spec_;
  std::vector<ChainBuf> buf_;
  std::vector<int64_t> rec_read_;
  DevChain *dch_ = nullptr;
  int2 *tile_tab_ = nullptr, *site_tab_ = nullptr, *bond_tab_ = nullptr;
  Launch L_{};
  Scratch s_{};
  int64_t ncell_tot_ = 0, nsub_tot_ = 0, bpar_tot_ = 0;
  int64_t ntile_tot_ = 0, nsiteblk_tot_ = 0, nbondblk_tot_ = 0;
  int64_t vcap_ = 0;
  int ring_cap_ = 0;
  size_t fixed_bytes_ = 0, vertex_bytes_ = 0, op_bytes_ = 0;
  cudaGraphExec_t gexec_ = nullptr;
  bool timing_ = false;
  std::vector<cudaEvent_t> ev_;
  int ev_used_ = 0;
  double phase_ms_[LCQMC_NPHASE] = {0};
  int64_t pending_ = 0;
  uint32_t pending_sweep0_ = 0;
};

}  // namespace lcq
