// Loop labelling that allocates no device memory.
//
// lcqmc_loops_noalloc runs the union-find phase of the update (link the two
// fragments below every vertex, then label every node with the smallest node
// of its loop) on a graph the caller already holds in device memory.  Its only
// scratch is the parent forest, kept in a fixed array compiled into this
// library instead of being allocated per call.
//
// Why: some callers must not call cudaMalloc.  Callers that live inside
// another framework's memory pool, or on a device whose footprint was
// budgeted when they started, may not grow their allocation at all; and
// cudaMalloc synchronizes the device, which stalls every other stream of an
// application that overlaps work.  Such callers pass inputs and outputs they
// own and get a result with no allocation on the library's side.  The call
// does wait for its own stream, to read back the status word.
//
// The fixed array holds NOALLOC_MAX_NODES int32 parents (16 MiB plus one status
// word).  Every process that loads the library reserves it on every GPU it
// touches, until the process exits.
#include <cstdio>
#include <mutex>

#include "engine.h"
#include "uf.cuh"

namespace lcq {

constexpr int64_t NOALLOC_MAX_NODES = 1 << 22;

// [0, NOALLOC_MAX_NODES): parent forest; [NOALLOC_MAX_NODES]: status word.
static __device__ __align__(256) int32_t g_noalloc_scratch[NOALLOC_MAX_NODES + 64];

// Parent = self; status cleared (the array keeps the previous call's content).
static __global__ void k_na_init(int32_t *par, int *status, int32_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) par[i] = (int32_t)i;
  if (i == 0) *status = 0;
}

// Union of the two fragments below every vertex w: pl[w] with pr[w].
static __global__ void k_na_union(const int32_t *__restrict__ pl, const int32_t *__restrict__ pr,
                                  int32_t *par, int *status, int32_t n) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const int a = pl[w], b = pr[w];
  if (a < 0 || a >= n || b < 0 || b >= n) {  // caller data out of range: skip, report
    atomicOr(status, ST_BADSTATE);
    return;
  }
  uf_union(par, a, b, status);
}

// Smallest node of each node's loop, written to the caller's output.
static __global__ void k_na_root(const int32_t *par, int32_t *root, int *status, int32_t n) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) root[v] = uf_root(par, (int)v, status);
}

}  // namespace lcq

namespace {
std::mutex g_na_mu;
void *g_na_ptr[256] = {nullptr};  // device address of the fixed array, per device
}  // namespace

extern "C" int lcqmc_loops_noalloc(const int32_t *pl, const int32_t *pr, int64_t n, int32_t *root,
                                   void *cuda_stream) {
  using namespace lcq;
  if (n < 0 || (n > 0 && (!pl || !pr || !root))) {
    set_error("lcqmc_loops_noalloc: bad arguments");
    return LCQMC_E_INVAL;
  }
  if (n > NOALLOC_MAX_NODES) {
    char msg[160];
    std::snprintf(msg, sizeof msg,
                  "lcqmc_loops_noalloc: %lld nodes exceed the fixed maximum of %lld",
                  (long long)n, (long long)NOALLOC_MAX_NODES);
    set_error(msg);
    return LCQMC_E_TOO_LARGE;
  }
  if (n == 0) return LCQMC_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
    set_error("lcqmc_loops_noalloc: no current CUDA device");
    return LCQMC_E_CUDA;
  }
  void *base;
  {
    // First call on a device: look up the device address of the fixed array
    // (the symbol's name is only a host-side stand-in for it).
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      void *p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_error(std::string("lcqmc_loops_noalloc: cudaGetSymbolAddress failed: ") +
                  cudaGetErrorString(e));
        return LCQMC_E_CUDA;
      }
      g_na_ptr[dev] = p;
    }
    base = g_na_ptr[dev];
  }
  int32_t *par = (int32_t *)base;
  int *status = (int *)(par + NOALLOC_MAX_NODES);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  k_na_init<<<blocks, threads, 0, st>>>(par, status, (int32_t)n);
  k_na_union<<<blocks, threads, 0, st>>>(pl, pr, par, status, (int32_t)n);
  k_na_root<<<blocks, threads, 0, st>>>(par, root, status, (int32_t)n);
  int h_status = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    // Forget the device address: a later call looks it up again (a context
    // that has failed may be replaced by a new one with a new address).
    {
      std::lock_guard<std::mutex> lk(g_na_mu);
      g_na_ptr[dev] = nullptr;
    }
    set_error(std::string("lcqmc_loops_noalloc: ") + cudaGetErrorString(e));
    return LCQMC_E_CUDA;
  }
  if (h_status & ST_BADSTATE) {
    set_error("lcqmc_loops_noalloc: a node id in pl/pr is outside [0, n)");
    return LCQMC_E_INVAL;
  }
  if (h_status & ST_TIMEOUT) {
    set_error("lcqmc_loops_noalloc: a bounded union-find wait ran out");
    return LCQMC_E_DEVICE_TIMEOUT;
  }
  return LCQMC_OK;
}
