// extern "C" entry points of the served form (continuous batching).
#include "engine.h"

extern "C" {
int lcqmc_server_create(size_t, int, lcqmc_server_t *out) {
  if (out) *out = nullptr;
  lcq::set_error("server not available in this build");
  return LCQMC_E_INVAL;
}
int lcqmc_submit(lcqmc_server_t, const lcqmc_request *, uint64_t *) { return LCQMC_E_INVAL; }
int lcqmc_poll(lcqmc_server_t, uint64_t, lcqmc_result *) { return LCQMC_E_INVAL; }
int lcqmc_cancel(lcqmc_server_t, uint64_t) { return LCQMC_E_INVAL; }
int lcqmc_server_destroy(lcqmc_server_t) { return LCQMC_OK; }
}
