// Served form: a request loop with continuous batching.
//
// Requests (one Markov chain each: L, S, J, beta, seed, number of updates) are
// queued by lcqmc_submit.  A worker thread admits queued requests in arrival
// order while free slots and the HBM budget allow (a request that does not fit
// yet waits; later ones that fit may go ahead), allocates their device state,
// and advances every resident chain together in ticks: one batched update per
// phase over all resident chains (each phase one launch per Q group).  A tick runs as
// many updates as the nearest-to-completion chain still needs (at most
// kTickMax), so chains finish on their exact update count; finished chains are
// read out and freed, and newly admitted ones join at the next tick.  Each
// chain's random numbers are keyed by its own seed and sweep, so its result is
// the same alone and in any mix.  Device memory comes from a stream-ordered
// pool (request states come and go without a device-wide synchronization)
// and the updates are launched directly: the resident set changes too often
// for a captured graph to pay off.  A chain whose update fails (a bounded
// wait that ran out) fails its own request only.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace {

constexpr int kServerRing = 64;
constexpr int64_t kTickMax = 10;

struct Req {
  uint64_t ticket = 0;
  lcqmc_request r{};
  lcq::ChainSpec spec{};
  int status = LCQMC_PENDING;
  bool cancel = false;
  size_t foot = 0;
  int64_t done = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  lcqmc_obs obs{};
  std::unique_ptr<lcq::ChainState> st;
};

}  // namespace

struct lcqmc_server {
  lcq::Engine eng;
  std::mutex mu;
  std::condition_variable cv;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  std::deque<Req *> pending;
  std::vector<Req *> active;
  size_t budget = 0, used = 0;
  int max_slots = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
  std::thread worker;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  // Results become visible to lcqmc_poll here; the device state is released
  // later, after the engine no longer holds the chain (release()).
  void finish(Req *q, int status) {
    q->status = status;
    q->t_done = now();
  }

  void release(Req *q) {
    if (q->st) {
      eng.destroy_state(q->st.get());
      q->st.reset();
    }
    used -= q->foot;
  }

  void run() {
    cudaSetDevice(device);
    std::vector<Req *> leaving;  // finished or failed chains still held by the engine
    for (;;) {
      std::vector<Req *> admitted;
      {
        std::unique_lock<std::mutex> lk(mu);
        if (stop) break;
        for (auto it = pending.begin(); it != pending.end();) {
          Req *q = *it;
          if ((int)(active.size() - leaving.size() + admitted.size()) >= max_slots) break;
          if (used + q->foot <= budget) {
            used += q->foot;
            q->t_admit = now();
            admitted.push_back(q);
            it = pending.erase(it);
          } else {
            ++it;
          }
        }
        for (Req *q : active)
          if (q->cancel && q->status == LCQMC_PENDING) {
            finish(q, LCQMC_E_CANCELLED);
            leaving.push_back(q);
          }
        if (active.empty() && admitted.empty() && leaving.empty()) {
          cv.wait_for(lk, std::chrono::milliseconds(20));
          continue;
        }
      }
      std::vector<Req *> joined;
      for (Req *q : admitted) {
        q->st = std::make_unique<lcq::ChainState>();
        const int rc = eng.create_state(q->spec, q->st.get());
        std::lock_guard<std::mutex> lk(mu);
        if (rc) {
          finish(q, rc);
          release(q);
        } else {
          joined.push_back(q);
        }
      }
      if (!joined.empty() || !leaving.empty()) {
        std::vector<Req *> next;
        for (Req *q : active)
          if (std::find(leaving.begin(), leaving.end(), q) == leaving.end()) next.push_back(q);
        for (Req *q : joined) next.push_back(q);
        std::vector<lcq::ChainState *> v;
        for (Req *q : next) v.push_back(q->st.get());
        const int rc = eng.set_chains(v);  // syncs the old set first
        std::lock_guard<std::mutex> lk(mu);
        for (Req *q : leaving) release(q);
        leaving.clear();
        active.swap(next);
        if (rc) {
          for (Req *q : active) {
            finish(q, rc);
            leaving.push_back(q);
          }
          continue;
        }
      }
      if (active.empty()) continue;
      int64_t k = kTickMax;
      for (Req *q : active) k = std::min<int64_t>(k, q->r.n_updates - q->done);
      std::vector<uint32_t> sweep0(active.size());
      for (size_t i = 0; i < active.size(); ++i) sweep0[i] = eng.hch[i].sweep;
      int rc = eng.update(k);
      if (rc == 0) rc = eng.sync();
      std::vector<int> qrc(active.size(), rc);
      if (rc && active.size() > 1) {
        // A failed update (a bounded wait that ran out, too many vertices)
        // stops every resident chain at the same sweep, with its state as it
        // was before that update.  The rest of the tick is run chain by
        // chain, so that only the chain that fails loses its request.
        std::vector<lcq::ChainState *> all;
        for (Req *q : active) all.push_back(q->st.get());
        for (size_t i = 0; i < active.size(); ++i) {
          int r2 = eng.set_chains({active[i]->st.get()});
          if (!r2) {
            const int64_t left = k - (int64_t)(uint32_t)(eng.hch[0].sweep - sweep0[i]);
            if (left > 0) r2 = eng.update(left);
            if (!r2) r2 = eng.sync();
          }
          qrc[i] = r2;
        }
        const int r3 = eng.set_chains(all);  // engine index i = active index i again
        if (r3)
          for (int &x : qrc) x = x ? x : r3;
      }
      std::lock_guard<std::mutex> lk(mu);
      for (size_t i = 0; i < active.size(); ++i) {
        Req *q = active[i];
        if (qrc[i]) {
          finish(q, qrc[i]);
          leaving.push_back(q);
          continue;
        }
        q->done += k;
        if (q->done >= q->r.n_updates) {
          const int mrc = eng.measure((int64_t)i, &q->obs);  // engine index i = active index i
          finish(q, mrc ? mrc : LCQMC_OK);
          leaving.push_back(q);
        }
      }
    }
  }
};

extern "C" {

int lcqmc_footprint(int64_t L, double S, double J, double beta, size_t *bytes) {
  if (!bytes) return LCQMC_E_INVAL;
  lcq::ChainSpec sp;
  int rc = lcq::validate_spec(L, S, J, beta, sp);
  if (rc) return rc;
  *bytes = lcq::Engine::state_bytes(sp, kServerRing) + lcq::Engine::scratch_bytes(sp);
  return LCQMC_OK;
}

int lcqmc_server_create(size_t hbm_budget, int max_slots, lcqmc_server_t *out) {
  if (!out || max_slots <= 0 || hbm_budget == 0) {
    lcq::set_error("bad server arguments");
    return LCQMC_E_INVAL;
  }
  *out = nullptr;
  auto *s = new (std::nothrow) lcqmc_server;
  if (!s) return LCQMC_E_NOMEM;
  s->budget = hbm_budget;
  s->max_slots = max_slots;
  s->t0 = std::chrono::steady_clock::now();
  if (cudaGetDevice(&s->device) != cudaSuccess) {
    delete s;
    lcq::set_error("no CUDA device");
    return LCQMC_E_CUDA;
  }
  int rc = s->eng.open(nullptr, nullptr, kServerRing, /*serving=*/true);
  if (rc) {
    delete s;
    return rc;
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return LCQMC_OK;
}

int lcqmc_submit(lcqmc_server_t s, const lcqmc_request *req, uint64_t *ticket) {
  if (!s || !req || !ticket || req->n_updates <= 0) {
    lcq::set_error("bad request");
    return LCQMC_E_INVAL;
  }
  auto q = std::make_unique<Req>();
  int rc = lcq::validate_spec(req->L, req->S, req->J, req->beta, q->spec);
  if (rc) return rc;
  q->spec.seed = req->seed;
  q->r = *req;
  q->foot = lcq::Engine::state_bytes(q->spec, kServerRing) + lcq::Engine::scratch_bytes(q->spec);
  const double nvert = 0.8 * q->spec.Q * q->spec.Q * q->spec.J * q->spec.beta * (double)q->spec.L;
  if (nvert > 1.9e9) {
    lcq::set_error("request needs more than 2^31 graph vertices");
    return LCQMC_E_ID_OVERFLOW;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (q->foot > s->budget) {
    lcq::set_error("request footprint exceeds the server's HBM budget");
    return LCQMC_E_TOO_LARGE;
  }
  q->ticket = s->next_ticket++;
  q->t_submit = s->now();
  *ticket = q->ticket;
  s->pending.push_back(q.get());
  s->reqs.emplace(q->ticket, std::move(q));
  s->cv.notify_one();
  return LCQMC_OK;
}

int lcqmc_poll(lcqmc_server_t s, uint64_t ticket, lcqmc_result *out) {
  if (!s || !out) return LCQMC_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) {
    lcq::set_error("unknown ticket");
    return LCQMC_E_NOT_FOUND;
  }
  const Req &q = *it->second;
  std::memset(out, 0, sizeof(*out));
  out->status = q.status;
  out->t_submit = q.t_submit;
  out->t_admit = q.t_admit;
  out->t_done = q.t_done;
  if (q.status == LCQMC_OK) {
    out->obs = q.obs;
    out->vertices_edges = (int64_t)q.obs.sum[7];
  }
  return q.status == LCQMC_PENDING ? LCQMC_PENDING : LCQMC_OK;
}

int lcqmc_cancel(lcqmc_server_t s, uint64_t ticket) {
  if (!s) return LCQMC_E_INVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return LCQMC_E_NOT_FOUND;
  Req *q = it->second.get();
  if (q->status != LCQMC_PENDING) return LCQMC_OK;
  for (auto p = s->pending.begin(); p != s->pending.end(); ++p)
    if (*p == q) {
      s->pending.erase(p);
      q->status = LCQMC_E_CANCELLED;
      q->t_done = s->now();
      return LCQMC_OK;
    }
  q->cancel = true;
  return LCQMC_OK;
}

int lcqmc_server_destroy(lcqmc_server_t s) {
  if (!s) return LCQMC_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  s->eng.set_chains({});
  for (auto &kv : s->reqs)
    if (kv.second->st) s->eng.destroy_state(kv.second->st.get());
  delete s;
  return LCQMC_OK;
}

}  // extern "C"
