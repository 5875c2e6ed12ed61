// Serving loop: continuous batching of anneal requests on one GPU.
//
// Requests (a k-SAT formula or a QAP, a beta profile, a replica count and a seed) are queued
// by any host thread. One worker thread owns a private nmc context and repeats a tick:
//   1. admit queued requests while the number of active requests and the device memory they
//      will hold stay within the configured limits (instance, schedule and replica state are
//      then resident on the device until the request finishes);
//   2. advance every active request by one slice of sweeps in a single batched launch (k-SAT
//      words of all requests share the persistent kernel; the QAP launch shapes run beside it
//      on auxiliary streams), the slice being the smaller of about the same amount of work per
//      request (2^slice_log2 units) and the sweeps that fit kTickUs by the request's estimated
//      time per sweep, so that a small instance, whose sweeps are bound by the per-class latency
//      rather than by its work, does not stretch the tick for everyone;
//   3. read back and release the requests that reached the end of their schedule.
// A request that arrives while others run joins at the next tick. Because sweeps are
// segment-invariant (absolute sweep index in every random-number counter), a request's result
// does not depend on how its sweeps were sliced or on which requests shared its launches.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "nmc.h"
#include "nmc_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// Target GPU time of one tick's slice of a request (estimated, microseconds).
constexpr double kTickUs = 100000.0;

struct Request {
  int64_t id = 0;
  int kind = 0;
  int32_t n = 0, m = 0, kmax = 0, n_steps = 0, replicas = 0, n_colours = 0;
  uint64_t seed = 0;
  std::vector<int32_t> F, D;
  nmc::HostKsat prep;  // k-SAT instance prepared on the submitting thread
  std::vector<float> beta, base, factor;  // full profile, or the factored form
  // device residency
  int32_t inst = -1, rs = -1;
  int32_t t = 0;
  int64_t mem = 0;
  bool batchable = true;  // k-SAT sets the batched kernel accepts (degree <= 127, n fits)
  // results
  std::vector<uint8_t> states, best_states;
  std::vector<int64_t> energies, best_energies;
  int status = 0;  // 0 queued, 1 active, 2 done, <0 error code
  std::atomic<bool> cancelled{false};
  std::string error;
  Clock::time_point t_submit, t_admit, t_done;
};

}  // namespace

struct nmc_server {
  nmc_ctx *ctx = nullptr;
  nmc_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::vector<std::shared_ptr<Request>> active;
  std::map<int64_t, std::shared_ptr<Request>> all;
  int64_t next_id = 1;
  int64_t mem_in_use = 0;
  int32_t batch_max_vars = 0;
  bool stop = false;
  std::thread worker;
  // statistics
  int64_t ticks = 0, attempts = 0;
  double busy_s = 0.0;
  std::string err;
};

namespace {

int64_t estimate_bytes(const Request &r) {
  const int64_t words = (r.replicas + 31) / 32;
  if (r.kind == NMC_KIND_KSAT) {
    const int64_t occ = static_cast<int64_t>(r.m) * r.kmax;
    const int64_t instance = occ * 16 * 3 + static_cast<int64_t>(r.m) * r.kmax * 4 + r.n * 24;
    const int64_t sched = static_cast<int64_t>(r.n) * r.n_steps * 4;
    const int64_t reps = (4 * static_cast<int64_t>(r.n) + 2) * words * 4 + 64 * words * 4 + 8192;
    return instance + sched + reps + (1 << 20);
  }
  const int64_t n = r.n;
  return 2 * n * n + n * r.n_steps * 4 + r.replicas * (4 * n + 16) + (1 << 20);
}

void finish(nmc_server *s, const std::shared_ptr<Request> &r, int status, const std::string &msg) {
  if (r->rs >= 0) nmc_replicas_destroy(s->ctx, r->rs);
  if (r->inst >= 0) nmc_unload(s->ctx, r->inst);
  r->rs = r->inst = -1;
  std::lock_guard<std::mutex> g(s->mu);
  s->mem_in_use -= r->mem;
  r->mem = 0;
  r->status = status;
  r->error = msg;
  r->t_done = Clock::now();
  r->prep = nmc::HostKsat();
  r->beta.clear();
  r->beta.shrink_to_fit();
  r->base.clear();
  r->factor.clear();
  s->cv_done.notify_all();
}

bool admit(nmc_server *s, const std::shared_ptr<Request> &r) {
  nmc_ctx *c = s->ctx;
  int rc;
  if (r->kind == NMC_KIND_KSAT) {
    rc = nmc::upload_ksat(c, r->prep, &r->inst);
    r->prep = nmc::HostKsat();
  } else
    rc = nmc_load_qap(c, r->n, r->F.data(), r->D.data(), &r->inst);
  if (rc == NMC_OK)
    rc = r->beta.empty() ? nmc_set_schedule_factored(c, r->inst, r->n_steps, r->base.data(), r->factor.data())
                         : nmc_set_schedule(c, r->inst, r->n_steps, r->beta.data());
  if (rc == NMC_OK) rc = nmc_replicas_create(c, r->inst, r->replicas, r->seed, nullptr, &r->rs);
  if (rc != NMC_OK) {
    finish(s, r, rc, nmc_last_error(c));
    return false;
  }
  r->t_admit = Clock::now();
  std::lock_guard<std::mutex> g(s->mu);
  r->status = 1;
  return true;
}

void worker_loop(nmc_server *s) {
  const int64_t slice = int64_t(1) << s->cfg.slice_log2;
  while (true) {
    std::vector<std::shared_ptr<Request>> incoming;
    {
      std::unique_lock<std::mutex> g(s->mu);
      if (s->active.empty() && s->queue.empty() && !s->stop)
        s->cv_work.wait_for(g, std::chrono::milliseconds(50));
      if (s->stop) break;
      // admission: FIFO while slots and memory allow (a request larger than the whole budget
      // is rejected rather than blocking the queue)
      while (!s->queue.empty()) {
        auto r = s->queue.front();
        if (r->cancelled) {
          s->queue.pop_front();
          r->status = NMC_ESTATE;
          r->error = "cancelled before admission";
          r->t_done = Clock::now();
          s->cv_done.notify_all();
          continue;
        }
        if (r->mem > s->cfg.memory_budget) {
          s->queue.pop_front();
          r->status = NMC_ENOMEM;
          r->error = "request exceeds the server's device-memory budget";
          r->t_done = Clock::now();
          s->cv_done.notify_all();
          continue;
        }
        if (static_cast<int64_t>(s->active.size() + incoming.size()) >= s->cfg.max_active ||
            s->mem_in_use + r->mem > s->cfg.memory_budget)
          break;
        s->queue.pop_front();
        s->mem_in_use += r->mem;
        incoming.push_back(r);
      }
    }
    // the worker alone changes `active`, under the lock so that nmc_server_stats may read it
    for (auto &r : incoming)
      if (admit(s, r)) {
        std::lock_guard<std::mutex> g(s->mu);
        s->active.push_back(r);
      }
    if (s->active.empty()) continue;
    // one tick: equal-work slices, k-SAT in one batched launch, QAP after it
    const auto t0 = Clock::now();
    std::vector<int32_t> rs, a, b, qrs, qa, qb;
    int64_t tick_attempts = 0;
    int rc = NMC_OK;
    for (auto &r : s->active) {
      if (r->cancelled) continue;
      // work of one sweep / step in occurrence-word updates (one clause occurrence of one
      // variable for 32 replicas); a QAP swap attempt on one replica costs about n/3 of them
      const int64_t per_sweep =
          r->kind == NMC_KIND_KSAT
              ? static_cast<int64_t>(r->m) * r->kmax * ((r->replicas + 31) / 32)
              : static_cast<int64_t>(r->n) * r->n * r->replicas / 3;
      const double t_us = r->kind == NMC_KIND_KSAT ? nmc::ksat_sweep_us(r->n, r->n_colours)
                                                   : nmc::qap_step_us(r->n);
      const int64_t by_time = std::max<int64_t>(1, static_cast<int64_t>(kTickUs / t_us));
      const int64_t sweeps =
          std::min(by_time, std::max<int64_t>(1, slice / std::max<int64_t>(1, per_sweep)));
      const int32_t t1 = static_cast<int32_t>(std::min<int64_t>(r->n_steps, r->t + sweeps));
      if (r->kind == NMC_KIND_KSAT && r->batchable) {
        rs.push_back(r->rs);
        a.push_back(r->t);
        b.push_back(t1);
      } else if (r->kind == NMC_KIND_QAP) {
        qrs.push_back(r->rs);
        qa.push_back(r->t);
        qb.push_back(t1);
      } else if (rc == NMC_OK) {
        rc = nmc_replicas_run(s->ctx, r->rs, r->t, t1);
      }
      tick_attempts += static_cast<int64_t>(t1 - r->t) * r->n * r->replicas;
      r->t = t1;
    }
    // QAP shapes on their own streams first, then the k-SAT launch on the context's stream:
    // the two run side by side and are joined before the tick's synchronisation
    uint32_t qjoin = 0;
    if (rc == NMC_OK && !qrs.empty())
      rc = nmc::qap_batch_enqueue(s->ctx, static_cast<int32_t>(qrs.size()), qrs.data(), qa.data(),
                                  qb.data(), &qjoin);
    if (rc == NMC_OK && !rs.empty())
      rc = nmc_batch_run(s->ctx, static_cast<int32_t>(rs.size()), rs.data(), a.data(), b.data());
    const int rcj = nmc::qap_batch_join(s->ctx, qjoin);
    if (rc == NMC_OK) rc = rcj;
    if (rc == NMC_OK) rc = nmc_sync(s->ctx);
    const double dt = std::chrono::duration<double>(Clock::now() - t0).count();
    if (rc != NMC_OK) {
      const std::string msg = nmc_last_error(s->ctx);
      for (auto &r : s->active) finish(s, r, rc, msg);
      std::lock_guard<std::mutex> g(s->mu);
      s->active.clear();
      continue;
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      s->ticks++;
      s->attempts += tick_attempts;
      s->busy_s += dt;
    }
    // retire finished (or cancelled) requests
    std::vector<std::shared_ptr<Request>> keep;
    for (auto &r : s->active) {
      if (r->cancelled) {
        finish(s, r, NMC_ESTATE, "cancelled");
        continue;
      }
      if (r->t < r->n_steps) {
        keep.push_back(r);
        continue;
      }
      const size_t cnt = static_cast<size_t>(r->replicas) * r->n;
      const size_t elem = r->kind == NMC_KIND_KSAT ? 1 : 2;
      r->states.assign(cnt * elem, 0);
      r->best_states.assign(cnt * elem, 0);
      r->energies.assign(r->replicas, 0);
      r->best_energies.assign(r->replicas, 0);
      nmc_result out{r->states.data(), r->energies.data(), r->best_energies.data(),
                     r->best_states.data()};
      const int rr = nmc_replicas_read(s->ctx, r->rs, &out);
      finish(s, r, rr == NMC_OK ? 2 : rr, rr == NMC_OK ? "" : nmc_last_error(s->ctx));
    }
    std::lock_guard<std::mutex> g(s->mu);
    s->active.swap(keep);
  }
  for (auto &r : s->active) finish(s, r, NMC_ESTATE, "server stopped");
  std::lock_guard<std::mutex> g(s->mu);
  s->active.clear();
}

// t_arrive: when the submit call began, so that a request's latency includes the host-side
// build of its instance (checks, colouring, lists) as well as its queueing and device time.
int submit(nmc_server *s, std::shared_ptr<Request> r, Clock::time_point t_arrive,
           int64_t *id_out) {
  r->mem = estimate_bytes(*r);
  r->t_submit = t_arrive;
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stop) return NMC_ESTATE;
  r->id = s->next_id++;
  s->all[r->id] = r;
  s->queue.push_back(r);
  *id_out = r->id;
  s->cv_work.notify_one();
  return NMC_OK;
}

// Copies a schedule given in either form; false if it is malformed.
bool copy_schedule(Request &r, const nmc_schedule *sc, int32_t n_units) {
  if (!sc || sc->n_steps < 1) return false;
  r.n_steps = sc->n_steps;
  if (sc->beta) {
    r.beta.assign(sc->beta, sc->beta + static_cast<size_t>(n_units) * sc->n_steps);
    return true;
  }
  if (!sc->base || !sc->factor) return false;
  r.base.assign(sc->base, sc->base + sc->n_steps);
  r.factor.assign(sc->factor, sc->factor + n_units);
  return true;
}

}  // namespace

extern "C" {

int nmc_server_create(int device, const nmc_server_config *cfg, nmc_server **out) {
  if (!out || !cfg) return NMC_EINVAL;
  *out = nullptr;
  if (cfg->max_active < 1 || cfg->memory_budget < 1 || cfg->slice_log2 < 10 || cfg->slice_log2 > 40)
    return NMC_EINVAL;
  nmc_server *s = new nmc_server();
  s->cfg = *cfg;
  const int rc = nmc_create(&s->ctx, device, nullptr);
  if (rc != NMC_OK) {
    delete s;
    return rc;
  }
  s->batch_max_vars = nmc_batch_max_vars(s->ctx);
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return NMC_OK;
}

int nmc_server_submit_ksat(nmc_server *s, int32_t n_vars, int32_t n_clauses, int32_t k_max,
                           const int32_t *lits, const nmc_schedule *sched, int32_t replicas,
                           uint64_t seed, int64_t *req_out) {
  const auto t_arrive = Clock::now();
  if (!s || !req_out || n_vars < 1 || n_clauses < 0 || k_max < 1 || k_max > 8 ||
      (n_clauses > 0 && !lits) || replicas < 1 || replicas > 4096)
    return NMC_EINVAL;
  auto r = std::make_shared<Request>();
  r->kind = NMC_KIND_KSAT;
  r->n = n_vars;
  r->m = n_clauses;
  r->kmax = k_max;
  r->replicas = replicas;
  r->seed = seed;
  if (!copy_schedule(*r, sched, n_vars)) return NMC_EINVAL;
  // host-side build (checks, colouring, lists) here, on the caller's thread; a malformed
  // formula is reported by the request's status, as any admission failure
  nmc::prepare_ksat(n_vars, n_clauses, k_max, lits, &r->prep);
  r->n_colours = r->prep.n_colours;
  r->batchable = r->prep.code == NMC_OK && r->prep.nb <= 7 && n_vars <= s->batch_max_vars;
  return submit(s, r, t_arrive, req_out);
}

int nmc_server_submit_qap(nmc_server *s, int32_t n, const int32_t *F, const int32_t *D,
                          const nmc_schedule *sched, int32_t replicas, uint64_t seed,
                          int64_t *req_out) {
  const auto t_arrive = Clock::now();
  if (!s || !req_out || n < 1 || !F || !D || replicas < 1 || replicas > 4096) return NMC_EINVAL;
  auto r = std::make_shared<Request>();
  r->kind = NMC_KIND_QAP;
  r->n = n;
  r->replicas = replicas;
  r->seed = seed;
  if (!copy_schedule(*r, sched, n)) return NMC_EINVAL;
  r->F.assign(F, F + static_cast<size_t>(n) * n);
  r->D.assign(D, D + static_cast<size_t>(n) * n);
  return submit(s, r, t_arrive, req_out);
}

int nmc_server_poll(nmc_server *s, int64_t req, int32_t wait_ms, int32_t *status) {
  if (!s || !status) return NMC_EINVAL;
  std::unique_lock<std::mutex> g(s->mu);
  auto it = s->all.find(req);
  if (it == s->all.end()) return NMC_EINVAL;
  auto r = it->second;
  if (wait_ms > 0)
    s->cv_done.wait_for(g, std::chrono::milliseconds(wait_ms),
                        [&] { return r->status == 2 || r->status < 0; });
  *status = r->status;
  return NMC_OK;
}

int nmc_server_result(nmc_server *s, int64_t req, const nmc_result *out, double *latency_s) {
  if (!s) return NMC_EINVAL;
  std::shared_ptr<Request> r;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(req);
    if (it == s->all.end()) return NMC_EINVAL;
    r = it->second;
    if (r->status < 0) {
      s->err = r->error;
      s->all.erase(it);
      return r->status;
    }
    if (r->status != 2) return NMC_ESTATE;
    s->all.erase(it);
  }
  if (out) {
    if (out->states) std::memcpy(out->states, r->states.data(), r->states.size());
    if (out->best_states) std::memcpy(out->best_states, r->best_states.data(), r->best_states.size());
    if (out->energies) std::memcpy(out->energies, r->energies.data(), 8 * r->energies.size());
    if (out->best_energies)
      std::memcpy(out->best_energies, r->best_energies.data(), 8 * r->best_energies.size());
  }
  if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
  return NMC_OK;
}

int nmc_server_cancel(nmc_server *s, int64_t req) {
  if (!s) return NMC_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->all.find(req);
  if (it == s->all.end()) return NMC_EINVAL;
  it->second->cancelled = true;
  s->cv_work.notify_one();
  return NMC_OK;
}

int nmc_server_stats(nmc_server *s, int64_t *ticks, int64_t *attempts, double *busy_s,
                     int32_t *queued, int32_t *active, int64_t *mem_in_use) {
  if (!s) return NMC_EINVAL;
  std::lock_guard<std::mutex> g(s->mu);
  if (ticks) *ticks = s->ticks;
  if (attempts) *attempts = s->attempts;
  if (busy_s) *busy_s = s->busy_s;
  if (queued) *queued = static_cast<int32_t>(s->queue.size());
  if (active) *active = static_cast<int32_t>(s->active.size());
  if (mem_in_use) *mem_in_use = s->mem_in_use;
  return NMC_OK;
}

const char *nmc_server_last_error(nmc_server *s) { return s ? s->err.c_str() : "nmc: no server"; }

void nmc_server_destroy(nmc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (auto &r : s->queue) {
      r->status = NMC_ESTATE;
      r->error = "server stopped";
    }
    s->queue.clear();
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->worker.joinable()) s->worker.join();
  nmc_destroy(s->ctx);
  delete s;
}

}  // extern "C"
