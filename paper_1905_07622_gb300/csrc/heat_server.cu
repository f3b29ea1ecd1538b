// The request server (include/heat.h, "serving"): a worker thread that admits
// transient simulations by device footprint as they arrive and advances every
// admitted one together through the tick engine (continuous batching).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

using namespace heat;
using Clock = std::chrono::steady_clock;

namespace {

enum ReqState { RQ_PENDING = 0, RQ_ACTIVE = 1, RQ_DONE = 2 };

struct Req {
  uint64_t ticket = 0;
  heat_request r{};
  std::vector<double> rho_c, k, u0;
  long long nn = 0, ne = 0;
  size_t footprint = 0;
  Clock::time_point t_submit, t_done;
  int state = RQ_PENDING;
  heat_status status = HEAT_OK;
  std::string error;
  heat_mesh* mesh = nullptr;
  heat_sim* sim = nullptr;
  std::vector<double> result;
  heat_step_stats stats{};
};

}  // namespace

struct heat_server {
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> active;  // worker-owned while admitted
  std::unordered_map<uint64_t, Req*> all;
  size_t budget = 0, used = 0;
  int max_active = 1;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  bool stop = false;
  uint64_t next_ticket = 1;
  heat_server_stats st{};
  std::thread worker;
};

static void release(Req* q) {
  if (q->sim) heat_destroy_sim(q->sim);
  if (q->mesh) heat_destroy_mesh(q->mesh);
  q->sim = nullptr;
  q->mesh = nullptr;
}

// Builds a request's simulation on the worker's stream.
static heat_status start_request(heat_server* srv, Req* q) {
  heat_status s = heat_create_mesh(q->r.nx, q->r.ny, q->r.nz, q->r.origin, q->r.extent, &q->mesh);
  if (s == HEAT_OK) s = heat_sim_create(q->mesh, &q->r.bc, &q->r.params, srv->stream, &q->sim);
  if (s == HEAT_OK) s = heat_set_coeffs(q->sim, q->rho_c.data(), q->k.data(), 0);
  if (s == HEAT_OK && !q->u0.empty()) s = heat_set_state(q->sim, q->u0.data(), 0);
  if (s == HEAT_OK) s = sim_prepare_steps(q->sim, q->r.nsteps);
  if (s != HEAT_OK) {
    q->error = heat_last_error();
    release(q);
  }
  return s;
}

static void finish_request(heat_server* srv, Req* q, heat_status status) {
  if (status == HEAT_OK && q->sim) {
    q->result.resize((size_t)q->nn);
    status = heat_get_state(q->sim, q->result.data(), 0);
    if (status == HEAT_OK) {
      sim_stats(q->sim, &q->stats);
      if (q->stats.status != HEAT_OK) status = (heat_status)q->stats.status;
    }
    if (status != HEAT_OK) q->error = heat_last_error();
  }
  release(q);
  std::lock_guard<std::mutex> lock(srv->mu);
  q->status = status;
  q->state = RQ_DONE;
  q->t_done = Clock::now();
  srv->used -= q->footprint;
  if (status == HEAT_OK) {
    srv->st.completed += 1;
    srv->st.dof_cg_iters += (double)q->nn * (double)q->stats.iters;
  } else {
    srv->st.failed += 1;
  }
  srv->cv_done.notify_all();
}

// Ticks launched between two reads of the members' phases (and admissions):
// about 30 CG iterations at six per tick. Longer rounds keep a finished
// request's slot idle for longer before the next admission takes it.
constexpr int kTicksPerPoll = 5;
// Work-list and descriptor capacity of a server engine relative to the member
// set it is built for: later sets that fit run under the same captured graph.
constexpr double kEngineHeadroom = 2.0;

static void worker_loop(heat_server* srv) {
  cudaSetDevice(srv->device);
  if (!srv->stream) {
    cudaStreamCreateWithFlags(&srv->stream, cudaStreamNonBlocking);
    srv->own_stream = true;
  }
  Engine* eng = nullptr;
  long long launches_done = 0;  // of engines already destroyed
  std::vector<int> phases;
  bool members_changed = false;
  auto active_sims = [&]() {
    std::vector<heat_sim*> sims;
    for (Req* q : srv->active) sims.push_back(q->sim);
    return sims;
  };
  // Runs the current active set: the engine takes the new members in place
  // when they fit its capacities, else a new engine is built.
  auto rebuild = [&]() -> heat_status {
    const std::vector<heat_sim*> sims = active_sims();
    heat_status s = eng ? engine_set_members(eng, sims.data(), (int)sims.size()) : HEAT_ERR_ARG;
    // a new engine only when the set outgrew this one's capacities; any other
    // failure means the set cannot run
    if (s == HEAT_OK || (eng && s != HEAT_ERR_ARG)) return s;
    if (eng) {
      launches_done += engine_launches(eng);
      engine_destroy(eng);
      eng = nullptr;
    }
    return engine_create(sims.data(), (int)sims.size(), srv->active[0]->r.params.precision, srv->stream, &eng,
                         nullptr, kEngineHeadroom);
  };
  for (;;) {
    // admission: arrival order, first fit by footprint and free slots
    std::vector<Req*> admit;
    {
      std::unique_lock<std::mutex> lock(srv->mu);
      if (srv->stop) break;
      if (srv->active.empty() && srv->pending.empty()) {
        srv->cv_work.wait_for(lock, std::chrono::milliseconds(50));
        continue;
      }
      // one engine runs one precision and one element type: a request of
      // another waits until the running set has drained
      int prec = srv->active.empty() ? -1 : srv->active[0]->r.params.precision;
      int elem = srv->active.empty() ? -1 : srv->active[0]->r.params.element;
      for (auto it = srv->pending.begin(); it != srv->pending.end();) {
        Req* q = *it;
        if (prec < 0) {
          prec = q->r.params.precision;
          elem = q->r.params.element;
        }
        if (q->r.params.precision == prec && q->r.params.element == elem &&
            (int)(srv->active.size() + admit.size()) < srv->max_active &&
            srv->used + q->footprint <= srv->budget) {
          srv->used += q->footprint;
          q->state = RQ_ACTIVE;
          admit.push_back(q);
          it = srv->pending.erase(it);
        } else {
          ++it;
        }
      }
    }
    std::vector<Req*> added;
    for (Req* q : admit) {
      const heat_status s = start_request(srv, q);
      if (s == HEAT_OK) {
        std::lock_guard<std::mutex> lock(srv->mu);  // `active` is written by this thread only, read under the lock
        srv->active.push_back(q);
        added.push_back(q);
        members_changed = true;
      } else {
        finish_request(srv, q, s);
      }
    }
    if (srv->active.empty()) continue;
    if (members_changed || !eng) {
      heat_status s = rebuild();
      if (s != HEAT_OK && !added.empty()) {
        // the new set cannot run: refuse this round's admissions and keep
        // the requests that were already running
        const std::string why = heat_last_error();
        {
          std::lock_guard<std::mutex> lock(srv->mu);
          std::vector<Req*> keep;
          for (Req* q : srv->active)
            if (std::find(added.begin(), added.end(), q) == added.end()) keep.push_back(q);
          srv->active.swap(keep);
        }
        for (Req* q : added) {
          q->error = "admission refused: " + why;
          finish_request(srv, q, s);
        }
        s = srv->active.empty() ? HEAT_OK : rebuild();
      }
      if (s != HEAT_OK) {  // not even the running set can be run: fail it
        std::vector<Req*> failed;
        {
          std::lock_guard<std::mutex> lock(srv->mu);
          failed.swap(srv->active);
        }
        for (Req* q : failed) {
          q->error = heat_last_error();
          finish_request(srv, q, s);
        }
        if (eng) {
          launches_done += engine_launches(eng);
          engine_destroy(eng);
          eng = nullptr;
        }
        members_changed = false;
        continue;
      }
      members_changed = false;
      if (srv->active.empty()) continue;
    }
    heat_status s = engine_launch_ticks(eng, kTicksPerPoll);
    phases.assign(srv->active.size(), 0);
    if (s == HEAT_OK) s = engine_read_phases(eng, phases.data());
    std::vector<Req*> keep;
    for (size_t i = 0; i < srv->active.size(); ++i) {
      Req* q = srv->active[i];
      if (s != HEAT_OK) {
        q->error = heat_last_error();
        finish_request(srv, q, s);
        members_changed = true;
      } else if (phases[i] == PH_DONE || phases[i] == PH_FAILED) {
        heat_status rs = sim_read_scalars(q->sim);
        finish_request(srv, q, rs);
        members_changed = true;
      } else {
        keep.push_back(q);
      }
    }
    {
      std::lock_guard<std::mutex> lock(srv->mu);
      srv->active.swap(keep);
      srv->st.kernel_launches = launches_done + (eng ? engine_launches(eng) : 0);
    }
  }
  if (eng) engine_destroy(eng);
  std::vector<Req*> left;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    left.swap(srv->active);
  }
  for (Req* q : left) {
    q->error = "server stopped";
    finish_request(srv, q, HEAT_ERR_BUSY);
  }
  if (srv->own_stream) cudaStreamDestroy(srv->stream);
}

extern "C" heat_status heat_server_create(size_t hbm_budget_bytes, int max_active, void* cuda_stream,
                                          heat_server** out) {
  if (!out) return set_error(HEAT_ERR_ARG, "heat_server_create: out is NULL");
  *out = nullptr;
  if (hbm_budget_bytes == 0 || max_active < 1)
    return set_error(HEAT_ERR_ARG, "heat_server_create: need a budget > 0 and max_active >= 1");
  heat_server* srv = new heat_server();
  srv->budget = hbm_budget_bytes;
  srv->max_active = max_active;
  srv->stream = (cudaStream_t)cuda_stream;
  srv->st.hbm_budget = hbm_budget_bytes;
  if (cudaGetDevice(&srv->device) != cudaSuccess) {
    cudaGetLastError();
    delete srv;
    return set_error(HEAT_ERR_CUDA, "heat_server_create: no CUDA device");
  }
  srv->worker = std::thread(worker_loop, srv);
  *out = srv;
  return HEAT_OK;
}

extern "C" heat_status heat_submit(heat_server* srv, const heat_request* req, uint64_t* ticket) {
  if (!srv || !req || !ticket) return set_error(HEAT_ERR_ARG, "heat_submit: null argument");
  if (req->nx < 1 || req->ny < 1 || req->nz < 1 || req->nsteps < 1 || !req->rho_c || !req->k)
    return set_error(HEAT_ERR_ARG, "heat_submit: bad mesh, step count or coefficient pointer");
  if (req->params.precision != HEAT_FP64 && req->params.precision != HEAT_FP32_REFINED &&
      req->params.precision != HEAT_FP32_PLAIN)
    return set_error(HEAT_ERR_ARG, "heat_submit: bad precision");
  Req* q = new Req();
  q->r = *req;
  q->nn = (long long)(req->nx + 1) * (req->ny + 1) * (req->nz + 1);
  q->ne = (long long)req->nx * req->ny * req->nz;
  if (q->nn >= (1LL << 31) - 1) {
    delete q;
    return set_error(HEAT_ERR_ARG, "heat_submit: mesh too large");
  }
  for (long long e = 0; e < q->ne; ++e) {
    if (!std::isfinite(req->rho_c[e]) || !std::isfinite(req->k[e]) || !(req->rho_c[e] > 0.0) || !(req->k[e] > 0.0)) {
      delete q;
      return set_error(HEAT_ERR_NONFINITE, "heat_submit: coefficient %lld is non-finite or not > 0", e);
    }
  }
  q->rho_c.assign(req->rho_c, req->rho_c + q->ne);
  q->k.assign(req->k, req->k + q->ne);
  if (req->u0) q->u0.assign(req->u0, req->u0 + q->nn);
  q->r.rho_c = q->r.k = q->r.u0 = nullptr;
  // the server's engines hold kEngineHeadroom times each member's work lists
  q->footprint = sim_footprint(q->nn, q->ne) +
                 (size_t)(kEngineHeadroom * (double)engine_footprint(q->nn, req->nx, req->ny, req->nz));
  std::lock_guard<std::mutex> lock(srv->mu);
  if (q->footprint > srv->budget) {
    delete q;
    return set_error(HEAT_ERR_NOMEM, "heat_submit: request needs %zu bytes, the budget is %zu", q->footprint,
                     srv->budget);
  }
  q->ticket = srv->next_ticket++;
  q->t_submit = Clock::now();
  srv->all[q->ticket] = q;
  srv->pending.push_back(q);
  srv->st.submitted += 1;
  *ticket = q->ticket;
  srv->cv_work.notify_one();
  return HEAT_OK;
}

extern "C" heat_status heat_poll(heat_server* srv, uint64_t ticket, int* done) {
  if (!srv || !done) return set_error(HEAT_ERR_ARG, "heat_poll: null argument");
  std::lock_guard<std::mutex> lock(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return set_error(HEAT_ERR_ARG, "heat_poll: unknown ticket %llu", (unsigned long long)ticket);
  *done = it->second->state == RQ_DONE ? 1 : 0;
  return HEAT_OK;
}

extern "C" heat_status heat_wait(heat_server* srv, uint64_t ticket, double timeout_s, double* u_out,
                                 heat_step_stats* stats, double* latency_s) {
  if (!srv) return set_error(HEAT_ERR_ARG, "heat_wait: server is NULL");
  std::unique_lock<std::mutex> lock(srv->mu);
  auto it = srv->all.find(ticket);
  if (it == srv->all.end()) return set_error(HEAT_ERR_ARG, "heat_wait: unknown ticket %llu", (unsigned long long)ticket);
  Req* q = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(std::max(0.0, timeout_s)));
  while (q->state != RQ_DONE) {
    if (srv->cv_done.wait_until(lock, deadline) == std::cv_status::timeout && q->state != RQ_DONE)
      return set_error(HEAT_ERR_TIMEOUT, "heat_wait: ticket %llu not finished after %g s", (unsigned long long)ticket,
                       timeout_s);
  }
  if (u_out && q->status == HEAT_OK) std::memcpy(u_out, q->result.data(), sizeof(double) * q->result.size());
  if (stats) *stats = q->stats;
  if (latency_s) *latency_s = std::chrono::duration<double>(q->t_done - q->t_submit).count();
  const heat_status st = q->status;
  const std::string err = q->error;
  srv->all.erase(it);
  delete q;
  if (st != HEAT_OK) return set_error(st, "request failed: %s", err.c_str());
  return HEAT_OK;
}

extern "C" heat_status heat_server_get_stats(heat_server* srv, heat_server_stats* out) {
  if (!srv || !out) return set_error(HEAT_ERR_ARG, "heat_server_get_stats: null argument");
  std::lock_guard<std::mutex> lock(srv->mu);
  *out = srv->st;
  out->active = (int)srv->active.size();
  out->pending = (int)srv->pending.size();
  out->hbm_in_use = srv->used;
  return HEAT_OK;
}

extern "C" void heat_destroy_server(heat_server* srv) {
  if (!srv) return;
  {
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  if (srv->worker.joinable()) srv->worker.join();
  for (auto& kv : srv->all) {
    release(kv.second);
    delete kv.second;
  }
  delete srv;
}
