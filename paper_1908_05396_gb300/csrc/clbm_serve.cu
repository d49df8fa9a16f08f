// clbm_serve.cu -- continuous-batching solve server (include/clbm.h).
//
// A worker thread owns one batch (clbm_batch) and loops:
//   1. admit queued requests, first come first served, while a slot is free
//      and the request's device memory fits in what is left of the budget;
//   2. step every admitted lattice by one check interval (one graph launch);
//   3. read each lattice's residual, divergence flag and step count, and
//      retire the ones that converged (residual <= tol), diverged, reached
//      their step cap, or stopped improving (plateau), freeing their memory.
// Requests submitted while others run join at the next interval boundary.
// Because lattices join only at interval boundaries and the batch kernel
// treats every lattice independently, a request's steps, checks and result
// do not depend on what else is being solved.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/clbm.h"
#include "ctx.h"
#include "launch.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Pending {
  int64_t id;
  clbm_request req;
  double t_submit;
};

struct Active {
  int64_t id;
  clbm_request req;
  clbm_handle h = nullptr;
  int slot = -1;
  size_t bytes = 0;
  double t_submit = 0, t_admit = 0;
  double best = INFINITY;
  int since_best = 0;
};

struct Done {
  clbm_result res;
  std::vector<double> rho, u, gd;
};

}  // namespace

struct clbm_server_ctx {
  clbm_dtype dtype = CLBM_F16S;
  bool sround = false;              // F16S: lattices round their stores stochastically
  double budget = 0;
  int max_active = 0;
  int check_interval = 100;
  int device = 0;
  clbm_batch batch = nullptr;
  Clock::time_point t0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;       // new work or stop
  std::condition_variable done_cv;  // a request finished
  std::deque<Pending> queue;
  std::vector<Active> active;
  std::map<int64_t, Done> done;
  double used = 0;
  bool stop = false;
  int64_t next_id = 1;
  int64_t lups = 0;                 // lattice-node updates done
  double busy = 0;                  // seconds with at least one lattice active
  // per-slot check results of the batch (max_active entries)
  std::vector<double> st_R, st_mass;
  std::vector<int> st_div;
  std::vector<int64_t> st_steps;
  std::string err;
};

namespace {

double now(const clbm_server_ctx* s) {
  return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

int sfail(clbm_server_ctx* s, int code, const std::string& m) {
  if (s) s->err = m;
  clbm::set_unbound_error(m.c_str());
  return code;
}

// Device bytes of one lattice of this form (two population buffers, the
// check velocities, the F16R reference moments, small work buffers), with the
// library's padding.
double lattice_bytes(clbm_dtype t, const clbm_domain& d) {
  const int64_t elem = t == CLBM_F64 ? 8 : t == CLBM_F32 ? 4 : 2;
  const int64_t rs = t == CLBM_F64 ? 8 : 4;
  const int64_t per_row = 128 / elem;
  const int64_t pitch = (d.nx + per_row - 1) / per_row * per_row;
  const int64_t plane = pitch * d.ny;
  const int64_t qs = (plane * d.nz + 255) / 256 * 256;
  const int64_t refs = t == CLBM_F16R ? int64_t(2 * clbm::f16r_ref_bytes(plane * d.nz)) : 0;
  return double(2 * 19 * qs * elem + 3 * plane * d.nz * rs + refs + 4096);
}

void finish(clbm_server_ctx* s, Active& a, int status, double R, double mass, int64_t steps) {
  Done d;
  std::memset(&d.res, 0, sizeof(d.res));
  d.res.id = a.id;
  d.res.status = status;
  d.res.steps = steps;
  d.res.residual = R;
  d.res.mass = mass;
  d.res.t_submit = a.t_submit;
  d.res.t_admit = a.t_admit;
  d.res.N = int64_t(a.req.dom.nx) * a.req.dom.ny * a.req.dom.nz;
  if (a.req.keep_fields && a.h && status != CLBM_SOLVE_ERROR) {
    const size_t N = size_t(d.res.N);
    d.rho.resize(N);
    d.u.resize(3 * N);
    d.gd.resize(N);
    if (clbm_fields(a.h, d.rho.data(), d.u.data(), d.gd.data()) != CLBM_OK) {
      d.res.status = CLBM_SOLVE_ERROR;
      d.rho.clear();
      d.u.clear();
      d.gd.clear();
    }
  }
  if (a.h) clbm_destroy(a.h);  // leaves the batch, frees its memory
  a.h = nullptr;
  d.res.t_done = now(s);
  s->used -= double(a.bytes);
  s->done[a.id] = std::move(d);
}

void worker_loop(clbm_server_ctx* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    // 1. admission, first come first served
    while (!s->queue.empty() && int(s->active.size()) < s->max_active) {
      Pending& p = s->queue.front();
      const double need = lattice_bytes(s->dtype, p.req.dom);
      if (s->used + need > s->budget) {
        if (s->active.empty()) {  // can never fit: reject rather than wait forever
          Active a;
          a.id = p.id;
          a.req = p.req;
          a.t_submit = p.t_submit;
          a.t_admit = now(s);
          a.bytes = 0;
          finish(s, a, CLBM_SOLVE_REJECTED, INFINITY, 0.0, 0);
          s->queue.pop_front();
          s->done_cv.notify_all();
          continue;
        }
        break;
      }
      Active a;
      a.id = p.id;
      a.req = p.req;
      a.t_submit = p.t_submit;
      a.bytes = size_t(need);
      clbm_domain dom = p.req.dom;
      dom.check_interval = s->check_interval;
      dom.stream = nullptr;
      dom.in_place = 0;   // the batched step works on two buffers
      int rc = clbm_create(&dom, p.req.K, p.req.n, p.req.U_lid, p.req.body_force, s->dtype, &a.h);
      if (rc == CLBM_OK && s->sround) rc = clbm_set_rounding(a.h, CLBM_ROUND_STOCHASTIC);
      if (rc == CLBM_OK) rc = clbm_batch_add(s->batch, a.h, &a.slot);
      a.t_admit = now(s);
      s->queue.pop_front();
      if (rc != CLBM_OK) {
        a.bytes = 0;
        finish(s, a, CLBM_SOLVE_ERROR, INFINITY, 0.0, 0);
        s->done_cv.notify_all();
        continue;
      }
      s->used += need;
      s->active.push_back(a);
    }
    if (s->active.empty()) {
      s->cv.wait(lk, [s] { return s->stop || !s->queue.empty(); });
      continue;
    }
    // 2. one check interval for every admitted lattice, outside the lock
    int64_t nodes = 0;
    for (const Active& a : s->active) nodes += int64_t(a.req.dom.nx) * a.req.dom.ny * a.req.dom.nz;
    lk.unlock();
    const double t_step = now(s);
    int rc = clbm_batch_step(s->batch, s->check_interval);
    if (rc == CLBM_OK) rc = clbm_batch_sync(s->batch);
    lk.lock();
    s->busy += now(s) - t_step;
    if (rc != CLBM_OK) {
      s->err = std::string("batch step failed: ") + clbm_batch_last_error(s->batch);
      for (Active& a : s->active) finish(s, a, CLBM_SOLVE_ERROR, INFINITY, 0.0, 0);
      s->active.clear();
      s->done_cv.notify_all();
      s->stop = true;
      break;
    }
    s->lups += nodes * s->check_interval;
    // 3. retirement, from every slot's check results (one synchronisation)
    const bool stats_ok = clbm_batch_stats_all(s->batch, s->st_R.data(), s->st_mass.data(),
                                               s->st_div.data(), s->st_steps.data()) == CLBM_OK;
    std::vector<Active> keep;
    for (Active& a : s->active) {
      if (!stats_ok) {
        finish(s, a, CLBM_SOLVE_ERROR, INFINITY, 0.0, 0);
        continue;
      }
      const double R = s->st_R[size_t(a.slot)], mass = s->st_mass[size_t(a.slot)];
      const int div = s->st_div[size_t(a.slot)];
      const int64_t steps = s->st_steps[size_t(a.slot)];
      if (div) {
        finish(s, a, CLBM_SOLVE_DIVERGED, R, mass, steps);
      } else if (R <= a.req.tol) {
        finish(s, a, CLBM_SOLVE_CONVERGED, R, mass, steps);
      } else if (a.req.max_steps > 0 && steps >= a.req.max_steps) {
        finish(s, a, CLBM_SOLVE_MAX_STEPS, R, mass, steps);
      } else {
        if (R < 0.9 * a.best) {
          a.best = R;
          a.since_best = 0;
        } else if (std::isfinite(R)) {
          a.since_best += 1;
        }
        if (a.req.plateau_checks > 0 && a.since_best >= a.req.plateau_checks)
          finish(s, a, CLBM_SOLVE_PLATEAU, R, mass, steps);
        else
          keep.push_back(a);
      }
    }
    const bool any_done = keep.size() != s->active.size();
    s->active.swap(keep);
    if (any_done) s->done_cv.notify_all();
  }
  // stopping: cancel what is left
  for (Active& a : s->active) finish(s, a, CLBM_SOLVE_CANCELLED, INFINITY, 0.0, 0);
  s->active.clear();
  for (Pending& p : s->queue) {
    Active a;
    a.id = p.id;
    a.req = p.req;
    a.t_submit = p.t_submit;
    finish(s, a, CLBM_SOLVE_CANCELLED, INFINITY, 0.0, 0);
  }
  s->queue.clear();
  s->done_cv.notify_all();
}

bool valid(const clbm_server_ctx* s) { return s && s->batch; }

}  // namespace

extern "C" {

int clbm_server_create(clbm_dtype dtype, double hbm_budget_bytes, int max_active,
                       int check_interval, clbm_server* out) {
  if (!out) return sfail(nullptr, CLBM_ERR_ARG, "null output");
  *out = nullptr;
  if (!(hbm_budget_bytes > 0)) return sfail(nullptr, CLBM_ERR_ARG, "budget must be > 0");
  if (max_active < 1 || max_active > 65536) return sfail(nullptr, CLBM_ERR_ARG, "max_active must be in [1, 65536]");
  if (check_interval <= 0) check_interval = 100;
  if (check_interval % 2) return sfail(nullptr, CLBM_ERR_ARG, "check_interval must be even");
  clbm_server_ctx* s = new (std::nothrow) clbm_server_ctx();
  if (!s) return sfail(nullptr, CLBM_ERR_OOM, "host allocation failed");
  s->dtype = dtype;
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->st_R.assign(size_t(max_active), 0.0);
  s->st_mass.assign(size_t(max_active), 0.0);
  s->st_div.assign(size_t(max_active), 0);
  s->st_steps.assign(size_t(max_active), 0);
  s->check_interval = check_interval;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  int rc = clbm_batch_create(dtype, max_active, check_interval, nullptr, &s->batch);
  if (rc != CLBM_OK) {
    delete s;
    return rc;
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return CLBM_OK;
}

int clbm_server_submit(clbm_server s, const clbm_request* req, int64_t* id) {
  if (!valid(s) || !req) return sfail(s, CLBM_ERR_ARG, "invalid server or request");
  if (!(req->tol >= 0.0)) return sfail(s, CLBM_ERR_ARG, "tol must be >= 0");
  const double t = now(s);  // arrival time, before any wait for the lock
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return sfail(s, CLBM_ERR_ARG, "server is stopped");
    Pending p;
    p.id = s->next_id++;
    p.req = *req;
    p.t_submit = t;
    s->queue.push_back(p);
    if (id) *id = p.id;
  }
  s->cv.notify_all();
  return CLBM_OK;
}

int clbm_server_wait(clbm_server s, int64_t id, double timeout_s, clbm_result* out) {
  if (!valid(s)) return sfail(s, CLBM_ERR_ARG, "invalid server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [s, id] { return s->done.count(id) != 0; };
  if (timeout_s < 0) {
    s->done_cv.wait(lk, ready);
  } else if (!s->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return sfail(s, CLBM_ERR_TIMEOUT, "request not finished within the timeout");
  }
  if (out) *out = s->done[id].res;
  return CLBM_OK;
}

int clbm_server_results(clbm_server s, clbm_result* out, int max, int* n) {
  if (!valid(s) || !n) return sfail(s, CLBM_ERR_ARG, "invalid server or output");
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  for (auto& kv : s->done) {
    if (k >= max) break;
    if (out) out[k] = kv.second.res;
    ++k;
  }
  *n = k;
  return CLBM_OK;
}

int clbm_server_fields(clbm_server s, int64_t id, double* rho, double* u, double* gamma_dot) {
  if (!valid(s)) return sfail(s, CLBM_ERR_ARG, "invalid server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(id);
  if (it == s->done.end()) return sfail(s, CLBM_ERR_ARG, "unknown or unfinished request");
  const Done& d = it->second;
  if (d.rho.empty()) return sfail(s, CLBM_ERR_ARG, "request was not submitted with keep_fields");
  if (rho) std::memcpy(rho, d.rho.data(), d.rho.size() * sizeof(double));
  if (u) std::memcpy(u, d.u.data(), d.u.size() * sizeof(double));
  if (gamma_dot) std::memcpy(gamma_dot, d.gd.data(), d.gd.size() * sizeof(double));
  return CLBM_OK;
}

int clbm_server_release(clbm_server s, int64_t id) {
  if (!valid(s)) return sfail(s, CLBM_ERR_ARG, "invalid server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->done.erase(id)) return sfail(s, CLBM_ERR_ARG, "unknown or unfinished request");
  return CLBM_OK;
}

int clbm_server_set_rounding(clbm_server s, clbm_rounding mode) {
  if (!valid(s)) return sfail(s, CLBM_ERR_ARG, "invalid server");
  if (mode != CLBM_ROUND_NEAREST && mode != CLBM_ROUND_STOCHASTIC)
    return sfail(s, CLBM_ERR_ARG, "unknown rounding mode");
  const bool sr = mode == CLBM_ROUND_STOCHASTIC;
  if (s->dtype == CLBM_F16R && !sr)
    return sfail(s, CLBM_ERR_UNSUPPORTED, "the F16R form always rounds stochastically");
  if (s->dtype != CLBM_F16R && s->dtype != CLBM_F16S && sr)
    return sfail(s, CLBM_ERR_UNSUPPORTED, "stochastic rounding is an F16S option");
  std::lock_guard<std::mutex> lk(s->mu);
  s->sround = sr && s->dtype == CLBM_F16S;
  return CLBM_OK;
}

int clbm_server_info(clbm_server s, clbm_server_stats* out) {
  if (!valid(s) || !out) return sfail(s, CLBM_ERR_ARG, "invalid server or output");
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = int64_t(s->queue.size());
  out->active = int64_t(s->active.size());
  out->done = int64_t(s->done.size());
  out->used_bytes = s->used;
  out->lattice_updates = double(s->lups);
  out->busy_seconds = s->busy;
  out->clock = now(s);
  return CLBM_OK;
}

int clbm_server_destroy(clbm_server s) {
  if (!s) return CLBM_OK;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  if (s->batch) clbm_batch_destroy(s->batch);
  delete s;
  return CLBM_OK;
}

const char* clbm_server_last_error(clbm_server s) { return s ? s->err.c_str() : ""; }

}  // extern "C"
