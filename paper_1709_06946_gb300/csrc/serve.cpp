// Serving loop: requests (mobility product, Brownian sample, constrained step)
// for suspensions of any size arrive at any time; a fixed number of worker
// slots, each with its own CUDA stream, run them concurrently on the device.
// A request is admitted as soon as a slot is free and its suspension's state
// fits the device-memory budget: a resident handle with the same parameters is
// reused (tables, plans, grids and neighbour lists stay on the device between
// requests), otherwise a new handle is created if its estimated footprint fits,
// after evicting idle resident handles (least recently used first).  Requests
// that do not fit yet wait in arrival order while later ones that fit go ahead.
// The paper has no serving layer; this is the request loop around its method.
#include <algorithm>
#include <array>
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

#include <cuda_runtime.h>

#include "../../include/pse.h"

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// The options a handle is created with, as numbers (a request without options
// has the defaults), so that requests that differ in them get their own handles.
using OptVec = std::array<double, 32>;
OptVec opt_vec(const pse_options *q) {
  pse_options o;
  pse_default_options(&o);
  if (q) o = *q;
  OptVec v{};
  int n = 0;
  for (double x : {(double)o.rule, (double)o.Ng, (double)o.P, (double)o.table_points, o.rcut, o.lanczos_tol,
                   (double)o.lanczos_maxiter, o.krylov_tol, (double)o.krylov_maxiter, (double)o.tile[0],
                   (double)o.tile[1], (double)o.tile[2], (double)o.real_lanes, (double)o.grid_ladder,
                   (double)o.use_graph, (double)o.wave_kernel, (double)o.torque, (double)o.lambda_support})
    v[n++] = x;
  for (int i = 0; i < 9; ++i) v[n++] = o.deform[i];
  return v;
}

struct Key {
  int64_t N;
  double L, a, eta, kT, xi, tol;
  int prec;
  OptVec opt;
  bool operator<(const Key &o) const {
    return std::tie(N, L, a, eta, kT, xi, tol, prec, opt) <
           std::tie(o.N, o.L, o.a, o.eta, o.kT, o.xi, o.tol, o.prec, o.opt);
  }
  bool operator==(const Key &o) const { return !(*this < o) && !(o < *this); }
};

struct Resident {
  Key key;
  pse_handle h = nullptr;
  int64_t bytes = 0;      // estimate reserved against the budget
  bool busy = false;
  uint64_t last_use = 0;
};

struct Job {
  uint64_t id = 0;
  pse_request req;
  Key key;
  int64_t est = 0;
  Clock::time_point t_submit, t_start, t_end;
  pse_status status = PSE_OK;
  bool done = false;
};

Key key_of(const pse_request &r) {
  return Key{r.N, r.L, r.a, r.eta, r.kT, r.xi, r.tol, r.precision, opt_vec(r.options)};
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  double x = q * (double)(v.size() - 1);
  size_t i = (size_t)x;
  double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct pse_server {
  int slots = 1;
  int64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job *> queue;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<std::unique_ptr<Resident>> residents;
  int64_t resident_bytes = 0, peak_bytes = 0;
  std::vector<std::thread> workers;
  bool stop = false;
  uint64_t next_id = 1, use_clock = 0;
  int running = 0, peak_running = 0;
  std::vector<double> latency, wait, service;
  Clock::time_point t_first, t_last;
  bool any_done = false, first_set = false;
  int64_t created = 0, evicted = 0, reused = 0, rejected = 0;
  std::string err;

  // Under mu: finds the resident handle for job j, or reserves memory for a new
  // one (evicting idle handles); returns false if j cannot start now.
  bool admit(Job *j, Resident **out, std::vector<pse_handle> &to_destroy) {
    for (auto &r : residents)
      if (!r->busy && r->key == j->key) {
        r->busy = true;
        r->last_use = ++use_clock;
        *out = r.get();
        ++reused;
        return true;
      }
    int64_t idle = 0;
    for (auto &r : residents)
      if (!r->busy && r->h) idle += r->bytes;
    if (resident_bytes - idle + j->est > budget) return false;  // cannot fit even after evictions
    while (resident_bytes + j->est > budget) {
      Resident *lru = nullptr;
      for (auto &r : residents)
        if (!r->busy && r->h && (!lru || r->last_use < lru->last_use)) lru = r.get();
      if (!lru) return false;
      to_destroy.push_back(lru->h);
      resident_bytes -= lru->bytes;
      ++evicted;
      residents.erase(std::find_if(residents.begin(), residents.end(),
                                   [&](const std::unique_ptr<Resident> &r) { return r.get() == lru; }));
    }
    auto r = std::make_unique<Resident>();
    r->key = j->key;
    r->bytes = j->est;
    r->busy = true;
    r->last_use = ++use_clock;
    resident_bytes += j->est;
    peak_bytes = std::max(peak_bytes, resident_bytes);
    *out = r.get();
    residents.push_back(std::move(r));
    return true;
  }

  void run(Job *j, Resident *r, cudaStream_t s) {
    const pse_request &q = j->req;
    pse_status st = PSE_OK;
    if (!r->h) {
      pse_options o;
      pse_default_options(&o);
      if (q.options) o = *q.options;
      st = pse_create(&r->h, q.N, q.L, q.a, q.eta, q.kT, q.xi, q.tol, (pse_precision)q.precision, &o);
      if (st != PSE_OK) r->h = nullptr;
      std::lock_guard<std::mutex> g(mu);
      ++created;
    }
    if (st == PSE_OK) {
      pse_stream ps = (pse_stream)s;
      switch (q.kind) {
        case PSE_REQ_MOBILITY: st = pse_mobility_apply(r->h, q.pos, q.F, q.S, q.U, q.E, ps); break;
        case PSE_REQ_SAMPLE:
          st = pse_brownian_sample(r->h, q.pos, q.dt, q.seed, q.counter, nullptr, nullptr, q.U, q.E, q.stats, ps);
          break;
        case PSE_REQ_STEP:
          st = pse_constrained_step(r->h, q.pos, q.F, q.dt, q.seed, q.counter, q.S_out, q.stats, ps);
          break;
        default: st = PSE_ERR_INVALID_ARG;
      }
      if (cudaStreamSynchronize(s) != cudaSuccess && st == PSE_OK) st = PSE_ERR_CUDA;
    }
    std::lock_guard<std::mutex> g(mu);
    if (!r->h) {  // creation failed: release the reservation
      resident_bytes -= r->bytes;
      residents.erase(std::find_if(residents.begin(), residents.end(),
                                   [&](const std::unique_ptr<Resident> &x) { return x.get() == r; }));
    } else {
      r->busy = false;
      r->last_use = ++use_clock;
    }
    j->status = st;
    j->t_end = Clock::now();
    j->done = true;
    --running;
    latency.push_back(ms_between(j->t_submit, j->t_end));
    wait.push_back(ms_between(j->t_submit, j->t_start));
    service.push_back(ms_between(j->t_start, j->t_end));
    if (!any_done || j->t_end > t_last) t_last = j->t_end;
    any_done = true;
    cv_done.notify_all();
    cv_work.notify_all();  // memory or a resident handle may have become free
  }

  void worker() {
    cudaSetDevice(device);
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return;
    for (;;) {
      Job *j = nullptr;
      Resident *r = nullptr;
      std::vector<pse_handle> to_destroy;
      {
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
          if (stop) break;
          for (auto it = queue.begin(); it != queue.end(); ++it)
            if (admit(*it, &r, to_destroy)) {
              j = *it;
              queue.erase(it);
              break;
            }
          if (j) break;
          cv_work.wait_for(lk, std::chrono::milliseconds(50));
        }
        if (!j) break;
        j->t_start = Clock::now();
        ++running;
        peak_running = std::max(peak_running, running);
      }
      for (pse_handle h : to_destroy) pse_destroy(h);
      run(j, r, s);
    }
    cudaStreamDestroy(s);
  }
};

extern "C" {

pse_status pse_server_create(pse_server **out, int32_t slots, int64_t budget_bytes) {
  if (!out || slots < 1 || slots > 64 || budget_bytes <= 0) return PSE_ERR_INVALID_ARG;
  *out = nullptr;
  int dev = 0, n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n < 1 || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return PSE_ERR_CUDA;
  }
  auto *srv = new pse_server();
  srv->slots = slots;
  srv->budget = budget_bytes;
  srv->device = dev;
  for (int i = 0; i < slots; ++i) srv->workers.emplace_back([srv] { srv->worker(); });
  *out = srv;
  return PSE_OK;
}

pse_status pse_server_submit(pse_server *srv, const pse_request *req, uint64_t *ticket) {
  if (!srv || !req || !ticket || !req->pos) return PSE_ERR_INVALID_ARG;
  auto j = std::make_unique<Job>();
  j->req = *req;
  j->key = key_of(*req);
  int64_t L = 0;
  pse_status st = pse_estimate_bytes(1, &req->N, &req->L, req->a, req->eta, req->kT, req->xi, req->tol,
                                     (pse_precision)req->precision, req->options, &L);
  if (st != PSE_OK) return st;
  j->est = L;
  std::lock_guard<std::mutex> g(srv->mu);
  if (j->est > srv->budget) {
    ++srv->rejected;
    srv->err = "request needs " + std::to_string(j->est) + " bytes, more than the budget";
    return PSE_ERR_OOM;
  }
  j->id = srv->next_id++;
  j->t_submit = Clock::now();
  if (!srv->first_set) {
    srv->t_first = j->t_submit;
    srv->first_set = true;
  }
  *ticket = j->id;
  srv->queue.push_back(j.get());
  srv->jobs[j->id] = std::move(j);
  srv->cv_work.notify_one();
  return PSE_OK;
}

pse_status pse_server_wait(pse_server *srv, uint64_t ticket, double timeout_ms, pse_status *result,
                           double *latency_ms) {
  if (!srv) return PSE_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) return PSE_ERR_INVALID_ARG;
  Job *j = it->second.get();
  auto limit = Clock::now() + std::chrono::microseconds((int64_t)(timeout_ms * 1000.0));
  while (!j->done)
    if (srv->cv_done.wait_until(lk, limit) == std::cv_status::timeout && !j->done) return PSE_ERR_TIMEOUT;
  if (result) *result = j->status;
  if (latency_ms) *latency_ms = ms_between(j->t_submit, j->t_end);
  srv->jobs.erase(it);
  return PSE_OK;
}

pse_status pse_server_get_stats(pse_server *srv, pse_server_stats *o) {
  if (!srv || !o) return PSE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(srv->mu);
  std::memset(o, 0, sizeof(*o));
  o->completed = (int64_t)srv->latency.size();
  o->queued = (int64_t)srv->queue.size();
  o->running = srv->running;
  o->peak_running = srv->peak_running;
  o->p50_ms = percentile(srv->latency, 0.5);
  o->p99_ms = percentile(srv->latency, 0.99);
  o->wait_p50_ms = percentile(srv->wait, 0.5);
  o->wait_p99_ms = percentile(srv->wait, 0.99);
  o->service_p50_ms = percentile(srv->service, 0.5);
  double span = srv->any_done ? ms_between(srv->t_first, srv->t_last) : 0.0;
  o->requests_per_s = span > 0 ? 1000.0 * (double)o->completed / span : 0.0;
  o->resident_bytes = srv->resident_bytes;
  o->peak_resident_bytes = srv->peak_bytes;
  o->resident_handles = (int32_t)srv->residents.size();
  o->handles_created = srv->created;
  o->handles_reused = srv->reused;
  o->handles_evicted = srv->evicted;
  o->rejected = srv->rejected;
  return PSE_OK;
}

pse_status pse_server_reset_stats(pse_server *srv) {
  if (!srv) return PSE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(srv->mu);
  srv->latency.clear();
  srv->wait.clear();
  srv->service.clear();
  srv->any_done = false;
  srv->first_set = false;
  srv->peak_running = srv->running;
  srv->created = srv->reused = srv->evicted = srv->rejected = 0;
  return PSE_OK;
}

pse_status pse_server_destroy(pse_server *srv) {
  if (!srv) return PSE_ERR_INVALID_ARG;
  {
    std::lock_guard<std::mutex> g(srv->mu);
    srv->stop = true;
    srv->cv_work.notify_all();
  }
  for (auto &t : srv->workers) t.join();
  for (auto &r : srv->residents)
    if (r->h) pse_destroy(r->h);
  delete srv;
  return PSE_OK;
}

}  // extern "C"
