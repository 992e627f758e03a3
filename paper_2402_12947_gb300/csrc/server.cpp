// Solve server: continuous batching of MG-PCG solve requests on one GPU.
//
// Every request is a mesh hierarchy plus a right-hand side. Its life:
//   queued -> host set-up (a worker thread: DoF maps, assembly, transfer, Galerkin, patches,
//   eigenvalues) -> waits for admission (FIFO; the request's device-byte estimate must fit
//   under the HBM budget and an active slot must be free) -> device set-up and the solve
//   graph launch on the request's own stream -> done (the poller thread sees the stream's
//   completion event, copies the result out and frees the hierarchy's device memory, which
//   admits the next requests).
// Requests that arrive while others are on the GPU are admitted as soon as memory and a
// slot free up, and the solves of all active requests overlap on the device (one stream
// each). A request's arithmetic does not depend on what else is running: its kernels see
// only its own buffers (with fixed layouts, sell_sigma >= 1, the result is bitwise the same
// alone and in the mix).
#include <algorithm>
#include <climits>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "internal.hpp"

namespace nnmg {
namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

struct Request {
  int64_t id = 0;
  // inputs (copied at submission)
  int L = 0, degree = 1;
  double thr = 0.1, rtol = 1e-8;
  int maxit = 500;
  mg_options_t opt{};
  std::vector<mg_mesh_t> meshes;
  std::vector<std::vector<double>> coords;
  std::vector<std::vector<int32_t>> cells;
  std::vector<std::vector<uint8_t>> masks;
  std::vector<double> b;
  // progress
  int status = -1;  // -1 while pending
  std::string err;
  mg_hierarchy* h = nullptr;
  int64_t est = 0, bytes = 0, n = 0;
  double *pin_b = nullptr, *pin_x = nullptr;
  cudaEvent_t ev = nullptr, ev0 = nullptr;   // solve done; solve start (timing)
  double t_solve_ms = 0.0;
  std::vector<double> x;
  mg_solve_info_t info{};
  Clock::time_point t_submit, t_setup0, t_setup1, t_admit, t_done;
};

}  // namespace
}  // namespace nnmg

using nnmg::Clock;
using nnmg::Request;

struct mg_server {
  int64_t budget = 0;
  int max_active = 1;
  std::mutex mu;
  std::condition_variable cv_work, cv_admit, cv_done, cv_poll;
  std::deque<Request*> pending;          // waiting for host set-up
  std::set<int64_t> admit_queue;         // ids waiting for admission, FIFO by id
  std::vector<Request*> active;          // launched on the device
  std::map<int64_t, std::unique_ptr<Request>> all;
  int64_t next_id = 1, in_use = 0, peak_bytes = 0;
  int64_t submitted = 0, completed = 0, failed = 0;
  int n_active = 0, peak_active = 0;
  int n_setup = 0;                       // requests in host set-up on a worker
  bool stop = false;
  std::vector<std::thread> workers;
  std::thread poller;

  void finish_locked(Request* r, int status, const std::string& err) {
    r->status = status;
    r->err = err;
    r->t_done = Clock::now();
    ++completed;
    if (status != MG_OK) ++failed;
    cv_done.notify_all();
  }

  void worker() {
    for (;;) {
      Request* r = nullptr;
      int busy = 1;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || !pending.empty(); });
        if (stop && pending.empty()) return;
        r = pending.front();
        pending.pop_front();
        busy = ++n_setup;
      }
      // the host cores are shared among the requests in set-up when this one starts: alone it
      // may use all of them, with k others a 1/(k+1) share (the set-up arithmetic does not
      // depend on the number of threads)
      nnmg::set_thread_budget(std::max(1, (int)std::thread::hardware_concurrency() / busy));
      struct SetupDone {   // leaves the count when the host set-up ends, on every path
        mg_server* s;
        bool in = true;
        void leave() {
          if (!in) return;
          in = false;
          std::lock_guard<std::mutex> lk(s->mu);
          --s->n_setup;
        }
        ~SetupDone() { leave(); }
      } setup_done{this};
      r->t_setup0 = Clock::now();
      try {
        r->h = nnmg::build_host_hierarchy(r->meshes.data(), r->L, r->degree, r->thr, &r->opt);
        r->n = nnmg::hierarchy_dofs(r->h);
        if (r->b.empty()) r->b = nnmg::hierarchy_unit_load(r->h);
        if ((int64_t)r->b.size() != r->n) throw nnmg::Error(MG_ERR_INVALID_ARG, "right-hand side has the wrong length");
        r->est = nnmg::estimate_device_bytes(r->h);
      } catch (const nnmg::Error& e) {
        std::lock_guard<std::mutex> lk(mu);
        if (r->h) nnmg::destroy_hierarchy(r->h), r->h = nullptr;
        finish_locked(r, e.code, e.what());
        continue;
      } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lk(mu);
        if (r->h) nnmg::destroy_hierarchy(r->h), r->h = nullptr;
        finish_locked(r, MG_ERR_OOM, e.what());
        continue;
      }
      r->t_setup1 = Clock::now();
      setup_done.leave();
      // admission: first in line, a free slot, and room under the budget
      {
        std::unique_lock<std::mutex> lk(mu);
        if (r->est > budget) {
          nnmg::destroy_hierarchy(r->h);
          r->h = nullptr;
          finish_locked(r, MG_ERR_OOM, "request needs more device memory than the whole budget");
          continue;
        }
        admit_queue.insert(r->id);
        cv_admit.wait(lk, [&] {
          return stop || (*admit_queue.begin() == r->id && n_active < max_active && in_use + r->est <= budget);
        });
        admit_queue.erase(r->id);
        if (stop) {
          nnmg::destroy_hierarchy(r->h);
          r->h = nullptr;
          finish_locked(r, MG_ERR_INVALID_ARG, "server stopped");
          cv_admit.notify_all();
          continue;
        }
        in_use += r->est;
        peak_bytes = std::max(peak_bytes, in_use);
        ++n_active;
        peak_active = std::max(peak_active, n_active);
        cv_admit.notify_all();
      }
      r->t_admit = Clock::now();
      try {
        nnmg::build_device_hierarchy(r->h);
        r->bytes = nnmg::hierarchy_device_bytes(r->h);
        r->pin_b = nnmg::pinned_acquire(r->n);
        r->pin_x = nnmg::pinned_acquire(r->n);
        std::memcpy(r->pin_b, r->b.data(), sizeof(double) * r->n);
        if (cudaEventCreate(&r->ev) != cudaSuccess || cudaEventCreate(&r->ev0) != cudaSuccess)
          throw nnmg::Error(MG_ERR_CUDA, "cudaEventCreate failed");
        nnmg::enqueue_host_solve(r->h, r->pin_b, r->pin_x, r->rtol, r->maxit, r->ev, r->ev0);
      } catch (const nnmg::Error& e) {
        std::lock_guard<std::mutex> lk(mu);
        release_locked(r);
        finish_locked(r, e.code, e.what());
        continue;
      } catch (const std::exception& e) {
        std::lock_guard<std::mutex> lk(mu);
        release_locked(r);
        finish_locked(r, MG_ERR_OOM, e.what());
        continue;
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        active.push_back(r);
      }
      cv_poll.notify_one();
    }
  }

  // Frees a request's device and staging resources and gives its budget back.
  void release_locked(Request* r) {
    if (r->h) nnmg::destroy_hierarchy(r->h);
    r->h = nullptr;
    nnmg::pinned_release(r->pin_b);
    nnmg::pinned_release(r->pin_x);
    r->pin_b = r->pin_x = nullptr;
    if (r->ev) cudaEventDestroy(r->ev);
    if (r->ev0) cudaEventDestroy(r->ev0);
    r->ev = r->ev0 = nullptr;
    in_use -= r->est;
    --n_active;
    cv_admit.notify_all();
  }

  void poll() {
    for (;;) {
      std::vector<Request*> finished;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_poll.wait_for(lk, std::chrono::microseconds(200), [&] { return stop || !active.empty(); });
        // admitted requests (n_active) include those still in their device set-up
        if (stop && active.empty() && n_active == 0 && pending.empty() && admit_queue.empty()) return;
        for (size_t i = 0; i < active.size();) {
          if (cudaEventQuery(active[i]->ev) == cudaSuccess) {
            finished.push_back(active[i]);
            active[i] = active.back();
            active.pop_back();
          } else {
            ++i;
          }
        }
      }
      if (finished.empty()) std::this_thread::sleep_for(std::chrono::microseconds(50));
      for (Request* r : finished) {
        int st = nnmg::collect_host_solve(r->h, &r->info);
        float ms = 0.f;
        if (r->ev0 && cudaEventElapsedTime(&ms, r->ev0, r->ev) == cudaSuccess) r->t_solve_ms = ms;
        r->x.assign(r->pin_x, r->pin_x + r->n);
        std::lock_guard<std::mutex> lk(mu);
        release_locked(r);
        finish_locked(r, st, st == MG_OK ? "" : "solve did not converge");
      }
    }
  }
};

namespace {
thread_local std::string g_server_error;

void fill_result(const Request* r, mg_request_result_t* out) {
  std::memset(out, 0, sizeof(*out));
  out->status = r->status;
  out->iterations = r->info.iterations;
  out->rel_residual = r->info.rel_residual;
  out->true_rel_residual = r->info.true_rel_residual;
  out->n = r->n;
  out->device_bytes = r->bytes;
  if (r->status < 0) return;
  Clock::time_point setup0 = r->t_setup0.time_since_epoch().count() ? r->t_setup0 : r->t_done;
  Clock::time_point setup1 = r->t_setup1.time_since_epoch().count() ? r->t_setup1 : r->t_done;
  Clock::time_point admit = r->t_admit.time_since_epoch().count() ? r->t_admit : r->t_done;
  out->t_queue_ms = nnmg::ms_between(r->t_submit, setup0);
  out->t_setup_ms = nnmg::ms_between(setup0, setup1);
  out->t_wait_ms = nnmg::ms_between(setup1, admit);
  out->t_device_ms = nnmg::ms_between(admit, r->t_done);
  out->t_total_ms = nnmg::ms_between(r->t_submit, r->t_done);
  out->t_solve_ms = r->t_solve_ms;
}
}  // namespace

extern "C" {

int mg_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t setup_threads, mg_server_t** out) {
  if (!out || hbm_budget_bytes <= 0 || max_active < 1 || setup_threads < 1 || setup_threads > 64) {
    g_server_error = "invalid server arguments";
    return MG_ERR_INVALID_ARG;
  }
  mg_server* s = new mg_server();
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  for (int i = 0; i < setup_threads; ++i) s->workers.emplace_back(&mg_server::worker, s);
  s->poller = std::thread(&mg_server::poll, s);
  *out = s;
  return MG_OK;
}

int mg_server_submit(mg_server_t* s, const mg_request_t* q, int64_t* id) {
  if (!s || !q || !id || !q->levels || q->L < 2 || q->L > 32) {
    g_server_error = "invalid request";
    return MG_ERR_INVALID_ARG;
  }
  std::unique_ptr<Request> r(new Request());
  r->L = q->L;
  r->degree = q->degree;
  r->thr = q->quality_threshold;
  r->rtol = q->rtol;
  r->maxit = q->maxit;
  if (q->opt) r->opt = *q->opt;
  else mg_default_options(&r->opt);
  r->opt.host_only = 0;
  r->opt.use_graph = 1;
  if (!q->tune) r->opt.tune_min_nnz = INT32_MAX;
  r->meshes.resize(q->L);
  r->coords.resize(q->L);
  r->cells.resize(q->L);
  r->masks.resize(q->L);
  for (int l = 0; l < q->L; ++l) {
    const mg_mesh_t& m = q->levels[l];
    if ((m.dim != 2 && m.dim != 3) || m.nv < 1 || m.nc < 1 || !m.coords || !m.cells) {
      g_server_error = "invalid mesh in request";
      return MG_ERR_INVALID_ARG;
    }
    r->coords[l].assign(m.coords, m.coords + m.nv * m.dim);
    r->cells[l].assign(m.cells, m.cells + m.nc * (m.dim + 1));
    r->meshes[l] = m;
    r->meshes[l].coords = r->coords[l].data();
    r->meshes[l].cells = r->cells[l].data();
    if (m.dirichlet_vertex_mask) {
      r->masks[l].assign(m.dirichlet_vertex_mask, m.dirichlet_vertex_mask + m.nv);
      r->meshes[l].dirichlet_vertex_mask = r->masks[l].data();
    }
  }
  if (q->b && q->n_b > 0) r->b.assign(q->b, q->b + q->n_b);
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    *id = r->id;
    s->pending.push_back(r.get());
    s->all[r->id] = std::move(r);
    ++s->submitted;
  }
  s->cv_work.notify_one();
  return MG_OK;
}

int mg_server_poll(mg_server_t* s, int64_t id, mg_request_result_t* out) {
  if (!s || !out) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return MG_ERR_INVALID_ARG;
  fill_result(it->second.get(), out);
  return MG_OK;
}

int mg_server_wait(mg_server_t* s, int64_t id, double timeout_s, mg_request_result_t* out) {
  if (!s) return MG_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end()) return MG_ERR_INVALID_ARG;
  Request* r = it->second.get();
  bool ok = s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->status >= 0; });
  if (out) fill_result(r, out);
  return ok ? MG_OK : MG_ERR_TIMEOUT;
}

int mg_server_fetch(mg_server_t* s, int64_t id, double* x, int64_t n) {
  if (!s) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(id);
  if (it == s->all.end() || it->second->status < 0) return MG_ERR_INVALID_ARG;
  Request* r = it->second.get();
  if (x) {
    if (n != (int64_t)r->x.size()) return MG_ERR_INVALID_ARG;
    std::memcpy(x, r->x.data(), sizeof(double) * n);
  }
  s->all.erase(it);
  return MG_OK;
}

int mg_server_stats(mg_server_t* s, mg_server_stats_t* out) {
  if (!s || !out) return MG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->bytes_in_use = s->in_use;
  out->peak_bytes = s->peak_bytes;
  out->active = s->n_active;
  out->peak_active = s->peak_active;
  out->queued = (int32_t)(s->pending.size() + s->admit_queue.size());
  return MG_OK;
}

const char* mg_server_last_error(void) { return g_server_error.c_str(); }

void mg_server_destroy(mg_server_t* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->cv_admit.notify_all();
  s->cv_poll.notify_all();
  for (auto& t : s->workers) t.join();
  // the poller drains the solves already on the device
  s->poller.join();
  delete s;
}

}  // extern "C"
