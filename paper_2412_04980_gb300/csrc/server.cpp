// Serving: a request loop that admits Helmholtz solves of different sizes and wavenumbers
// against a device-memory budget and runs them concurrently.
//
// Each request owns a handle (its level hierarchy and Krylov bases stay resident on the
// device for the whole solve) and a CUDA stream.  A pool of worker threads takes requests in
// arrival order; a request whose estimated footprint does not fit the remaining budget waits
// while later, smaller requests that do fit are admitted (first fit), so slots and memory are
// reused as soon as they free up.  Work of concurrent requests overlaps on the GPU; every
// request's arithmetic is independent of the others, so its result equals the result of
// running it alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "hz_core.h"

namespace hz {
const char* last_error_message();
}
using namespace hz;

namespace {

typedef std::chrono::steady_clock Clock;

struct Req {
  uint64_t id = 0;
  hz_grid grid{};
  hz_config cfg{};
  int nrhs = 1;
  double tol = 1e-6;
  std::vector<double> k, b;  // host copies taken at submit
  double* u_out = nullptr;
  hz_stats* stats_out = nullptr;
  size_t bytes = 0;
  int status = HZ_PENDING;
  std::string err;           // detailed message of a failed request (set by its worker)
  bool done = false;
  Clock::time_point t_submit, t_start, t_end;
};

}  // namespace

struct hz_server_s {
  size_t budget = 0, used = 0, peak = 0;
  int max_active = 1, active = 0, device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> queue;
  std::map<uint64_t, std::unique_ptr<Req>> reqs;
  std::vector<std::thread> workers;
  uint64_t next_id = 1;
  bool stop = false;
  Clock::time_point t_first, t_last;
  bool any = false;
  std::vector<double> latencies_ms;
  long long completed = 0, failed = 0;
};

namespace {

// Run one admitted request to completion on its own stream and handle.
int run_request(hz_server_s* S, Req* r) {
  cudaStream_t s = nullptr;
  int st = status_of(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
  if (st) return st;
  const size_t n = (size_t)r->grid.nx * r->grid.ny, nk = r->k.size();
  void *kd = nullptr, *bd = nullptr, *ud = nullptr;
  hz_handle h = nullptr;
  std::vector<hz_stats> stats(r->nrhs);
  do {
    if ((st = status_of(cudaMalloc(&kd, nk * 8), "cudaMalloc"))) break;
    if ((st = status_of(cudaMalloc(&bd, (size_t)r->nrhs * n * 16), "cudaMalloc"))) break;
    if ((st = status_of(cudaMalloc(&ud, (size_t)r->nrhs * n * 16), "cudaMalloc"))) break;
    if ((st = status_of(cudaMemcpyAsync(kd, r->k.data(), nk * 8, cudaMemcpyHostToDevice, s), "copy k"))) break;
    if ((st = status_of(cudaMemcpyAsync(bd, r->b.data(), (size_t)r->nrhs * n * 16, cudaMemcpyHostToDevice, s), "copy b")))
      break;
    if ((st = status_of(cudaStreamSynchronize(s), "sync"))) break;
    if ((st = hz_setup(&r->grid, (const double*)kd, &r->cfg, s, &h))) break;
    st = hz_solve(h, bd, ud, r->nrhs, r->tol, 0, stats.data());
    if (st != HZ_OK && st != HZ_ENOTCONV) break;
    int cst = status_of(cudaMemcpyAsync(r->u_out, ud, (size_t)r->nrhs * n * 16, cudaMemcpyDeviceToHost, s), "copy u");
    if (!cst) cst = status_of(cudaStreamSynchronize(s), "sync");
    if (cst) st = cst;
  } while (false);
  if (h) hz_destroy(h);
  if (kd) cudaFree(kd);
  if (bd) cudaFree(bd);
  if (ud) cudaFree(ud);
  cudaStreamDestroy(s);
  if (r->stats_out && (st == HZ_OK || st == HZ_ENOTCONV))
    std::memcpy(r->stats_out, stats.data(), sizeof(hz_stats) * r->nrhs);
  (void)S;
  return st;
}

void worker(hz_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Req* r = nullptr;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop) return;
        // first request (in arrival order) whose footprint fits the remaining budget
        for (auto it = S->queue.begin(); it != S->queue.end(); ++it)
          if (S->used + (*it)->bytes <= S->budget) {
            r = *it;
            S->queue.erase(it);
            break;
          }
        if (r) break;
        S->cv_work.wait(lk);
      }
      S->used += r->bytes;
      S->peak = std::max(S->peak, S->used);
      S->active += 1;
      r->t_start = Clock::now();
    }
    const int st = run_request(S, r);
    std::vector<double>().swap(r->k);  // host copies are no longer needed
    std::vector<double>().swap(r->b);
    {
      std::lock_guard<std::mutex> lk(S->mu);
      r->t_end = Clock::now();
      r->status = st;
      if (st != HZ_OK) r->err = last_error_message();
      r->done = true;
      S->used -= r->bytes;
      S->active -= 1;
      if (st == HZ_OK) {
        S->completed += 1;
        S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count());
      } else {
        S->failed += 1;
      }
      S->t_last = r->t_end;
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(q * v.size()) - 1);
  return v[i];
}

}  // namespace

extern "C" {

int hz_estimate_bytes(const hz_grid* grid, const hz_config* cfg, size_t* bytes) {
  if (!grid || !cfg || !bytes) {
    set_error("null argument");
    return HZ_EINVAL;
  }
  *bytes = estimate_bytes(*grid, *cfg);
  return HZ_OK;
}

int hz_server_create(size_t mem_budget_bytes, int max_active, hz_server* out) {
  if (!out || max_active < 1 || mem_budget_bytes == 0) {
    set_error("hz_server_create: null output, max_active < 1 or zero budget");
    return HZ_EINVAL;
  }
  auto* S = new (std::nothrow) hz_server_s();
  if (!S) return HZ_ENOMEM;
  S->budget = mem_budget_bytes;
  S->max_active = max_active;
  if (int st = status_of(cudaGetDevice(&S->device), "cudaGetDevice")) {
    delete S;
    return st;
  }
  try {
    for (int i = 0; i < max_active; ++i) S->workers.emplace_back(worker, S);
  } catch (...) {
    set_error("hz_server_create: could not start the worker threads");
    hz_server_destroy(S);
    return HZ_ENOMEM;
  }
  *out = S;
  return HZ_OK;
}

int hz_submit(hz_server S, const hz_request* q, uint64_t* ticket) {
  if (!S || !q || !ticket || !q->k_host || !q->b_host || !q->u_host || q->nrhs < 1) {
    set_error("hz_submit: null argument or nrhs < 1");
    return HZ_EINVAL;
  }
  if ((q->grid.bc != HZ_BC_SOMMERFELD && q->grid.bc != HZ_BC_DIRICHLET) || q->config.max_rhs < q->nrhs ||
      !(q->tol > 0 && q->tol < 1)) {
    set_error("hz_submit: known boundary type, config.max_rhs >= nrhs and tol in (0, 1) required");
    return HZ_EINVAL;
  }
  auto r = std::make_unique<Req>();
  r->grid = q->grid;
  r->cfg = q->config;
  r->nrhs = q->nrhs;
  r->tol = q->tol;
  const size_t n = (size_t)q->grid.nx * q->grid.ny;
  const size_t nk = n * (q->config.per_rhs_k ? (size_t)q->config.max_rhs : 1);  // wavenumber fields
  r->k.assign(q->k_host, q->k_host + nk);
  r->b.assign(q->b_host, q->b_host + 2 * n * q->nrhs);
  r->u_out = q->u_host;
  r->stats_out = q->stats_host;
  // footprint: handle workspace + the request's own device copies of k, b, u
  r->bytes = estimate_bytes(q->grid, q->config) + nk * 8 + 2 * n * 16 * (size_t)q->nrhs;
  if (r->bytes > S->budget) {
    set_error("request footprint exceeds the server memory budget");
    return HZ_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    r->t_submit = Clock::now();
    if (!S->any) {
      S->any = true;
      S->t_first = r->t_submit;
    }
    *ticket = r->id;
    S->queue.push_back(r.get());
    S->reqs[r->id] = std::move(r);
  }
  S->cv_work.notify_all();
  return HZ_OK;
}

int hz_poll(hz_server S, uint64_t ticket, double* latency_ms) {
  if (!S) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown ticket");
    return HZ_EINVAL;
  }
  Req* r = it->second.get();
  if (!r->done) return HZ_PENDING;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count();
  if (r->status != HZ_OK) set_error(r->err);
  return r->status;
}

int hz_wait(hz_server S, uint64_t ticket, double timeout_s, double* latency_ms) {
  if (!S) return HZ_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("unknown ticket");
    return HZ_EINVAL;
  }
  Req* r = it->second.get();
  if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), [&] { return r->done; })) {
    set_error("hz_wait: request still running after the given timeout");
    return HZ_ETIMEOUT;
  }
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_end - r->t_submit).count();
  if (r->status != HZ_OK) set_error(r->err);
  return r->status;
}

int hz_server_report(hz_server S, hz_server_stats* out) {
  if (!S || !out) return HZ_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof(*out));
  out->completed = S->completed;
  out->failed = S->failed;
  out->queued = (long long)S->queue.size();
  out->active = S->active;
  out->p50_ms = percentile(S->latencies_ms, 0.50);
  out->p99_ms = percentile(S->latencies_ms, 0.99);
  const double span = S->any ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
  out->solves_per_s = span > 0 ? S->completed / span : 0.0;
  out->peak_bytes = S->peak;
  out->budget_bytes = S->budget;
  return HZ_OK;
}

int hz_server_destroy(hz_server S) {
  if (!S) return HZ_OK;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // finish what is running; drop what has not started
    for (Req* r : S->queue) {
      r->status = HZ_EINVAL;
      r->err = "server destroyed before the request started";
      r->done = true;
    }
    S->queue.clear();
    S->stop = true;
  }
  S->cv_done.notify_all();
  S->cv_work.notify_all();
  for (auto& t : S->workers) t.join();
  delete S;
  return HZ_OK;
}

}  // extern "C"
