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
//
// With batching on (hz_server_set_batching), a worker that takes a request also takes the queued
// requests with the same grid, configuration and tolerance, in arrival order, while the merged
// right-hand sides stay within the batch limit and the merged footprint within the budget.  The
// group runs as one multi-instance solve (per_rhs_k: every right-hand side keeps its request's
// wavenumber field), so each sweep is one launch over all of them; the results are scattered back
// to the requests, each with its own statistics and status.
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
#include <new>
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
  int batch_rhs = 0;                 // right-hand sides of a merged solve (<= 1: no merging)
  long long merged_solves = 0, merged_requests = 0;
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

// Requests that may share one multi-instance solve: same grid and tolerance, and the same
// configuration apart from max_rhs and per_rhs_k.
bool same_grid_config(const Req* a, const Req* b) {
  const hz_grid &g = a->grid, &h = b->grid;
  if (g.nx != h.nx || g.ny != h.ny || g.h != h.h || g.bc != h.bc || a->tol != b->tol) return false;
  const hz_config &x = a->cfg, &y = b->cfg;
  if (x.levels != y.levels || x.precision != y.precision || x.beta1 != y.beta1 || x.beta2 != y.beta2 ||
      x.restart != y.restart || x.max_outer != y.max_outer || x.l2_tol != y.l2_tol || x.l2_maxit != y.l2_maxit ||
      x.cslp_tol != y.cslp_tol || x.c_it != y.c_it || x.coarsest_tol != y.coarsest_tol ||
      x.negdef_from_level != y.negdef_from_level || x.mg_max_level != y.mg_max_level || x.mg_omega != y.mg_omega ||
      x.mg_nu1 != y.mg_nu1 || x.mg_nu2 != y.mg_nu2 || x.mg_coarsest_side != y.mg_coarsest_side ||
      x.timeout_s != y.timeout_s || x.device_gmres != y.device_gmres || x.reorth_eta != y.reorth_eta ||
      x.graphs != y.graphs || x.autotune != y.autotune || x.cycle_m != y.cycle_m ||
      x.cslp_solver != y.cslp_solver || x.sym_rows != y.sym_rows)
    return false;
  for (int l = 0; l < HZ_MAX_LEVELS; ++l)
    if (x.level_tol[l] != y.level_tol[l]) return false;
  return true;
}

// Footprint of a merged solve of nb right-hand sides: handle workspace with one wavenumber field
// per right-hand side, plus the device copies of the fields, b and u.
size_t group_bytes(const Req* r, int nb) {
  hz_config c = r->cfg;
  c.max_rhs = nb;
  c.per_rhs_k = 1;
  const size_t n = (size_t)r->grid.nx * r->grid.ny;
  return estimate_bytes(r->grid, c) + (size_t)nb * n * (8 + 2 * 16);
}

// Run a group of compatible requests as one multi-instance solve on its own stream and handle.
// Returns the status of the shared part (set-up, copies); st_out always receives one status per
// request of the group.
int run_group(const std::vector<Req*>& grp, std::vector<int>& st_out) {
  const Req* r0 = grp[0];
  const size_t n = (size_t)r0->grid.nx * r0->grid.ny;
  int nb = 0;
  for (const Req* r : grp) nb += r->nrhs;
  // wavenumber field of every right-hand side (its request's field), right-hand sides in order
  std::vector<double> k, b;
  try {
    k.resize((size_t)nb * n);
    b.resize((size_t)nb * n * 2);
  } catch (const std::bad_alloc&) {
    set_error("host memory for a merged solve could not be allocated");
    st_out.assign(grp.size(), HZ_ENOMEM);
    return HZ_ENOMEM;
  }
  size_t o = 0;
  for (const Req* r : grp) {
    for (int q = 0; q < r->nrhs; ++q) {
      const double* src = r->k.data() + (r->cfg.per_rhs_k ? (size_t)q * n : 0);
      std::memcpy(k.data() + (o + q) * n, src, n * 8);
    }
    std::memcpy(b.data() + o * n * 2, r->b.data(), (size_t)r->nrhs * n * 16);
    o += r->nrhs;
  }
  hz_config cfg = r0->cfg;
  cfg.max_rhs = nb;
  cfg.per_rhs_k = 1;
  cudaStream_t s = nullptr;
  int st = status_of(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
  if (st) {
    st_out.assign(grp.size(), st);
    return st;
  }
  void *kd = nullptr, *bd = nullptr, *ud = nullptr;
  hz_handle h = nullptr;
  std::vector<hz_stats> stats(nb);
  int sst = HZ_OK;
  do {
    if ((st = status_of(cudaMalloc(&kd, (size_t)nb * n * 8), "cudaMalloc"))) break;
    if ((st = status_of(cudaMalloc(&bd, (size_t)nb * n * 16), "cudaMalloc"))) break;
    if ((st = status_of(cudaMalloc(&ud, (size_t)nb * n * 16), "cudaMalloc"))) break;
    if ((st = status_of(cudaMemcpyAsync(kd, k.data(), (size_t)nb * n * 8, cudaMemcpyHostToDevice, s), "copy k"))) break;
    if ((st = status_of(cudaMemcpyAsync(bd, b.data(), (size_t)nb * n * 16, cudaMemcpyHostToDevice, s), "copy b")))
      break;
    if ((st = status_of(cudaStreamSynchronize(s), "sync"))) break;
    if ((st = hz_setup(&r0->grid, (const double*)kd, &cfg, s, &h))) break;
    sst = hz_solve(h, bd, ud, nb, r0->tol, 0, stats.data());
    if (sst != HZ_OK && sst != HZ_ENOTCONV && sst != HZ_EBREAKDOWN) {
      st = sst;
      break;
    }
    o = 0;
    for (const Req* r : grp) {
      st = status_of(cudaMemcpyAsync(r->u_out, (const char*)ud + o * n * 16, (size_t)r->nrhs * n * 16,
                                     cudaMemcpyDeviceToHost, s),
                     "copy u");
      if (st) break;
      o += r->nrhs;
    }
    if (!st) st = status_of(cudaStreamSynchronize(s), "sync");
  } while (false);
  if (h) hz_destroy(h);
  if (kd) cudaFree(kd);
  if (bd) cudaFree(bd);
  if (ud) cudaFree(ud);
  cudaStreamDestroy(s);
  st_out.assign(grp.size(), st);
  if (st) return st;
  o = 0;
  for (size_t i = 0; i < grp.size(); ++i) {
    const Req* r = grp[i];
    int rs = HZ_OK;  // the first failing right-hand side decides, as hz_solve does
    for (int q = 0; q < r->nrhs && rs == HZ_OK; ++q) rs = stats[o + q].status;
    st_out[i] = rs;
    if (r->stats_out) std::memcpy(r->stats_out, stats.data() + o, sizeof(hz_stats) * r->nrhs);
    o += r->nrhs;
  }
  return HZ_OK;
}

void worker(hz_server_s* S) {
  cudaSetDevice(S->device);
  for (;;) {
    Req* r = nullptr;
    std::vector<Req*> grp;
    size_t gbytes = 0;
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
      grp.push_back(r);
      gbytes = r->bytes;
      if (S->batch_rhs > 1 && r->nrhs < S->batch_rhs) {
        // compatible queued requests join while the batch and the budget allow
        int nb = r->nrhs;
        for (auto it = S->queue.begin(); it != S->queue.end();) {
          Req* q = *it;
          if (nb + q->nrhs <= S->batch_rhs && same_grid_config(r, q)) {
            const size_t gb = group_bytes(r, nb + q->nrhs);
            if (S->used + gb <= S->budget) {
              grp.push_back(q);
              nb += q->nrhs;
              gbytes = gb;
              it = S->queue.erase(it);
              continue;
            }
          }
          ++it;
        }
        if (grp.size() > 1) {
          S->merged_solves += 1;
          S->merged_requests += (long long)grp.size();
        }
      }
      S->used += gbytes;
      S->peak = std::max(S->peak, S->used);
      S->active += 1;
      for (Req* q : grp) q->t_start = Clock::now();
    }
    std::vector<int> sts(1, HZ_OK);
    if (grp.size() == 1) {
      sts[0] = run_request(S, r);
    } else {
      run_group(grp, sts);
      sts.resize(grp.size(), HZ_ECUDA);  // one status per request, whatever path run_group took
    }
    const std::string msg = last_error_message();
    for (Req* q : grp) {
      std::vector<double>().swap(q->k);  // host copies are no longer needed
      std::vector<double>().swap(q->b);
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      const Clock::time_point t_end = Clock::now();
      for (size_t i = 0; i < grp.size(); ++i) {
        Req* q = grp[i];
        const int st = sts[i];
        q->t_end = t_end;
        q->status = st;
        if (st != HZ_OK) q->err = msg;
        q->done = true;
        if (st == HZ_OK) {
          S->completed += 1;
          S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(q->t_end - q->t_submit).count());
        } else {
          S->failed += 1;
        }
      }
      S->used -= gbytes;
      S->active -= 1;
      S->t_last = t_end;
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
  std::unique_ptr<Req> r;
  try {  // the host copies of k and b can be large: a failed allocation is the caller's HZ_ENOMEM
    r = std::make_unique<Req>();
    const size_t n = (size_t)q->grid.nx * q->grid.ny;
    r->k.assign(q->k_host, q->k_host + n * (q->config.per_rhs_k ? (size_t)q->config.max_rhs : 1));
    r->b.assign(q->b_host, q->b_host + 2 * n * q->nrhs);
  } catch (const std::bad_alloc&) {
    set_error("hz_submit: host memory for the request's copies of k and b could not be allocated");
    return HZ_ENOMEM;
  }
  r->grid = q->grid;
  r->cfg = q->config;
  r->nrhs = q->nrhs;
  r->tol = q->tol;
  const size_t n = (size_t)q->grid.nx * q->grid.ny;
  const size_t nk = r->k.size();  // wavenumber fields
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
  out->merged_solves = S->merged_solves;
  out->merged_requests = S->merged_requests;
  return HZ_OK;
}

int hz_server_set_batching(hz_server S, int max_batch_rhs) {
  if (!S || max_batch_rhs < 0 || max_batch_rhs > 1024) {
    set_error("hz_server_set_batching: null server or max_batch_rhs outside [0, 1024]");
    return HZ_EINVAL;
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->batch_rhs = max_batch_rhs;
  }
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
