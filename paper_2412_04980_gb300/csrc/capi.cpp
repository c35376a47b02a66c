// extern "C" entry points declared in include/hz.h: argument validation, status codes,
// and dispatch to the runtime in hz_core.cpp.
#include <chrono>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "hz_core.h"

namespace hz {
const char* last_error_message();
}

using namespace hz;

struct hz_handle_s {
  Handle h;
};

static int bad(const char* msg) {
  set_error(msg);
  return HZ_EINVAL;
}

#define GUARD_HANDLE(hp)                         \
  if (!(hp)) return bad("null handle");          \
  Handle* H_ = &(hp)->h;                         \
  (void)H_

static int check_level(Handle* H, int level) {
  if (level < 1 || level > (int)H->lv.size()) return bad("level out of range");
  return HZ_OK;
}
static int check_dtype(int dt) { return (dt == HZ_C128 || dt == HZ_C64) ? HZ_OK : bad("dtype must be HZ_C128 or HZ_C64"); }
static int check_nrhs(Handle* H, int nrhs, bool workspace) {
  if (nrhs < 1) return bad("nrhs must be >= 1");
  if (workspace && nrhs > H->nbmax) return bad("nrhs exceeds the handle's max_rhs");
  if (H->cfg.per_rhs_k && nrhs > H->nbmax)
    return bad("with per_rhs_k every right-hand side needs its own wavenumber field: nrhs <= max_rhs");
  return HZ_OK;
}

extern "C" {

int hz_config_init(hz_config* c) {
  if (!c) return bad("null config");
  std::memset(c, 0, sizeof(*c));
  c->levels = 1;
  c->precision = HZ_PREC_FP64;
  c->beta1 = 1.0;
  c->beta2 = 0.5;
  c->restart = 30;
  c->max_outer = 300;
  c->l2_tol = 0.3;
  c->l2_maxit = 30;
  c->cslp_tol = 0.1;
  c->c_it = 6.0;
  c->coarsest_tol = 0.1;
  c->negdef_from_level = 0;
  c->mg_max_level = 2;
  c->mg_omega = 0.8;
  c->mg_nu1 = 1;
  c->mg_nu2 = 1;
  c->mg_coarsest_side = 20;
  c->max_rhs = 1;
  c->timeout_s = 600.0;
  c->device_gmres = 1;
  c->reorth_eta = 0.1;
  c->autotune = 1;
  c->graphs = 1;
  c->cycle_m = 1;
  return HZ_OK;
}

int hz_setup(const hz_grid* grid, const double* k_dev, const hz_config* cfg, void* stream, hz_handle* out) {
  if (!grid || !k_dev || !cfg || !out) return bad("null argument");
  *out = nullptr;
  const hz_grid& g = *grid;
  if (g.nx < 3 || g.ny < 3) return bad("grid must have at least 3 nodes per side");
  if (!(g.h > 0) || !std::isfinite(g.h)) return bad("h must be finite and positive");
  if (g.bc != HZ_BC_SOMMERFELD && g.bc != HZ_BC_DIRICHLET) return bad("unknown boundary condition");
  const hz_config& c = *cfg;
  if (c.levels < 1 || c.levels > HZ_MAX_LEVELS) return bad("levels must be in [1, HZ_MAX_LEVELS]");
  if (c.precision != HZ_PREC_FP64 && c.precision != HZ_PREC_MIXED) return bad("unknown precision");
  if (c.restart < 1 || c.max_outer < 1 || c.l2_maxit < 1 || c.max_rhs < 1) return bad("iteration caps and max_rhs must be >= 1");
  if (!(c.c_it > 0) || !(c.mg_omega > 0) || c.mg_nu1 < 0 || c.mg_nu2 < 0 || c.mg_nu1 + c.mg_nu2 < 1)
    return bad("invalid multigrid or Krylov-cap parameter");
  if (c.mg_max_level < 0 || c.mg_coarsest_side < 3) return bad("invalid multigrid level settings");
  if (!(c.timeout_s > 0)) return bad("timeout_s must be positive");
  if (!(c.reorth_eta >= 0 && c.reorth_eta <= 1)) return bad("reorth_eta must be in [0, 1]");
  if (c.autotune != 0 && c.autotune != 1) return bad("autotune must be 0 or 1");
  if (c.graphs != 0 && c.graphs != 1) return bad("graphs must be 0 or 1");
  if (c.device_gmres < 0 || c.device_gmres > 4) return bad("device_gmres must be 0, 1, 2, 3 or 4");
  if (c.cycle_m < 1) return bad("cycle_m must be >= 1");
  if (c.cslp_solver != HZ_CSLP_GMRES && c.cslp_solver != HZ_CSLP_BICGSTAB) return bad("unknown cslp_solver");
  if (c.sym_rows != 0 && c.sym_rows != 1) return bad("sym_rows must be 0 or 1");
  if (c.per_rhs_k != 0 && c.per_rhs_k != 1) return bad("per_rhs_k must be 0 or 1");
  if (c.sym_rows && g.bc != HZ_BC_SOMMERFELD) return bad("sym_rows scales Sommerfeld boundary rows (Sommerfeld grids only)");
  if (!(c.l2_tol >= 0 && c.l2_tol < 1)) return bad("l2_tol must be in [0, 1)");
  for (int l = 1; l <= HZ_MAX_LEVELS; ++l) {
    const double t = c.level_tol[l - 1];
    if (!(t >= 0 && t < 1)) return bad("level_tol entries must be in [0, 1)");
    if (t > 0 && (l < 3 || l >= c.levels)) return bad("level_tol is set for levels 3 .. levels-1 only");
  }
  int nx = g.nx, ny = g.ny;
  const bool dir = g.bc == HZ_BC_DIRICHLET;
  for (int l = 1; l < c.levels; ++l) {
    // vertex grids: coarse node I at fine node 2I; Dirichlet grids (interior unknowns): 2I + 1
    if ((nx - 1) % 2 || (ny - 1) % 2 || std::min(nx, ny) < (dir ? 3 : 5))
      return bad(dir ? "Dirichlet grid cannot be coarsened levels-1 times (needs odd sizes >= 3)"
                     : "grid cannot be coarsened levels-1 times (needs odd sizes >= 5)");
    nx = dir ? (nx - 1) / 2 : (nx + 1) / 2;
    ny = dir ? (ny - 1) / 2 : (ny + 1) / 2;
  }
  hz_handle_s* hs = new (std::nothrow) hz_handle_s();
  if (!hs) return HZ_ENOMEM;
  Handle* H = &hs->h;
  H->g = g;
  H->cfg = c;
  H->ctx.s = reinterpret_cast<cudaStream_t>(stream);
  H->ctx.prof = &H->prof;
  const int st = setup(H, k_dev);
  if (st) {
    destroy(H);
    delete hs;
    return st;
  }
  *out = hs;
  return HZ_OK;
}

int hz_destroy(hz_handle hp) {
  if (!hp) return HZ_OK;
  destroy(&hp->h);
  delete hp;
  return HZ_OK;
}

int hz_memory_bytes(hz_handle hp, size_t* bytes) {
  GUARD_HANDLE(hp);
  if (!bytes) return bad("null argument");
  *bytes = H_->bytes;
  return HZ_OK;
}

int hz_apply(hz_handle hp, const void* x, void* y, int nrhs) {
  GUARD_HANDLE(hp);
  if (!x || !y) return bad("null vector");
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  Level& L = H_->lv[0];
  OpDesc A = L.opA(C128);
  A.bc = H_->g.bc;
  A.srow = H_->cfg.sym_rows;  // the handle's outer operator (row-scaled with sym_rows)
  return status_of(launch_level_op(H_->ctx, A, 0, C128, C128, C128, x, nullptr, y, 0.0, nrhs), "hz_apply");
}

int hz_precond(hz_handle hp, const void* v, void* x, int nrhs) {
  GUARD_HANDLE(hp);
  if (!v || !x) return bad("null vector");
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  Level& L = H_->lv[0];
  for (int q = 0; q < nrhs; ++q) H_->st[q] = RhsStats();
  if (L.dx == C128) {
    int s = precond(H_, 1, v, C128, x, nrhs);
    return s ? s : collect_gmres_stats(H_, nrhs);
  }
  int s = precond(H_, 1, v, C128, L.X, nrhs);
  if (s) return s;
  s = status_of(launch_convert(H_->ctx, C64, C128, L.X, x, (size_t)nrhs * L.n), "hz_precond");
  return s ? s : collect_gmres_stats(H_, nrhs);
}

static void fill_stats(Handle* H, hz_stats* stats, int nrhs, double ms) {
  if (!stats) return;
  for (int q = 0; q < nrhs; ++q) {
    hz_stats& s = stats[q];
    std::memset(&s, 0, sizeof(s));
    const RhsStats& r = H->st[q];
    s.status = r.status;
    s.outer_iterations = r.outer;
    for (int l = 0; l < HZ_MAX_LEVELS; ++l) {
      s.level_iterations[l] = r.lev_it[l];
      s.level_calls[l] = r.lev_calls[l];
      s.cslp_gmres_iterations[l] = r.cslp_it[l];
      s.cslp_gmres_reorth[l] = r.cslp_reorth[l];
    }
    s.true_relres = r.true_rel;
    s.est_relres = r.est;
    s.ms = ms;
  }
}

int hz_solve(hz_handle hp, const void* b, void* u, int nrhs, double tol, unsigned flags, hz_stats* stats) {
  GUARD_HANDLE(hp);
  if (!b || !u) return bad("null vector");
  if (!(tol > 0) || !(tol < 1)) return bad("tol must be in (0, 1)");
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  auto t0 = std::chrono::steady_clock::now();
  int st = solve(H_, b, u, nrhs, tol, flags);
  double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (st == HZ_OK || st == HZ_ENOTCONV || st == HZ_EBREAKDOWN) fill_stats(H_, stats, nrhs, ms);
  return st;
}

int hz_solve_host(hz_handle hp, const double* b_host, double* u_host, int nrhs, double tol, unsigned flags,
                  hz_stats* stats) {
  GUARD_HANDLE(hp);
  if (!b_host || !u_host) return bad("null vector");
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  const size_t bytes = (size_t)nrhs * H_->lv[0].n * 16;
  void *bd = nullptr, *ud = nullptr;
  if (cudaMalloc(&bd, bytes) != cudaSuccess || cudaMalloc(&ud, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (bd) cudaFree(bd);
    set_error("device buffers for hz_solve_host");
    return HZ_ENOMEM;
  }
  int st = status_of(cudaMemcpyAsync(bd, b_host, bytes, cudaMemcpyHostToDevice, H_->ctx.s), "hz_solve_host");
  if (!st && (flags & HZ_SOLVE_INITIAL_GUESS))
    st = status_of(cudaMemcpyAsync(ud, u_host, bytes, cudaMemcpyHostToDevice, H_->ctx.s), "hz_solve_host");
  int sst = HZ_OK;
  if (!st) sst = hz_solve(hp, bd, ud, nrhs, tol, flags, stats);
  if (!st && (sst == HZ_OK || sst == HZ_ENOTCONV))
    st = status_of(cudaMemcpyAsync(u_host, ud, bytes, cudaMemcpyDeviceToHost, H_->ctx.s), "hz_solve_host");
  if (!st) st = status_of(cudaStreamSynchronize(H_->ctx.s), "hz_solve_host");
  cudaFree(bd);
  cudaFree(ud);
  return st ? st : sst;
}

int hz_level_size(hz_handle hp, int level, int* nx, int* ny) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (nx) *nx = H_->lv[level - 1].nx;
  if (ny) *ny = H_->lv[level - 1].ny;
  return HZ_OK;
}

int hz_level_gmres_form(hz_handle hp, int level, int* form, int* ctas, int* cluster) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  const Level& L = H_->lv[level - 1];
  int f = L.gtiles > 0 ? HZ_GMRES_TILE : (L.ggrid > 0 ? HZ_GMRES_SLICE : HZ_GMRES_NONE);
  if (H_->cfg.device_gmres == 3 && L.gcl > 0) f = HZ_GMRES_CLUSTER;
  if (form) *form = f;
  if (ctas)
    *ctas = f == HZ_GMRES_TILE ? L.gtiles : (f == HZ_GMRES_SLICE ? L.ggrid : (f == HZ_GMRES_CLUSTER ? L.gcl : 0));
  if (cluster) *cluster = L.gcl;
  return HZ_OK;
}

int hz_level_apply(hz_handle hp, int level, int op, int dtype, const void* x, void* y, int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (int s = check_dtype(dtype)) return s;
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  if (!x || !y) return bad("null vector");
  if (op != HZ_OP_A && op != HZ_OP_M) return bad("op must be HZ_OP_A or HZ_OP_M");
  Level& L = H_->lv[level - 1];
  OpDesc d = op == HZ_OP_A ? L.opA(dtype) : L.opM(dtype, H_->cfg.beta1, H_->cfg.beta2);
  d.bc = H_->g.bc;
  return status_of(launch_level_op(H_->ctx, d, 0, dtype, dtype, dtype, x, nullptr, y, 0.0, nrhs), "hz_level_apply");
}

int hz_level_jacobi(hz_handle hp, int level, int dtype, const void* u, const void* f, void* u_out, int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (int s = check_dtype(dtype)) return s;
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  if (!u || !f || !u_out) return bad("null vector");
  Level& L = H_->lv[level - 1];
  OpDesc d = L.opM(dtype, H_->cfg.beta1, H_->cfg.beta2);
  d.bc = H_->g.bc;
  return status_of(launch_level_op(H_->ctx, d, 2, dtype, dtype, dtype, u, f, u_out, H_->cfg.mg_omega, nrhs),
                   "hz_level_jacobi");
}

int hz_defl_restrict(hz_handle hp, int level, int dtype, const void* v, void* vhat, int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (level >= (int)H_->lv.size()) return bad("level has no coarser level");
  if (int s = check_dtype(dtype)) return s;
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  if (!v || !vhat) return bad("null vector");
  Level& L = H_->lv[level - 1];
  return status_of(launch_defl_restrict(H_->ctx, dtype, dtype, L.nx, L.ny, v, vhat, nrhs, L.bc), "hz_defl_restrict");
}

int hz_defl_prolong(hz_handle hp, int level, int dtype, const void* w, void* t, int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (level >= (int)H_->lv.size()) return bad("level has no coarser level");
  if (int s = check_dtype(dtype)) return s;
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  if (!w || !t) return bad("null vector");
  Level& L = H_->lv[level - 1];
  return status_of(launch_defl_prolong(H_->ctx, dtype, L.nx, L.ny, w, t, nrhs, L.bc), "hz_defl_prolong");
}

int hz_defl_prolong_residual(hz_handle hp, int level, int dtype, const void* vtil, const void* v, void* t, void* rtil,
                             int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (level >= (int)H_->lv.size()) return bad("level has no coarser level");
  if (int s = check_dtype(dtype)) return s;
  if (int s = check_nrhs(H_, nrhs, false)) return s;
  if (!vtil || !v || !rtil) return bad("null vector");
  Level& L = H_->lv[level - 1];
  Level& C = H_->lv[level];
  return status_of(launch_defl_prolong_resid(H_->ctx, L.opA(dtype), dtype, dtype, vtil, C.nx, C.ny, v, t, rtil, nrhs),
                   "hz_defl_prolong_residual");
}

int hz_mg_size(hz_handle hp, int level, int mg_level, int* nx, int* ny) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  Level& L = H_->lv[level - 1];
  if (mg_level < 0 || mg_level >= (int)L.mg.size()) return bad("multigrid level out of range");
  if (nx) *nx = L.mg[mg_level].op.nx;
  if (ny) *ny = L.mg[mg_level].op.ny;
  return HZ_OK;
}

int hz_mg_vcycle(hz_handle hp, int level, int dtype, const void* f, void* u, int nrhs) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  if (!f || !u) return bad("null vector");
  Level& L = H_->lv[level - 1];
  if (L.mg.empty()) return bad("level has no multigrid hierarchy (level > mg_max_level)");
  if (dtype != L.dpre) return bad("dtype must match the handle's preconditioner precision on this level");
  return vcycle(H_, level, dtype, f, u, nullptr, nrhs);
}

int hz_cslp_gmres(hz_handle hp, int level, int dtype, const void* b, void* x, int nrhs, int* iterations) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  if (!b || !x) return bad("null vector");
  Level& L = H_->lv[level - 1];
  if (!L.Vg) return bad("level uses multigrid for the CSLP inverse (level <= mg_max_level)");
  if (dtype != L.dpre) return bad("dtype must match the handle's preconditioner precision on this level");
  for (int q = 0; q < nrhs; ++q) H_->st[q] = RhsStats();
  int st = status_of(cudaMemsetAsync(x, 0, (size_t)nrhs * L.n * elem_bytes(dtype), H_->ctx.s), "hz_cslp_gmres");
  if (st) return st;
  st = cslp_gmres(H_, level, b, x, nrhs, iterations);
  return st ? st : collect_gmres_stats(H_, nrhs);
}

int hz_cslp_bicgstab(hz_handle hp, int level, int dtype, const void* b, void* x, int nrhs, int* iterations) {
  GUARD_HANDLE(hp);
  if (int s = check_level(H_, level)) return s;
  if (int s = check_nrhs(H_, nrhs, true)) return s;
  if (!b || !x) return bad("null vector");
  Level& L = H_->lv[level - 1];
  if (!L.bcg) return bad("level has no Bi-CGSTAB CSLP solver (cslp_solver or level <= mg_max_level)");
  if (dtype != L.dpre) return bad("dtype must match the handle's preconditioner precision on this level");
  for (int q = 0; q < nrhs; ++q) H_->st[q] = RhsStats();
  int st = status_of(cudaMemsetAsync(x, 0, (size_t)nrhs * L.n * elem_bytes(dtype), H_->ctx.s), "hz_cslp_bicgstab");
  if (st) return st;
  st = cslp_bicgstab(H_, level, b, x, nrhs, iterations);
  return st ? st : collect_gmres_stats(H_, nrhs);
}

const char* hz_strerror(int s) {
  switch (s) {
    case HZ_OK: return "HZ_OK";
    case HZ_EINVAL: return "HZ_EINVAL: invalid argument";
    case HZ_ENOMEM: return "HZ_ENOMEM: out of device memory";
    case HZ_ENOTCONV: return "HZ_ENOTCONV: iteration cap reached before the tolerance";
    case HZ_EBREAKDOWN: return "HZ_EBREAKDOWN: non-finite value or Krylov breakdown";
    case HZ_ETIMEOUT: return "HZ_ETIMEOUT: device wait exceeded the limit";
    case HZ_ECUDA: return "HZ_ECUDA: CUDA runtime error";
    case HZ_ENOTSUP: return "HZ_ENOTSUP: not supported by this build";
    case HZ_PENDING: return "HZ_PENDING: request still running";
  }
  return "unknown status";
}

const char* hz_last_error(void) { return last_error_message(); }

int hz_profile_enable(hz_handle hp, int family, int enable) {
  GUARD_HANDLE(hp);
  if (family < 0 || family >= F_COUNT) return bad("unknown kernel family");
  H_->prof.drain(family);
  H_->prof.on[family] = enable != 0;
  if (enable) {
    H_->prof.launches[family] = 0;
    H_->prof.ms[family] = 0;
    H_->prof.bytes[family] = 0;
    for (int l = 0; l < kProfLevels; ++l) {
      H_->prof.launches_lv[family][l] = 0;
      H_->prof.ms_lv[family][l] = 0;
      H_->prof.bytes_lv[family][l] = 0;
    }
  }
  return HZ_OK;
}

int hz_profile_read(hz_handle hp, int family, long long* launches, double* ms, double* bytes) {
  GUARD_HANDLE(hp);
  const int fam = family & 0xff, lev = family >> 8;
  if (fam < 0 || fam >= F_COUNT || lev < 0 || lev >= kProfLevels) return bad("unknown kernel family or level");
  int st = status_of(cudaStreamSynchronize(H_->ctx.s), "hz_profile_read");
  if (st) return st;
  H_->prof.drain(fam);
  const Prof& P = H_->prof;
  if (launches) *launches = lev ? P.launches_lv[fam][lev] : P.launches[fam];
  if (ms) *ms = lev ? P.ms_lv[fam][lev] : P.ms[fam];
  if (bytes) *bytes = lev ? P.bytes_lv[fam][lev] : P.bytes[fam];
  return HZ_OK;
}

int hz_launch_count(hz_handle hp, long long* launches) {
  GUARD_HANDLE(hp);
  if (!launches) return bad("null argument");
  *launches = H_->prof.total_launches;
  return HZ_OK;
}

int hz_gmres_device_time(hz_handle hp, int level, int reset, long long* launches, double* ms, double* bytes) {
  GUARD_HANDLE(hp);
  if (level < 0 || level > HZ_MAX_LEVELS) return bad("level out of range");
  long long n = 0;
  double t = 0, b = 0;
  for (int l = (level ? level : 1); l <= (level ? level : HZ_MAX_LEVELS); ++l) {
    n += H_->gdev_launches[l];
    t += H_->gdev_ms[l];
    b += H_->gdev_bytes[l];
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (bytes) *bytes = b;
  if (reset)
    for (int l = 0; l <= HZ_MAX_LEVELS; ++l) {
      H_->gdev_launches[l] = 0;
      H_->gdev_ms[l] = 0;
      H_->gdev_bytes[l] = 0;
    }
  return HZ_OK;
}

const char* hz_kernel_family_name(int family) { return family_name(family); }
int hz_kernel_family_count(void) { return F_COUNT; }

}  // extern "C"
