// Host runtime of the library: hierarchy set-up, workspace, and the solver drivers of
// Algorithm 1 (recursive deflated FGMRES with the MADP schedule of Section 4.4).
//
// Every vector operation runs in the CUDA kernels of kern_stencil.cu / kern_vec.cu.  The
// host holds only scalars: the Hessenberg matrices of the Krylov cycles, their Givens
// rotations and least-squares solutions (Algorithm 1 line 22), and the stopping tests.
// A batch of nb right-hand sides advances in lockstep; each right-hand side keeps its own
// Hessenberg matrix, stopping iteration and solution, so its result does not depend on
// the rest of the batch.
#include "hz_core.h"

#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <tuple>
#include <string>
#include <thread>
#include <unordered_map>

namespace hz {

// ---------------------------------------------------------------------------------- errors
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
const char* last_error_message() { return g_err.c_str(); }

cudaError_t ensure_dyn_smem(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::unordered_map<const void*, size_t> limit;
  if (bytes <= 48 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = limit[func];
  if (cur >= bytes) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) cur = bytes;
  return e;
}

int status_of(cudaError_t e, const char* where) {
  if (e == cudaSuccess) return HZ_OK;
  set_error(std::string(where) + ": " + cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HZ_ENOMEM : HZ_ECUDA;
}

#define CK(expr)                                          \
  do {                                                    \
    int s_ = ::hz::status_of((expr), #expr);              \
    if (s_) return s_;                                    \
  } while (0)
#define CS(expr)          \
  do {                    \
    int s_ = (expr);      \
    if (s_) return s_;    \
  } while (0)

static const char* kFamilies[F_COUNT] = {"level_op", "mg_down", "mg_up",  "defl_restrict", "defl_prolong",
                                         "multidot", "axpy",    "reduce", "dense",         "misc",
                                         "gmres_persistent", "bicgstab_persistent"};
const char* family_name(int f) { return (f >= 0 && f < F_COUNT) ? kFamilies[f] : "?"; }

// ---------------------------------------------------------------------------------- profiler
cudaEvent_t Prof::get() {
  if (pool.empty()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}
void Prof::drain(int fam) {
  for (auto& r : pending[fam]) {
    float ms_ = 0;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms_, r.a, r.b) == cudaSuccess) {
      ms[fam] += ms_;
      launches[fam] += 1;
      bytes[fam] += r.bytes;
      int lv = (r.level >= 0 && r.level < kProfLevels) ? r.level : 0;
      ms_lv[fam][lv] += ms_;
      launches_lv[fam][lv] += 1;
      bytes_lv[fam][lv] += r.bytes;
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending[fam].clear();
}
Prof::~Prof() {
  for (int f = 0; f < F_COUNT; ++f)
    for (auto& r : pending[f]) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
  for (auto e : pool) cudaEventDestroy(e);
}
ProfScope::ProfScope(Ctx& c_, int fam_, double bytes_) : c(c_), fam(fam_), bytes(bytes_), level(c_.level) {
  if (c.prof) c.prof->total_launches += 1;
  if (c.prof && c.prof->on[fam]) {
    a = c.prof->get();
    if (a) cudaEventRecord(a, c.s);
  }
}
ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b = c.prof->get();
  if (!b) return;
  cudaEventRecord(b, c.s);
  c.prof->pending[fam].push_back({a, b, bytes, level});
  if (c.prof->pending[fam].size() > 8192) c.prof->drain(fam);
}

// ---------------------------------------------------------------------------------- helpers
int dalloc(Handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return HZ_OK;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
    *p = nullptr;
    return HZ_ENOMEM;
  }
  h->allocs.push_back(*p);
  h->bytes += bytes;
  return HZ_OK;
}

int wait_event(Handle* h, cudaEvent_t ev) {
  CK(cudaEventRecord(ev, h->ctx.s));
  auto t0 = std::chrono::steady_clock::now();
  long spins = 0;
  for (;;) {
    cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return HZ_OK;
    if (e != cudaErrorNotReady) return status_of(e, "cudaEventQuery");
    if (++spins > 2000) {
      std::this_thread::yield();
      double s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (s > h->cfg.timeout_s) {
        set_error("device wait exceeded the configured timeout");
        return HZ_ETIMEOUT;
      }
    }
  }
}

static int krylov_cap(double c_it, size_t nodes) { return (int)std::floor(c_it * std::pow((double)nodes, 0.25)); }

// Deflated FGMRES schedule of level l (Algorithm 1 with the MADP schedule of Section 4.4 and its
// variants): the relative tolerance (0 = run exactly `cap` iterations) and the iteration cap.
//   level 1      : tolerance of the solve call, cap = restart length (set by the caller);
//   level ml     : one iteration when negative definite, else coarsest_tol within the Krylov cap
//                  (Section 4.1);
//   level 2      : l2_tol within l2_maxit;
//   levels 3..ml-1: level_tol[l-1] within l2_maxit where set (Sections 4.3.3, 4.5), else
//                  exactly cycle_m iterations (m = 1 V-cycle, m = 2 W-cycle, Section 3.2).
static void level_schedule(const hz_config& cfg, int l, size_t nodes, double* tol, int* cap) {
  const int ml = cfg.levels;
  if (l == 1) {
    *tol = 0.0;
    *cap = cfg.restart;
  } else if (l == ml) {
    const bool negdef = cfg.negdef_from_level > 0 && l >= cfg.negdef_from_level;
    *tol = negdef ? 0.0 : cfg.coarsest_tol;
    *cap = negdef ? 1 : krylov_cap(cfg.c_it, nodes);
  } else if (l == 2) {
    *tol = cfg.l2_tol;
    *cap = cfg.l2_maxit;
  } else if (cfg.level_tol[l - 1] > 0) {
    *tol = cfg.level_tol[l - 1];
    *cap = cfg.l2_maxit;
  } else {
    *tol = 0.0;
    *cap = cfg.cycle_m;
  }
  *cap = std::max(*cap, 1);
}

OpDesc Level::opA(int dt) const {
  OpDesc d;
  d.nx = nx;
  d.ny = ny;
  d.R = R;
  d.bc = bc;
  d.H = H;
  d.ks = ks;
  d.c = ks / (H * H);  // = 1 / h^2 on every level (Galerkin scale 4^(l-1) over H_l^2)
  d.sr = 1;
  d.si = 0;
  for (int i = 0; i < 7; ++i) {
    d.m[i] = m[i];
    d.l[i] = L[i];
  }
  d.k_d = k_d;
  d.k_f = k_f;
  d.kstride = kstride;
  (void)dt;
  return d;
}

// The operator of right-hand side q alone (its own wavenumber field), for launches on one
// right-hand side.
static OpDesc op_of_rhs(const OpDesc& d, int q) {
  OpDesc o = d;
  if (d.kstride) {
    o.k_d += (size_t)q * d.kstride;
    o.k_f += (size_t)q * d.kstride;
    o.kstride = 0;
  }
  return o;
}
OpDesc Level::opM(int dt, double b1, double b2) const {
  OpDesc d = opA(dt);
  d.sr = b1;
  d.si = b2;
  return d;
}

static int alloc_scalars(Handle* h, Scalars& s, int cap, int nb) {
  s.hA = 0;
  size_t per = (size_t)nb * 2 * (cap + 1);
  s.hB = per;
  s.nrm = 2 * per;
  s.csc = s.nrm + nb;
  s.ccomb = s.csc + 2 * (size_t)nb;
  s.total = s.ccomb + (size_t)nb * 2 * (cap + 1);
  void* p;
  CS(dalloc(h, &p, s.total * sizeof(double)));
  s.dev = reinterpret_cast<double*>(p);
  CK(cudaMallocHost((void**)&s.host, s.total * sizeof(double)));
  CK(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
  return HZ_OK;
}

static void free_scalars(Scalars& s) {
  if (s.host) cudaFreeHost(s.host);
  if (s.ev) cudaEventDestroy(s.ev);
  s.host = nullptr;
  s.ev = nullptr;
}

// Gauss-Jordan inverse with partial pivoting (row-major n x n, in place).
static bool invert(std::vector<cd>& A, int n) {
  std::vector<cd> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int p = c;
    double best = std::abs(A[(size_t)c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (std::abs(A[(size_t)r * n + c]) > best) {
        best = std::abs(A[(size_t)r * n + c]);
        p = r;
      }
    if (!(best > 0)) return false;
    if (p != c)
      for (int k = 0; k < n; ++k) {
        std::swap(A[(size_t)p * n + k], A[(size_t)c * n + k]);
        std::swap(I[(size_t)p * n + k], I[(size_t)c * n + k]);
      }
    cd piv = 1.0 / A[(size_t)c * n + c];
    for (int k = 0; k < n; ++k) {
      A[(size_t)c * n + k] *= piv;
      I[(size_t)c * n + k] *= piv;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      cd f = A[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int k = 0; k < n; ++k) {
        A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
        I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
      }
    }
  }
  A.swap(I);
  return true;
}

// Dense inverse of a grid operator: columns from the FP64 level kernel applied to unit vectors.
// With per-right-hand-side wavenumbers (op.kstride != 0) one inverse per field, `ninst` of them
// back to back.
static int dense_inverse(Handle* h, const OpDesc& op_all, int ninst, double** inv_out) {
  const int N = (int)op_all.n();
  if (N > 2048) {
    set_error("multigrid coarsest grid has " + std::to_string(N) + " unknowns (limit 2048)");
    return HZ_ENOTSUP;
  }
  size_t bytes = (size_t)N * N * 16;
  void *E = nullptr, *Y = nullptr;
  CK(cudaMalloc(&E, bytes));
  if (cudaMalloc(&Y, bytes) != cudaSuccess) {
    cudaFree(E);
    return status_of(cudaErrorMemoryAllocation, "dense_inverse");
  }
  void* p = nullptr;
  int st = dalloc(h, &p, bytes * (op_all.kstride ? ninst : 1));
  std::vector<cd> unit((size_t)N * N, 0.0), cols((size_t)N * N), A((size_t)N * N);
  for (int i = 0; i < N; ++i) unit[(size_t)i * N + i] = 1.0;
  cudaError_t e = cudaMemcpyAsync(E, unit.data(), bytes, cudaMemcpyHostToDevice, h->ctx.s);
  for (int q = 0; q < (op_all.kstride ? ninst : 1) && st == HZ_OK && e == cudaSuccess; ++q) {
    e = launch_level_op(h->ctx, op_of_rhs(op_all, q), 0, C128, C128, C128, E, nullptr, Y, 0.0, N);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cols.data(), Y, bytes, cudaMemcpyDeviceToHost, h->ctx.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->ctx.s);
    if (e != cudaSuccess) break;
    for (int c = 0; c < N; ++c)
      for (int r = 0; r < N; ++r) A[(size_t)r * N + c] = cols[(size_t)c * N + r];
    if (!invert(A, N)) {
      set_error("singular multigrid coarsest operator");
      st = HZ_EBREAKDOWN;
      break;
    }
    e = cudaMemcpyAsync((char*)p + (size_t)q * bytes, A.data(), bytes, cudaMemcpyHostToDevice, h->ctx.s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->ctx.s);
  }
  cudaFree(E);
  cudaFree(Y);
  if (e != cudaSuccess) return status_of(e, "dense_inverse");
  if (st) return st;
  *inv_out = reinterpret_cast<double*>(p);
  return HZ_OK;
}

static int upload_k(Handle* h, const std::vector<double>& k, double** kd, float** kf) {
  void* p;
  CS(dalloc(h, &p, k.size() * 8));
  *kd = reinterpret_cast<double*>(p);
  CK(cudaMemcpyAsync(p, k.data(), k.size() * 8, cudaMemcpyHostToDevice, h->ctx.s));
  std::vector<float> kf32(k.size());
  for (size_t i = 0; i < k.size(); ++i) kf32[i] = (float)k[i];
  CS(dalloc(h, &p, k.size() * 4));
  *kf = reinterpret_cast<float*>(p);
  CK(cudaMemcpyAsync(p, kf32.data(), k.size() * 4, cudaMemcpyHostToDevice, h->ctx.s));
  CK(cudaStreamSynchronize(h->ctx.s));
  return HZ_OK;
}

// Nodes per side of the next coarser grid: vertex grids keep their boundary nodes (coarse node I
// at fine node 2I), homogeneous Dirichlet grids hold interior unknowns only (coarse unknown I at
// fine unknown 2I + 1).
static int coarse_side(int n, int bc) { return bc == HZ_BC_DIRICHLET ? (n - 1) / 2 : (n + 1) / 2; }

// The multigrid CSLP coarsens while both sides are odd, above the coarsest side and large enough
// to halve (a vertex grid keeps at least 3 nodes, a Dirichlet grid at least 1 unknown).
static bool mg_coarsens(int mx, int my, int coarsest_side, int bc) {
  if (std::min(mx, my) <= coarsest_side || (mx - 1) % 2 || (my - 1) % 2) return false;
  return std::min(mx, my) >= (bc == HZ_BC_DIRICHLET ? 3 : 5);
}

// Wavenumbers of the next coarser grid: injection at the coincident nodes, for each of the
// `nf` fields stored back to back.
static std::vector<double> inject(const std::vector<double>& k, int nx, int ny, int bc, int nf = 1) {
  const int cx = coarse_side(nx, bc), cy = coarse_side(ny, bc), o = bc == HZ_BC_DIRICHLET ? 1 : 0;
  std::vector<double> out((size_t)nf * cx * cy);
  for (int f = 0; f < nf; ++f) {
    const double* kf = k.data() + (size_t)f * nx * ny;
    double* of = out.data() + (size_t)f * cx * cy;
    for (int j = 0; j < cy; ++j)
      for (int i = 0; i < cx; ++i) of[(size_t)j * cx + i] = kf[(size_t)(2 * j + o) * nx + 2 * i + o];
  }
  return out;
}

// Cooperative grid of the persistent GMRES kernel: one CTA per 32 x 16 stencil tile and at
// least ~256 nodes per CTA slice, at most one CTA per SM (every grid barrier then serialises
// at most #SM arrivals).
// With device_gmres = 1, calls on at least kClusterMinRhs right-hand sides of a level with at
// most kClusterMaxN nodes run the persistent GMRES as one thread-block cluster per right-hand
// side (all at once); otherwise the cooperative grid runs per right-hand side.  A 16-CTA cluster
// alone streams far less than the whole GPU (measured on GB300: 513^2, 9 iterations, 1 rhs
// 0.92 ms cluster vs 0.36 ms grid; 8 rhs 2.28 ms vs 2.67 ms; at 1025^2 the grid wins at 8 rhs).
constexpr int kClusterMinRhs = 4;
constexpr size_t kClusterMaxN = 300000;

// The cluster form may run on a level of n nodes (it then needs per-rhs GMRES workspace), for
// FP32 and FP64 vectors alike.
static bool cluster_form_possible(const hz_config& cfg, size_t n) {
  if (cfg.cslp_solver != HZ_CSLP_GMRES) return false;
  return cfg.device_gmres == 3 || (cfg.device_gmres == 1 && cfg.max_rhs >= kClusterMinRhs && n <= kClusterMaxN);
}

int gmres_grid_want(int nx, int ny) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const long long n = (long long)nx * ny;
  return (int)std::min<long long>(sms, std::max<long long>(((nx + 31) / 32) * ((ny + 15) / 16), (n + 255) / 256));
}

// Device bytes hz_setup allocates for this grid and configuration (an upper bound: the
// cooperative grid is taken at its largest), used for admission against a memory budget.
size_t estimate_bytes(const hz_grid& g, const hz_config& cfg) {
  const int ml = cfg.levels, nb = cfg.max_rhs;
  const size_t nf = cfg.per_rhs_k ? (size_t)nb : 1;  // wavenumber fields
  const bool mixed = cfg.precision == HZ_PREC_MIXED;
  size_t total = 0, maxnv = 2;
  if (cfg.sym_rows) total += (size_t)nb * g.nx * g.ny * 16;  // D b
  auto scal = [&](int cap) { return sizeof(double) * ((size_t)nb * 4 * (cap + 1) + 3 * (size_t)nb + 2 * (size_t)nb * (cap + 1)); };
  int nx = g.nx, ny = g.ny;
  for (int l = 1; l <= ml; ++l) {
    const size_t n = (size_t)nx * ny, bn = (size_t)nb * n;
    const size_t eb = (l == 1 || !mixed) ? 16 : 8, ep = mixed ? 8 : 16, ex = ep;
    total += n * 12 * nf;  // k in FP64 and FP32 (per field)
    int cap;
    double tol_unused;
    level_schedule(cfg, l, n, &tol_unused, &cap);
    maxnv = std::max(maxnv, (size_t)cap + 1);
    total += (cap + 1) * bn * eb + cap * bn * ex + bn * eb + 3 * bn * ep + (l >= 2 ? 2 * bn * eb : 0) + scal(cap);
    if (l >= 2 && cap == 1) total += sizeof(int) * 2 * (size_t)nb;  // one-iteration counters
    if (l <= cfg.mg_max_level) {
      int mx = nx, my = ny;
      const bool general = !(cfg.mg_nu1 == 1 && cfg.mg_nu2 == 1);
      if (general) total += 2 * bn * ep;
      for (;;) {
        if (!mg_coarsens(mx, my, cfg.mg_coarsest_side, g.bc)) break;
        mx = coarse_side(mx, g.bc);
        my = coarse_side(my, g.bc);
        const size_t m = (size_t)mx * my;
        total += m * 12 * nf + 2 * (size_t)nb * m * ep + (general ? 2 * (size_t)nb * m * ep : 0);
      }
      const size_t nc = (size_t)mx * my;
      total += nc * nc * 16 * nf;
    } else {
      const int capg = std::max(1, krylov_cap(cfg.c_it, n));
      maxnv = std::max(maxnv, (size_t)capg + 1);
      const bool bicg = cfg.cslp_solver == HZ_CSLP_BICGSTAB;
      const bool dev = cfg.device_gmres != 0 && !bicg;
      if (bicg)
        total += std::max(5 * bn, 7 * n) * ep + sizeof(BicgState) * (size_t)nb + bicg_part_bytes(n, nb) +
                 (cfg.device_gmres ? sizeof(BicgBarrier) + sizeof(double) * 8 * 1024 : 0);
      // upper bound: the cluster form keeps per-rhs workspace
      const bool clus = cluster_form_possible(cfg, n);
      const size_t gbr = (dev && !clus) ? n : bn;
      const size_t gq = clus ? (size_t)nb : 1;
      total += (capg + 1) * gbr * ep + gbr * ep + scal(bicg ? std::max(capg, 2) : capg);
      if (dev) {
        const size_t ps = 2 * (size_t)(capg + 1) + 2;
        total += gq * n * ep + 2 * sizeof(double) * std::max<size_t>(152, 16 * gq) * ps +
                 sizeof(unsigned) * std::max<size_t>(152, 16 * gq) +
                 sizeof(double) * gq * (2 * (size_t)capg * (capg + 1) + 2 * (size_t)capg + 3 * ps) +
                 sizeof(GmresState) * nb;
      }
    }
    if (l < ml) {
      nx = coarse_side(nx, g.bc);
      ny = coarse_side(ny, g.bc);
    }
  }
  total += dot_ws_bytes((int)maxnv, nb) + scal(1) + (size_t)nb * g.nx * g.ny * 16 + sizeof(int);
  return total;
}

// ---------------------------------------------------------------------------------- set-up
int setup(Handle* h, const double* k_dev) {
  const hz_grid& g = h->g;
  hz_config& cfg = h->cfg;
  const int ml = cfg.levels;
  h->nbmax = cfg.max_rhs;
  const int nb = h->nbmax;
  const bool mixed = cfg.precision == HZ_PREC_MIXED;
  CK(cudaGetDevice(&h->device));
  // host copy of k (one field, or one per right-hand side), validated
  const int nf = cfg.per_rhs_k ? nb : 1;
  std::vector<double> k((size_t)nf * g.nx * g.ny);
  CK(cudaMemcpy(k.data(), k_dev, k.size() * 8, cudaMemcpyDeviceToHost));
  for (double v : k)
    if (!(std::isfinite(v) && v > 0)) {
      set_error("wavenumber field must be finite and positive");
      return HZ_EINVAL;
    }
  h->lv.resize(ml);
  int nx = g.nx, ny = g.ny;
  std::vector<double> kl = k;
  for (int l = 1; l <= ml; ++l) {
    Level& L = h->lv[l - 1];
    L.l = l;
    L.bc = g.bc;
    L.nx = nx;
    L.ny = ny;
    L.n = (size_t)nx * ny;
    L.H = std::ldexp(g.h, l - 1);
    L.ks = std::ldexp(1.0, 2 * (l - 1));
    galerkin_masks(l, &L.R, L.m, L.L);
    CS(upload_k(h, kl, &L.k_d, &L.k_f));
    L.kstride = cfg.per_rhs_k ? L.n : 0;
    if (l == 1) {
      L.dvec = C128;
      L.dpre = mixed ? C64 : C128;
      L.dx = L.dpre;
    } else {
      L.dvec = L.dpre = L.dx = mixed ? C64 : C128;
    }
    if (l < ml) {
      kl = inject(kl, nx, ny, g.bc, nf);
      nx = coarse_side(nx, g.bc);
      ny = coarse_side(ny, g.bc);
    }
  }
  // per-level workspace
  size_t maxnv = 2;
  for (int l = 1; l <= ml; ++l) {
    Level& L = h->lv[l - 1];
    const size_t eb = elem_bytes(L.dvec), ep = elem_bytes(L.dpre), ex = elem_bytes(L.dx);
    const size_t bn = (size_t)nb * L.n;
    level_schedule(cfg, l, L.n, &L.tol, &L.cap);
    maxnv = std::max(maxnv, (size_t)L.cap + 1);
    CS(dalloc(h, &L.V, (L.cap + 1) * bn * eb));
    CS(dalloc(h, &L.X, L.cap * bn * ex));
    CS(dalloc(h, &L.w, bn * eb));
    CS(dalloc(h, &L.t, bn * ep));
    CS(dalloc(h, &L.rt, bn * ep));
    CS(dalloc(h, &L.r, bn * ep));
    if (l >= 2) {
      CS(dalloc(h, &L.b, bn * eb));
      CS(dalloc(h, &L.x, bn * eb));
    }
    CS(alloc_scalars(h, L.sc, L.cap, nb));
    if (l >= 2 && L.cap == 1) {  // one-iteration cycles run without a host round trip
      void* p;
      CS(dalloc(h, &p, sizeof(int) * 2 * (size_t)nb));
      L.m1cnt = (int*)p;
      CK(cudaMemsetAsync(L.m1cnt, 0, sizeof(int) * 2 * (size_t)nb, h->ctx.s));
    }
    if (l <= cfg.mg_max_level) {
      // multigrid CSLP hierarchy (level 0 = this deflation level)
      MGLevel m0;
      m0.op = L.opM(L.dpre, cfg.beta1, cfg.beta2);
      L.mg.push_back(m0);
      // wavenumber of this level on the host again (inject from fine k)
      std::vector<double> km = k;
      {
        int fx = g.nx, fy = g.ny;
        for (int q = 1; q < l; ++q) {
          km = inject(km, fx, fy, g.bc, nf);
          fx = coarse_side(fx, g.bc);
          fy = coarse_side(fy, g.bc);
        }
      }
      int mx = L.nx, my = L.ny;
      double Hm = L.H;
      const bool general = !(cfg.mg_nu1 == 1 && cfg.mg_nu2 == 1);
      for (;;) {
        if (!mg_coarsens(mx, my, cfg.mg_coarsest_side, g.bc)) break;
        km = inject(km, mx, my, g.bc, nf);
        mx = coarse_side(mx, g.bc);
        my = coarse_side(my, g.bc);
        Hm *= 2.0;
        MGLevel q;
        q.op.nx = mx;
        q.op.ny = my;
        q.op.R = 1;
        q.op.bc = g.bc;
        q.op.c = L.ks / (Hm * Hm);
        q.op.H = Hm;
        q.op.ks = L.ks;
        q.op.sr = cfg.beta1;
        q.op.si = cfg.beta2;
        double* kd;
        float* kf;
        CS(upload_k(h, km, &kd, &kf));
        q.op.k_d = kd;
        q.op.k_f = kf;
        q.op.kstride = cfg.per_rhs_k ? (size_t)mx * my : 0;
        CS(dalloc(h, &q.f, (size_t)nb * mx * my * ep));
        CS(dalloc(h, &q.e, (size_t)nb * mx * my * ep));
        L.mg.push_back(q);
      }
      if (general)
        for (auto& q : L.mg) {
          CS(dalloc(h, &q.tmp, (size_t)nb * q.op.n() * ep));
          CS(dalloc(h, &q.tmp2, (size_t)nb * q.op.n() * ep));
        }
      OpDesc last = L.mg.back().op;
      L.ninv = (int)last.n();
      L.invstride = last.kstride ? (size_t)L.ninv * L.ninv : 0;
      CS(dense_inverse(h, last, nf, &L.inv));
    } else {
      L.capg = std::max(1, krylov_cap(cfg.c_it, L.n));
      maxnv = std::max(maxnv, (size_t)L.capg + 1);
      if (cfg.cslp_solver == HZ_CSLP_BICGSTAB) {
        void* p;
        // launch-per-step kernels: r, p, v, s, t batches; persistent form: r, two p, two v, s, t of
        // one right-hand side at a time
        CS(dalloc(h, &L.bcg, std::max(5 * bn, 7 * L.n) * ep));
        CS(dalloc(h, &p, sizeof(BicgState) * (size_t)nb));
        L.bst = (BicgState*)p;
        CK(cudaMemsetAsync(L.bst, 0, sizeof(BicgState) * (size_t)nb, h->ctx.s));
        CS(dalloc(h, &p, bicg_part_bytes(L.n, nb)));
        L.bpart = (double*)p;
        if (cfg.device_gmres) {
          L.bgrid = std::min(bicg_persist_grid(L.dpre, L.R, L.nx, L.ny), 1024);
          if (L.bgrid > 0) {
            CS(dalloc(h, &p, sizeof(BicgBarrier)));
            L.bbar = (BicgBarrier*)p;
            CK(cudaMemsetAsync(L.bbar, 0, sizeof(BicgBarrier), h->ctx.s));
            CS(dalloc(h, &p, sizeof(double) * 8 * (size_t)L.bgrid));
            L.bgpart = (double*)p;
          }
        }
      } else if (cfg.device_gmres) {
        L.ggrid = std::min(gmres_max_grid(L.dpre, L.R, L.capg, L.n), gmres_grid_want(L.nx, L.ny));
        L.gcl = cluster_form_possible(cfg, L.n) ? gmres_cluster_size(L.dpre, L.R, L.capg) : 0;
        // one right-hand side at a time on levels whose tiling fits the grid: tile-owned form
        // (FP32 vectors; the FP64 variant is register-bound)
        if ((cfg.device_gmres == 1 || cfg.device_gmres == 2) && L.dpre == C64)
          L.gtiles = gmres_tile_form(L.dpre, L.R, L.nx, L.ny, L.capg, &L.gtx, &L.gty);
        if (L.ggrid <= 0 && L.gcl <= 0) {
          set_error("the persistent GMRES kernel cannot be launched on this device");
          return HZ_ENOTSUP;
        }
      }
      // the cooperative grid solves one right-hand side at a time (its workspace holds one rhs);
      // the cluster form solves all nb at once (workspace per rhs)
      const bool dev = L.ggrid > 0 || L.gcl > 0;
      const size_t gb_rhs = (dev && !L.gcl) ? L.n : bn;
      const size_t gq = L.gcl ? (size_t)nb : 1;
      CS(dalloc(h, &L.Vg, (L.capg + 1) * gb_rhs * ep));
      CS(dalloc(h, &L.wg, gb_rhs * ep));
      // (the Bi-CGSTAB stop flags come back through this buffer: at least two columns' worth)
      CS(alloc_scalars(h, L.scg, cfg.cslp_solver == HZ_CSLP_BICGSTAB ? std::max(L.capg, 2) : L.capg, nb));
      if (dev) {
        void* p;
        CS(dalloc(h, &L.wg2, gq * L.n * ep));
        L.gpstride = 2 * (L.capg + 1) + 2;
        const size_t nparts = std::max<size_t>(std::max<size_t>(L.ggrid, L.gtiles), gq * L.gcl);
        CS(dalloc(h, &p, sizeof(double) * nparts * L.gpstride));
        L.gpartA = (double*)p;
        CS(dalloc(h, &p, sizeof(double) * nparts * L.gpstride));
        L.gpartB = (double*)p;
        CS(dalloc(h, &p, sizeof(double) * gq * (2 * (size_t)L.capg * (L.capg + 1) + 2 * (size_t)L.capg +
                                                3 * (size_t)L.gpstride)));
        L.gR = (double*)p;
        CS(dalloc(h, &p, sizeof(GmresState) * nb));
        L.gst = (GmresState*)p;
        CS(dalloc(h, &p, sizeof(unsigned) * nparts));
        L.gflag = (unsigned*)p;
        CK(cudaMemsetAsync(L.gflag, 0, sizeof(unsigned) * nparts, h->ctx.s));
        CK(cudaMemsetAsync(L.gst, 0, sizeof(GmresState) * nb, h->ctx.s));
      }
    }
  }
  h->ws_bytes = dot_ws_bytes((int)maxnv, nb);
  CS(dalloc(h, &h->ws, h->ws_bytes));
  CS(alloc_scalars(h, h->outer_sc, 1, nb));
  CS(dalloc(h, &h->rres, (size_t)nb * h->lv[0].n * 16));
  if (cfg.sym_rows) CS(dalloc(h, &h->bscaled, (size_t)nb * h->lv[0].n * 16));
  {
    void* p;
    CS(dalloc(h, &p, sizeof(int)));
    h->derr = (int*)p;
    CK(cudaMemsetAsync(h->derr, 0, sizeof(int), h->ctx.s));
  }
  h->st.assign(nb, RhsStats());
  CS(noalloc_prepare(h));
  CK(cudaStreamSynchronize(h->ctx.s));
  if (cfg.device_gmres == 1 && cfg.autotune) CS(autotune_gmres(h));
  if (cfg.device_gmres == 1 && cfg.autotune) CS(autotune_batch(h));
  if (cfg.autotune) CS(autotune_mg(h));
  // the first level >= 3 from which every level runs one-iteration device cycles and a device
  // CSLP inverse (multigrid or persistent GMRES): its coarse solve issues no host decision
  if (cfg.graphs) {
    for (int l = ml; l >= 3; --l) {
      const Level& L = h->lv[l - 1];
      const bool dev_cslp = l <= cfg.mg_max_level || L.ggrid > 0 || L.gcl > 0 || L.gtiles > 0 || L.bgrid > 0;
      if (!(L.cap == 1 && L.m1cnt && dev_cslp)) break;
      h->graph_level = l;
    }
    h->graph_exec.assign(nb, nullptr);
    h->graph_launches.assign(nb, 0);
    if (h->graph_level > 0) CK(cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking));
  }
  return HZ_OK;
}

// ------------------------------------------------------------------------------ autotuning
// Per level shape (nx, ny, precision, stencil radius, iteration cap) the fastest GMRES form among
// the tile-owned form at every fitting tile shape (fewer, larger tiles mean fewer CTAs at each
// grid barrier) and the slice-distributed grid, measured once per process: each runs
// min(cap, 24) iterations (tolerance 0) on a fixed pseudo-random right-hand side, twice, and the
// second run's event time decides.  The workspace of the level is reused; statistics are reset.
namespace {
std::mutex g_tune_mu;
// (nx, ny, precision, radius, cap) -> fastest form: tile shape (TX, TY), or (0, 0) for the
// slice-distributed grid
std::map<std::tuple<int, int, int, int, int>, std::pair<int, int>> g_tune;

// (nx, ny, precision, radius, cap, batch) -> CTAs per cluster of the cluster form for a batch of
// that many right-hand sides, or 0 when one right-hand side at a time on the whole grid was faster
std::map<std::tuple<int, int, int, int, int, int>, int> g_tune_batch;

// tiles along a side of n nodes for tile width t (the last tile takes the remainder node)
static int tile_count(int n, int t) { return n > 1 ? (n - 1 + t - 1) / t : 1; }

// Fill the first nb right-hand sides of a level's CSLP input (L.t) with one fixed pseudo-random
// vector (xorshift32, values in [-1, 1)).
static int fill_tune_input(Handle* h, Level& L, int nb) {
  const size_t eb = elem_bytes(L.dpre);
  std::vector<float> hb(2 * L.n);
  uint32_t r = 12345u;
  for (auto& v : hb) {
    r ^= r << 13;
    r ^= r >> 17;
    r ^= r << 5;
    v = (float)((double)r / 2147483648.0 - 1.0);
  }
  std::vector<double> hd;
  if (eb == 16) hd.assign(hb.begin(), hb.end());
  const void* src = eb == 16 ? (const void*)hd.data() : (const void*)hb.data();
  for (int q = 0; q < nb; ++q)
    CK(cudaMemcpyAsync((char*)L.t + (size_t)q * L.n * eb, src, L.n * eb, cudaMemcpyHostToDevice, h->ctx.s));
  CK(cudaStreamSynchronize(h->ctx.s));
  return HZ_OK;
}
}  // namespace

int autotune_gmres(Handle* h) {
  for (auto& L : h->lv) {
    if (L.gtiles <= 0 || L.ggrid <= 0) continue;
    const auto key = std::make_tuple(L.nx, L.ny, L.dpre, L.R, L.capg);
    auto adopt = [&](int TX, int TY) {
      if (TX <= 0) {
        L.gtiles = 0;  // slice-distributed grid
        return;
      }
      L.gtx = TX;
      L.gty = TY;
      L.gtiles = tile_count(L.nx, TX) * tile_count(L.ny, TY);
    };
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune.find(key);
      if (it != g_tune.end()) {
        adopt(it->second.first, it->second.second);
        continue;
      }
    }
    const size_t eb = elem_bytes(L.dpre);
    std::vector<float> hb(2 * L.n);
    uint32_t r = 12345u;
    for (auto& v : hb) {  // xorshift32, values in [-1, 1)
      r ^= r << 13;
      r ^= r >> 17;
      r ^= r << 5;
      v = (float)((double)r / 2147483648.0 - 1.0);
    }
    if (eb == 16) {
      std::vector<double> hd(hb.begin(), hb.end());
      CK(cudaMemcpyAsync(L.t, hd.data(), L.n * eb, cudaMemcpyHostToDevice, h->ctx.s));
      CK(cudaStreamSynchronize(h->ctx.s));
    } else {
      CK(cudaMemcpyAsync(L.t, hb.data(), L.n * eb, cudaMemcpyHostToDevice, h->ctx.s));
      CK(cudaStreamSynchronize(h->ctx.s));
    }
    OpDesc M = op_of_rhs(L.opM(L.dpre, h->cfg.beta1, h->cfg.beta2), 0);
    const int K = std::min(L.capg, 24);
    const double eta2 = h->cfg.reorth_eta >= 1.0 ? 2.0 : h->cfg.reorth_eta * h->cfg.reorth_eta;
    // candidates: every fitting tile shape (at most as many tiles as the setup's default, whose
    // partial-sum buffers are sized for it), then the slice-distributed grid (TX = 0)
    int tx[5], ty[5];
    const int ntile = gmres_tile_forms(L.dpre, L.R, L.nx, L.ny, L.capg, tx, ty, 4);
    int nc = 0;
    for (int i = 0; i < ntile; ++i)
      if (tile_count(L.nx, tx[i]) * tile_count(L.ny, ty[i]) <= L.gtiles) {
        tx[nc] = tx[i];
        ty[nc++] = ty[i];
      }
    tx[nc] = 0;
    ty[nc++] = 0;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<float> ms(nc, 0.0f);
    int st = HZ_OK;
    for (int c = 0; c < nc && st == HZ_OK; ++c) {
      for (int rep = 0; rep < 2 && st == HZ_OK; ++rep) {
        st = status_of(cudaMemsetAsync(L.rt, 0, L.n * eb, h->ctx.s), "autotune");
        if (st) break;
        st = status_of(cudaEventRecord(e0, h->ctx.s), "autotune");
        if (st) break;
        cudaError_t e = tx[c] > 0 ? launch_gmres_tile(h->ctx, M, L.dpre, L.t, L.rt, L.Vg, L.wg, L.gflag, L.gpartA,
                                                      L.gpartB, L.gR, L.gst, K, 0.0, tx[c], ty[c], eta2)
                                  : launch_gmres_persistent(h->ctx, M, L.dpre, L.t, L.rt, L.Vg, L.wg, L.wg2, L.gpartA,
                                                            L.gpartB, L.gpstride, L.gR, L.gst, K, 0.0, L.ggrid, false,
                                                            1, eta2);
        st = status_of(e, "autotune launch");
        if (st) break;
        st = status_of(cudaEventRecord(e1, h->ctx.s), "autotune");
        if (st) break;
        st = wait_event(h, e1);
        if (st) break;
        st = status_of(cudaEventElapsedTime(&ms[c], e0, e1), "autotune");  // the second run counts
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    GmresState gs;
    CK(cudaMemcpy(&gs, L.gst, sizeof(gs), cudaMemcpyDeviceToHost));
    CK(cudaMemsetAsync(L.gst, 0, sizeof(GmresState) * h->nbmax, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    if (gs.err) {
      set_error("a grid barrier of the persistent GMRES kernel exceeded its wait budget");
      return HZ_ETIMEOUT;
    }
    int best = 0;
    for (int c = 1; c < nc; ++c)
      if (ms[c] < ms[best]) best = c;
    adopt(tx[best], ty[best]);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[key] = {tx[best], ty[best]};
  }
  return HZ_OK;
}

// Band heights of the radius-1 multigrid sweeps, timed once per level shape and precision on the
// handle's own multigrid buffers (their contents are rewritten by every V-cycle before use).
// Batches of max_rhs >= kClusterMinRhs right-hand sides on levels that can run the cluster form:
// time the batch as one launch with clusters of 16, 8 and 4 CTAs (a cluster per right-hand side;
// with 16 right-hand sides, clusters of 16 need two waves on 152 SMs, clusters of 8 fit in one)
// and as one whole-grid launch per right-hand side, min(cap, 24) iterations each, twice; keep
// the fastest per level shape and batch size.
int autotune_batch(Handle* h) {
  const int nb = h->nbmax;
  if (nb < kClusterMinRhs) return HZ_OK;
  for (auto& L : h->lv) {
    if (L.gcl <= 0) continue;
    const auto key = std::make_tuple(L.nx, L.ny, L.dpre, L.R, L.capg, nb);
    auto adopt = [&](int C) {
      if (C > 0) {
        L.gcl = C;
      } else {
        L.gseq = true;
      }
    };
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_batch.find(key);
      if (it != g_tune_batch.end()) {
        adopt(it->second);
        continue;
      }
    }
    CS(fill_tune_input(h, L, nb));
    const size_t eb = elem_bytes(L.dpre);
    const OpDesc M = L.opM(L.dpre, h->cfg.beta1, h->cfg.beta2);
    const int K = std::min(L.capg, 24);
    const double eta2 = h->cfg.reorth_eta >= 1.0 ? 2.0 : h->cfg.reorth_eta * h->cfg.reorth_eta;
    std::vector<int> cand;
    for (int C = L.gcl; C >= 4; C /= 2) cand.push_back(C);
    if (L.ggrid > 0) cand.push_back(0);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    std::vector<float> ms(cand.size(), 0.0f);
    int st = HZ_OK;
    for (size_t c = 0; c < cand.size() && st == HZ_OK; ++c) {
      for (int rep = 0; rep < 2 && st == HZ_OK; ++rep) {
        st = status_of(cudaMemsetAsync(L.rt, 0, (size_t)nb * L.n * eb, h->ctx.s), "autotune");
        if (!st) st = status_of(cudaEventRecord(e0, h->ctx.s), "autotune");
        cudaError_t e = cudaSuccess;
        if (!st && cand[c] > 0) {
          e = launch_gmres_persistent(h->ctx, M, L.dpre, L.t, L.rt, L.Vg, L.wg, L.wg2, L.gpartA, L.gpartB,
                                      L.gpstride, L.gR, L.gst, K, 0.0, cand[c], true, nb, eta2);
        } else if (!st) {
          for (int q = 0; q < nb && e == cudaSuccess; ++q) {
            const void* bq = (const char*)L.t + (size_t)q * L.n * eb;
            void* xq = (char*)L.rt + (size_t)q * L.n * eb;
            e = L.gtiles > 0 ? launch_gmres_tile(h->ctx, op_of_rhs(M, q), L.dpre, bq, xq, L.Vg, L.wg, L.gflag,
                                                 L.gpartA, L.gpartB, L.gR, L.gst + q, K, 0.0, L.gtx, L.gty, eta2)
                             : launch_gmres_persistent(h->ctx, op_of_rhs(M, q), L.dpre, bq, xq, L.Vg, L.wg, L.wg2,
                                                       L.gpartA, L.gpartB, L.gpstride, L.gR, L.gst + q, K, 0.0,
                                                       L.ggrid, false, 1, eta2);
          }
        }
        if (!st) st = status_of(e, "autotune launch");
        if (!st) st = status_of(cudaEventRecord(e1, h->ctx.s), "autotune");
        if (!st) st = wait_event(h, e1);
        if (!st) st = status_of(cudaEventElapsedTime(&ms[c], e0, e1), "autotune");  // the second run counts
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    std::vector<GmresState> gs(nb);
    CK(cudaMemcpy(gs.data(), L.gst, sizeof(GmresState) * nb, cudaMemcpyDeviceToHost));
    CK(cudaMemsetAsync(L.gst, 0, sizeof(GmresState) * nb, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    for (int q = 0; q < nb; ++q)
      if (gs[q].err) {
        set_error("a grid barrier of the persistent GMRES kernel exceeded its wait budget");
        return HZ_ETIMEOUT;
      }
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
      if (ms[c] < ms[best]) best = c;
    adopt(cand[best]);
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_batch[key] = cand[best];
  }
  return HZ_OK;
}

int autotune_mg(Handle* h) {
  for (auto& L : h->lv) {
    const int nm = (int)L.mg.size();
    for (int m = 0; m + 1 < nm; ++m) {
      const MGLevel& q = L.mg[m];
      if (q.op.R != 1 || mg_band_rows(0, q.op.nx, q.op.ny, L.dpre)) continue;
      const void* f = m == 0 ? L.rt : q.f;
      void* y = m == 0 ? L.t : q.e;
      CK(tune_mg_bands(h->ctx, q.op, L.dpre, f, L.mg[m + 1].f, L.mg[m + 1].e, y, h->cfg.mg_omega, h->nbmax));
    }
  }
  return HZ_OK;
}

void destroy(Handle* h) {
  cudaStreamSynchronize(h->ctx.s);
  for (auto g : h->graph_exec)
    if (g) cudaGraphExecDestroy(g);
  h->graph_exec.clear();
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  h->capture_stream = nullptr;
  for (auto& L : h->lv) {
    free_scalars(L.sc);
    free_scalars(L.scg);
  }
  free_scalars(h->outer_sc);
  for (void* p : h->allocs) cudaFree(p);
  h->allocs.clear();
}

// ---------------------------------------------------------------------------------- V-cycle
// One V(nu1, nu2) cycle approximating M_l^-1 f (zero initial guess); out = cycle [+ add].
int vcycle(Handle* h, int l, int dt, const void* f, void* out, const void* add, int nb) {
  LevelTag tag(h->ctx, l);
  Level& L = h->lv[l - 1];
  Ctx& c = h->ctx;
  const double om = h->cfg.mg_omega;
  const int nm = (int)L.mg.size();
  if (dt != L.dpre) {
    set_error("multigrid dtype differs from the handle's preconditioner dtype");
    return HZ_EINVAL;
  }
  const size_t eb = elem_bytes(dt);
  if (nm == 1) {  // the level itself is the coarsest: exact dense solve
    if (add) {
      CK(launch_dense(c, L.inv, L.ninv, dt, f, L.r, nb, L.invstride));
      CK(launch_add(c, dt, L.r, dt, add, dt, out, (size_t)nb * L.n));
    } else {
      CK(launch_dense(c, L.inv, L.ninv, dt, f, out, nb, L.invstride));
    }
    return HZ_OK;
  }
  if (h->cfg.mg_nu1 == 1 && h->cfg.mg_nu2 == 1) {
    const void* fm = f;
    for (int m = 0; m + 1 < nm; ++m) {
      CK(launch_mg_down(c, L.mg[m].op, dt, fm, L.mg[m + 1].f, om, nb));
      fm = L.mg[m + 1].f;
    }
    CK(launch_dense(c, L.inv, L.ninv, dt, L.mg[nm - 1].f, L.mg[nm - 1].e, nb, L.invstride));
    for (int m = nm - 2; m >= 0; --m) {
      const void* fmm = (m == 0) ? f : L.mg[m].f;
      void* y = (m == 0) ? out : L.mg[m].e;
      CK(launch_mg_up(c, L.mg[m].op, dt, fmm, L.mg[m + 1].e, y, om, m == 0 ? add : nullptr, dt, nullptr, dt, nb));
    }
    return HZ_OK;
  }
  // general V(nu1, nu2): explicit sweeps with ping-pong buffers
  std::function<int(int, const void*, void*)> rec = [&](int m, const void* fm, void* um) -> int {
    MGLevel& q = L.mg[m];
    const size_t nn = (size_t)nb * q.op.n();
    if (m == nm - 1) {
      CK(launch_dense(c, L.inv, L.ninv, dt, fm, um, nb, L.invstride));
      return HZ_OK;
    }
    void* a = um;
    void* b = q.tmp2;
    if (h->cfg.mg_nu1 >= 1) {
      CK(launch_jacobi_zero(c, q.op, dt, fm, a, om, nb));
      for (int s = 1; s < h->cfg.mg_nu1; ++s) {
        CK(launch_level_op(c, q.op, 2, dt, dt, dt, a, fm, b, om, nb));
        std::swap(a, b);
      }
    } else {
      CK(cudaMemsetAsync(a, 0, nn * eb, c.s));
    }
    CK(launch_level_op(c, q.op, 1, dt, dt, dt, a, fm, q.tmp, 0.0, nb));
    CK(launch_fw(c, dt, q.op.nx, q.op.ny, q.tmp, L.mg[m + 1].f, nb, q.op.bc));
    CS(rec(m + 1, L.mg[m + 1].f, L.mg[m + 1].e));
    CK(launch_prolong_add(c, dt, q.op.nx, q.op.ny, L.mg[m + 1].e, a, nb, q.op.bc));
    for (int s = 0; s < h->cfg.mg_nu2; ++s) {
      CK(launch_level_op(c, q.op, 2, dt, dt, dt, a, fm, b, om, nb));
      std::swap(a, b);
    }
    if (a != um) CK(cudaMemcpyAsync(um, a, nn * eb, cudaMemcpyDeviceToDevice, c.s));
    return HZ_OK;
  };
  void* target = add ? L.r : out;
  CS(rec(0, f, target));
  if (add) CK(launch_add(c, dt, L.r, dt, add, dt, out, (size_t)nb * L.n));
  return HZ_OK;
}

// ---------------------------------------------------------------------------------- Krylov
struct CycleOut {
  std::vector<int> its;
  std::vector<double> est;
  int status = HZ_OK;
};

// One (F)GMRES cycle of at most m iterations on nb right-hand sides (Algorithm 1 lines 2-23).
//  r0 (dvec): initial residuals; u (du): solutions, incremented by X y.
//  X == nullptr: plain GMRES (x_j = v_j, the basis is combined directly).
//  tol_abs_b = tol * (ref ? ref[b] : beta_b); active (optional) masks right-hand sides.
static int cycle(Handle* h, Scalars& sc, int dvec, int dx, size_t n, int nb, void* V, void* X, void* w, int m,
                 const void* r0, void* u, int du, double tol, const std::vector<double>* ref,
                 const std::vector<char>* active_in, const std::function<int(const void*, void*)>& prec,
                 const std::function<int(const void*, void*)>& op, CycleOut& out) {
  Ctx& c = h->ctx;
  const size_t ev = elem_bytes(dvec), ex = elem_bytes(X ? dx : dvec);
  const size_t bn = (size_t)nb * n;
  out.its.assign(nb, 0);
  out.est.assign(nb, 0.0);
  // beta = ||r0||
  CK(launch_multidot(c, dvec, r0, 0, 1, r0, n, nb, sc.dev, h->ws));
  CK(cudaMemcpyAsync(sc.host, sc.dev, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, c.s));
  CS(wait_event(h, sc.ev));
  std::vector<double> beta(nb), tolabs(nb);
  std::vector<char> act(nb, 0);
  int nact = 0;
  for (int b = 0; b < nb; ++b) {
    double s = sc.host[2 * b];
    beta[b] = s > 0 ? std::sqrt(s) : 0.0;
    if (!std::isfinite(beta[b])) {
      set_error("non-finite residual norm");
      out.status = HZ_EBREAKDOWN;
      return HZ_EBREAKDOWN;
    }
    act[b] = (beta[b] > 0) && (!active_in || (*active_in)[b]);
    tolabs[b] = tol * (ref ? (*ref)[b] : beta[b]);
    out.est[b] = beta[b];
    nact += act[b];
  }
  if (!nact) return HZ_OK;
  double* cs_h = sc.host + sc.csc;
  for (int b = 0; b < nb; ++b) {
    cs_h[2 * b] = act[b] ? 1.0 / beta[b] : 0.0;
    cs_h[2 * b + 1] = 0.0;
  }
  CK(cudaMemcpyAsync(sc.dev + sc.csc, cs_h, sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, c.s));
  CK(launch_scale_dev(c, dvec, r0, V, sc.dev + sc.csc, 0, n, nb));
  // host Hessenberg state per rhs
  std::vector<std::vector<cd>> H(nb, std::vector<cd>((size_t)(m + 1) * m, 0.0));
  std::vector<std::vector<double>> gc(nb, std::vector<double>(m, 0.0));
  std::vector<std::vector<cd>> gs(nb, std::vector<cd>(m, 0.0)), gg(nb, std::vector<cd>(m + 1, 0.0));
  for (int b = 0; b < nb; ++b) gg[b][0] = beta[b];
  std::vector<int> jstop(nb, 0);
  int j = 0;
  for (; j < m; ++j) {
    void* Vj = (char*)V + (size_t)j * bn * ev;
    void* Xj = X ? (char*)X + (size_t)j * bn * ex : Vj;
    if (X) CS(prec(Vj, Xj));
    CS(op(Xj, w));
    const int nv = j + 1;
    // Gram-Schmidt with selective reorthogonalisation ("twice is enough", eta = 1/sqrt(2)):
    // pass 1 returns h = V^H w and ||w||^2; a second classical pass runs only for the
    // right-hand sides whose norm dropped below eta ||w|| (decided on the device).
    const int ldA = 2 * nv + 1;
    double* hA = sc.dev + sc.hA;
    double* hB = hA + (size_t)nb * ldA;
    double* n1 = hB + (size_t)nb * 2 * nv;
    double* n2 = n1 + nb;
    double* flag = n2 + nb;
    CK(launch_multidot(c, dvec, V, bn, nv, w, n, nb, hA, h->ws, 1));
    CK(launch_update(c, dvec, V, bn, nv, hA, ldA, dvec, w, n, nb, n1, h->ws));
    const double eta2 = h->cfg.reorth_eta >= 1.0 ? 2.0 : h->cfg.reorth_eta * h->cfg.reorth_eta;
    CK(launch_dgks_flag(c, hA + 2 * nv, ldA, n1, flag, nb, eta2));
    CK(launch_multidot(c, dvec, V, bn, nv, w, n, nb, hB, h->ws, 0, flag));
    CK(launch_update(c, dvec, V, bn, nv, hB, 2 * nv, dvec, w, n, nb, n2, h->ws, flag));
    const size_t cnt = (size_t)nb * (ldA + 2 * nv + 3);
    CK(cudaMemcpyAsync(sc.host, hA, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.s));
    CS(wait_event(h, sc.ev));
    const double* hAh = sc.host;
    const double* hBh = hAh + (size_t)nb * ldA;
    const double* n1h = hBh + (size_t)nb * 2 * nv;
    const double* n2h = n1h + nb;
    const double* flh = n2h + nb;
    std::vector<double> nrh(nb);
    for (int b = 0; b < nb; ++b) nrh[b] = flh[b] != 0.0 ? n1h[b] : n2h[b];
    nact = 0;
    for (int b = 0; b < nb; ++b) {
      if (!act[b]) continue;
      std::vector<cd>& Hb = H[b];
      auto at = [&](int r, int col) -> cd& { return Hb[(size_t)col * (m + 1) + r]; };
      const bool second = flh[b] == 0.0;
      for (int i = 0; i <= j; ++i)
        at(i, j) = cd(hAh[(size_t)b * ldA + 2 * i] + (second ? hBh[(size_t)b * 2 * nv + 2 * i] : 0.0),
                      hAh[(size_t)b * ldA + 2 * i + 1] + (second ? hBh[(size_t)b * 2 * nv + 2 * i + 1] : 0.0));
      double hn = nrh[b] > 0 ? std::sqrt(nrh[b]) : 0.0;
      at(j + 1, j) = hn;
      // apply previous rotations
      for (int i = 0; i < j; ++i) {
        cd a = at(i, j), bb = at(i + 1, j);
        at(i, j) = gc[b][i] * a + gs[b][i] * bb;
        at(i + 1, j) = -std::conj(gs[b][i]) * a + gc[b][i] * bb;
      }
      cd a = at(j, j);
      double bb = hn;
      double t = std::sqrt(std::norm(a) + bb * bb);
      if (t == 0) {
        gc[b][j] = 1.0;
        gs[b][j] = 0.0;
      } else if (std::abs(a) == 0) {
        gc[b][j] = 0.0;
        gs[b][j] = 1.0;
      } else {
        gc[b][j] = std::abs(a) / t;
        gs[b][j] = (a / std::abs(a)) * bb / t;
      }
      at(j, j) = gc[b][j] * a + gs[b][j] * bb;
      at(j + 1, j) = 0.0;
      gg[b][j + 1] = -std::conj(gs[b][j]) * gg[b][j];
      gg[b][j] = gc[b][j] * gg[b][j];
      double est = std::abs(gg[b][j + 1]);
      out.est[b] = est;
      if (!std::isfinite(est) || !std::isfinite(hn)) {
        set_error("non-finite value in the Arnoldi process");
        out.status = HZ_EBREAKDOWN;
        return HZ_EBREAKDOWN;
      }
      if (est <= tolabs[b] || hn == 0.0 || j + 1 == m) {
        act[b] = 0;
        jstop[b] = j + 1;
      } else {
        ++nact;
      }
    }
    if (!nact) {
      ++j;
      break;
    }
    for (int b = 0; b < nb; ++b) {
      double hn = std::abs(H[b][(size_t)j * (m + 1) + j + 1]);  // zeroed by rotation; use norm instead
      (void)hn;
      double nrm = nrh[b] > 0 ? std::sqrt(nrh[b]) : 0.0;
      cs_h[2 * b] = act[b] && nrm > 0 ? 1.0 / nrm : 0.0;
      cs_h[2 * b + 1] = 0.0;
    }
    CK(cudaMemcpyAsync(sc.dev + sc.csc, cs_h, sizeof(double) * 2 * nb, cudaMemcpyHostToDevice, c.s));
    CK(launch_scale_dev(c, dvec, w, (char*)V + (size_t)(j + 1) * bn * ev, sc.dev + sc.csc, 0, n, nb));
  }
  // least squares by back substitution on the rotated Hessenberg (Algorithm 1 line 22)
  int J = 0;
  for (int b = 0; b < nb; ++b) J = std::max(J, jstop[b]);
  if (J == 0) return HZ_OK;
  double* cc = sc.host + sc.ccomb;
  std::memset(cc, 0, sizeof(double) * 2 * (size_t)nb * J);
  for (int b = 0; b < nb; ++b) {
    int k = jstop[b];
    out.its[b] = k;
    std::vector<cd> y(k);
    auto at = [&](int r, int col) -> cd { return H[b][(size_t)col * (m + 1) + r]; };
    for (int i = k - 1; i >= 0; --i) {
      cd s = gg[b][i];
      for (int q = i + 1; q < k; ++q) s -= at(i, q) * y[q];
      y[i] = s / at(i, i);
    }
    for (int i = 0; i < k; ++i) {
      cc[(size_t)b * 2 * J + 2 * i] = y[i].real();
      cc[(size_t)b * 2 * J + 2 * i + 1] = y[i].imag();
    }
  }
  CK(cudaMemcpyAsync(sc.dev + sc.ccomb, cc, sizeof(double) * 2 * (size_t)nb * J, cudaMemcpyHostToDevice, c.s));
  CK(launch_combine(c, X ? dx : dvec, X ? X : V, bn, J, sc.dev + sc.ccomb, du, u, n, nb));
  return HZ_OK;
}

int collect_gmres_stats(Handle* h, int nb) {
  for (auto& L : h->lv) {  // persistent Bi-CGSTAB: iterations, non-finite ends, barrier timeouts
    if (L.bgrid <= 0) continue;
    std::vector<BicgState> bs(nb);
    BicgBarrier bb;
    CK(cudaMemcpyAsync(bs.data(), L.bst, sizeof(BicgState) * nb, cudaMemcpyDeviceToHost, h->ctx.s));
    CK(cudaMemcpyAsync(&bb, L.bbar, sizeof(bb), cudaMemcpyDeviceToHost, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    double nonfinite = 0;
    for (int q = 0; q < nb; ++q) {
      h->st[q].cslp_it[L.l - 1] += (int)bs[q].total_its;
      nonfinite += bs[q].nonfinite;
      bs[q].total_its = 0;
      bs[q].nonfinite = 0;
    }
    CK(cudaMemcpyAsync(L.bst, bs.data(), sizeof(BicgState) * nb, cudaMemcpyHostToDevice, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    if (bb.err) {
      set_error("a grid barrier of the persistent Bi-CGSTAB kernel exceeded its wait budget");
      return HZ_ETIMEOUT;
    }
    if (nonfinite > 0) {
      set_error("non-finite residual in the Bi-CGSTAB CSLP solve");
      return HZ_EBREAKDOWN;
    }
  }
  for (auto& L : h->lv) {
    if (!L.m1cnt) continue;
    std::vector<int> cnt(2 * (size_t)nb);
    CK(cudaMemcpyAsync(cnt.data(), L.m1cnt, sizeof(int) * 2 * (size_t)nb, cudaMemcpyDeviceToHost, h->ctx.s));
    CK(cudaMemsetAsync(L.m1cnt, 0, sizeof(int) * 2 * (size_t)nb, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    for (int q = 0; q < nb; ++q) {
      h->st[q].lev_it[L.l - 1] += cnt[q];
      h->st[q].lev_calls[L.l - 1] += cnt[nb + q];
    }
  }
  {
    int err = 0;
    CK(cudaMemcpyAsync(&err, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->ctx.s));
    CK(cudaMemsetAsync(h->derr, 0, sizeof(int), h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    if (err) {
      set_error("non-finite value in a one-iteration coarse-level cycle");
      return HZ_EBREAKDOWN;
    }
  }
  for (auto& L : h->lv) {
    if (!L.gst) continue;
    std::vector<GmresState> gs(nb);
    CK(cudaMemcpyAsync(gs.data(), L.gst, sizeof(GmresState) * nb, cudaMemcpyDeviceToHost, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    int err = 0;
    double bytes = 0;
    for (int q = 0; q < nb; ++q) {
      h->st[q].cslp_it[L.l - 1] += (int)gs[q].total_its;
      h->st[q].cslp_reorth[L.l - 1] += (int)gs[q].total_reorth;
      bytes += gs[q].total_bytes;
      if (L.l <= HZ_MAX_LEVELS) {
        h->gdev_launches[L.l] += gs[q].launches;
        h->gdev_ms[L.l] += 1e-6 * (double)gs[q].total_ns;
        h->gdev_bytes[L.l] += gs[q].total_bytes;
      }
      gs[q].total_its = 0;
      gs[q].total_bytes = 0;
      gs[q].total_reorth = 0;
      gs[q].total_ns = 0;
      gs[q].launches = 0;
      err |= gs[q].err;
    }
    // the kernel's algorithmic bytes are known only after it ran: credit them to the family
    if (h->prof.on[F_GMRES]) {
      h->prof.bytes[F_GMRES] += bytes;
      if (L.l < kProfLevels) h->prof.bytes_lv[F_GMRES][L.l] += bytes;
    }
    CK(cudaMemcpyAsync(L.gst, gs.data(), sizeof(GmresState) * nb, cudaMemcpyHostToDevice, h->ctx.s));
    CK(cudaStreamSynchronize(h->ctx.s));
    if (err) {
      set_error("a grid barrier of the persistent GMRES kernel exceeded its wait budget");
      return HZ_ETIMEOUT;
    }
  }
  return HZ_OK;
}

// CSLP inverse by unpreconditioned GMRES on M_l (levels > mg_max_level): x += GMRES(b).
int cslp_gmres(Handle* h, int l, const void* b, void* x, int nb, int* its_out) {
  LevelTag tag(h->ctx, l);
  Level& L = h->lv[l - 1];
  const int dt = L.dpre;
  OpDesc M = L.opM(dt, h->cfg.beta1, h->cfg.beta2);
  if (L.ggrid > 0 || L.gcl > 0) {  // whole solve on the device
    const size_t eb = elem_bytes(dt);
    const double eta2 = h->cfg.reorth_eta >= 1.0 ? 2.0 : h->cfg.reorth_eta * h->cfg.reorth_eta;
    const bool use_cluster =
        L.gcl > 0 && (h->cfg.device_gmres == 3 || (nb >= kClusterMinRhs && !L.gseq) || L.ggrid <= 0);
    if (use_cluster) {  // one launch, one thread-block cluster per right-hand side
      CK(launch_gmres_persistent(h->ctx, M, dt, b, x, L.Vg, L.wg, L.wg2, L.gpartA, L.gpartB, L.gpstride, L.gR, L.gst,
                                 L.capg, h->cfg.cslp_tol, L.gcl, true, nb, eta2));
    } else if (L.gtiles > 0) {  // tile-owned form, one cooperative launch per right-hand side
      for (int q = 0; q < nb; ++q)
        CK(launch_gmres_tile(h->ctx, op_of_rhs(M, q), dt, (const char*)b + (size_t)q * L.n * eb, (char*)x + (size_t)q * L.n * eb,
                             L.Vg, L.wg, L.gflag, L.gpartA, L.gpartB, L.gR, L.gst + q, L.capg, h->cfg.cslp_tol,
                             L.gtx, L.gty, eta2));
    } else {  // one cooperative launch per right-hand side
      for (int q = 0; q < nb; ++q)
        CK(launch_gmres_persistent(h->ctx, op_of_rhs(M, q), dt, (const char*)b + (size_t)q * L.n * eb,
                                   (char*)x + (size_t)q * L.n * eb, L.Vg, L.wg, L.wg2, L.gpartA, L.gpartB, L.gpstride,
                                   L.gR, L.gst + q, L.capg, h->cfg.cslp_tol, L.ggrid, false, 1, eta2));
    }
    if (its_out) {
      std::vector<GmresState> gs(nb);
      CK(cudaMemcpyAsync(gs.data(), L.gst, sizeof(GmresState) * nb, cudaMemcpyDeviceToHost, h->ctx.s));
      CK(cudaStreamSynchronize(h->ctx.s));
      for (int q = 0; q < nb; ++q) its_out[q] = gs[q].its;
    }
    return HZ_OK;
  }
  auto op = [&](const void* xin, void* wout) -> int {
    CK(launch_level_op(h->ctx, M, 0, dt, dt, dt, xin, nullptr, wout, 0.0, nb));
    return HZ_OK;
  };
  std::function<int(const void*, void*)> noprec;
  CycleOut co;
  CS(cycle(h, L.scg, dt, dt, L.n, nb, L.Vg, nullptr, L.wg, L.capg, b, x, dt, h->cfg.cslp_tol, nullptr, nullptr,
           noprec, op, co));
  for (int q = 0; q < nb; ++q) {
    h->st[q].cslp_it[l - 1] += co.its[q];
    if (its_out) its_out[q] = co.its[q];
  }
  return HZ_OK;
}

// CSLP inverse by Bi-CGSTAB on M_l (levels > mg_max_level, cslp_solver = HZ_CSLP_BICGSTAB):
// x += BiCGSTAB(b), tolerance cslp_tol, at most capg iterations.  Scalars stay on the device;
// the host looks at the stop flags every kBicgCheck iterations and after the last one.
constexpr int kBicgCheck = 4;
int cslp_bicgstab(Handle* h, int l, const void* b, void* x, int nb, int* its_out) {
  LevelTag tag(h->ctx, l);
  Level& L = h->lv[l - 1];
  if (!L.bcg) {
    set_error("the level has no Bi-CGSTAB workspace (cslp_solver is not HZ_CSLP_BICGSTAB)");
    return HZ_EINVAL;
  }
  Ctx& c = h->ctx;
  const int dt = L.dpre;
  const size_t n = L.n, bn = (size_t)nb * n, eb = elem_bytes(dt);
  if (L.bgrid > 0) {  // persistent form: one cooperative launch per right-hand side, no host decision
    const OpDesc Mq = L.opM(dt, h->cfg.beta1, h->cfg.beta2);
    for (int q = 0; q < nb; ++q)
      CK(launch_bicg_persist(c, op_of_rhs(Mq, q), dt, (const char*)b + (size_t)q * n * eb,
                             (char*)x + (size_t)q * n * eb, L.bcg, L.bgpart, L.bst + q, L.bbar, L.capg,
                             h->cfg.cslp_tol, L.bgrid));
    if (its_out) {
      std::vector<BicgState> bs(nb);
      CK(cudaMemcpyAsync(bs.data(), L.bst, sizeof(BicgState) * nb, cudaMemcpyDeviceToHost, c.s));
      CK(cudaStreamSynchronize(c.s));
      for (int q = 0; q < nb; ++q) its_out[q] = (int)bs[q].its;
    }
    return HZ_OK;
  }
  char* base = (char*)L.bcg;
  const size_t stride = (size_t)h->nbmax * n * eb;
  void *r = base, *p = base + stride, *v = base + 2 * stride, *s = base + 3 * stride, *t = base + 4 * stride;
  OpDesc M = L.opM(dt, h->cfg.beta1, h->cfg.beta2);
  CK(cudaMemcpyAsync(r, b, bn * eb, cudaMemcpyDeviceToDevice, c.s));
  CK(cudaMemsetAsync(p, 0, bn * eb, c.s));
  CK(cudaMemsetAsync(v, 0, bn * eb, c.s));
  CK(launch_bicg_start(c, dt, b, n, nb, h->cfg.cslp_tol, L.bpart, L.bst));
  // stop flags come back through the level's pinned scalar buffer under the handle's timeout
  if (sizeof(BicgState) * (size_t)nb > L.scg.total * sizeof(double)) {
    set_error("Bi-CGSTAB state does not fit the level's host scalar buffer");
    return HZ_EINVAL;
  }
  const BicgState* hs = reinterpret_cast<const BicgState*>(L.scg.host);
  auto fetch = [&]() -> int {
    CK(cudaMemcpyAsync(L.scg.host, L.bst, sizeof(BicgState) * nb, cudaMemcpyDeviceToHost, c.s));
    return wait_event(h, L.scg.ev);
  };
  for (int it = 0; it < L.capg; ++it) {
    CK(launch_bicg_p(c, dt, r, p, v, n, nb, L.bst));
    CK(launch_level_op(c, M, 0, dt, dt, dt, p, nullptr, v, 0.0, nb));
    CK(launch_bicg_dots(c, dt, 0, b, v, nullptr, nullptr, n, nb, L.bpart, L.bst));
    CK(launch_bicg_s(c, dt, r, v, s, n, nb, L.bst));
    CK(launch_level_op(c, M, 0, dt, dt, dt, s, nullptr, t, 0.0, nb));
    CK(launch_bicg_dots(c, dt, 1, t, s, t, t, n, nb, L.bpart, L.bst));
    CK(launch_bicg_xr(c, dt, x, p, s, t, r, b, n, nb, L.bpart, L.bst));
    if ((it + 1) % kBicgCheck == 0 || it + 1 == L.capg) {
      CS(fetch());
      bool all = true;
      for (int q = 0; q < nb; ++q) all &= hs[q].done != 0.0;
      if (all) break;
    }
  }
  for (int q = 0; q < nb; ++q) {
    if (!std::isfinite(hs[q].rn2)) {
      set_error("non-finite residual in the Bi-CGSTAB CSLP solve");
      return HZ_EBREAKDOWN;
    }
    h->st[q].cslp_it[l - 1] += (int)hs[q].its;
    if (its_out) its_out[q] = (int)hs[q].its;
  }
  return HZ_OK;
}

// out = M_l^-1 rtil [+ add]  (Algorithm 1 line 14; with add = t also line 15)
int cslp_inverse(Handle* h, int l, const void* rtil, void* out, const void* add, int nb) {
  Level& L = h->lv[l - 1];
  if (l <= h->cfg.mg_max_level) return vcycle(h, l, L.dpre, rtil, out, add, nb);
  const size_t bytes = (size_t)nb * L.n * elem_bytes(L.dpre);
  if (add) CK(cudaMemcpyAsync(out, add, bytes, cudaMemcpyDeviceToDevice, h->ctx.s));
  else CK(cudaMemsetAsync(out, 0, bytes, h->ctx.s));
  if (h->cfg.cslp_solver == HZ_CSLP_BICGSTAB) return cslp_bicgstab(h, l, rtil, out, nb, nullptr);
  return cslp_gmres(h, l, rtil, out, nb, nullptr);
}

// coarse_solve(l) through a CUDA graph when level l's whole subtree runs on the device: captured
// on first use for this batch size, replayed afterwards.  Profiling runs it eagerly (the event
// pairs of the per-family timers are host-side records).  A capture the runtime refuses falls
// back to launching eagerly for the rest of the handle's life.
static int coarse_solve_graph(Handle* h, int l, int nb) {
  bool profiling = false;
  for (int f = 0; f < F_COUNT; ++f) profiling |= h->prof.on[f];
  if (l != h->graph_level || h->graph_failed || profiling || nb < 1 || nb > (int)h->graph_exec.size())
    return coarse_solve(h, l, nb);
  cudaGraphExec_t& ex = h->graph_exec[nb - 1];
  if (!ex) {
    // capture on the handle's private stream (the caller's stream may be the legacy default
    // stream, which cannot be captured); nothing runs during the capture
    cudaStream_t s = h->capture_stream;
    const long long l0 = h->prof.total_launches;
    cudaGraph_t g = nullptr;
    if (!s || cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graph_failed = true;
      return coarse_solve(h, l, nb);
    }
    const cudaStream_t user = h->ctx.s;
    h->ctx.s = s;
    const int st = coarse_solve(h, l, nb);
    h->ctx.s = user;
    const cudaError_t e = cudaStreamEndCapture(s, &g);
    if (st != HZ_OK || e != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
      cudaGetLastError();
      if (g) cudaGraphDestroy(g);
      ex = nullptr;
      h->graph_failed = true;
      h->prof.total_launches = l0;
      return coarse_solve(h, l, nb);
    }
    cudaGraphDestroy(g);
    h->graph_launches[nb - 1] = h->prof.total_launches - l0;
    h->prof.total_launches = l0;
  }
  CK(cudaGraphLaunch(ex, h->ctx.s));
  h->prof.total_launches += h->graph_launches[nb - 1];
  return HZ_OK;
}

// x = P v at level l (Algorithm 1 lines 5-15).  v has dtype dv; x has dtype lv[l-1].dx.
int precond(Handle* h, int l, const void* v, int dv, void* xout, int nb) {
  LevelTag tag(h->ctx, l);
  Level& L = h->lv[l - 1];
  Ctx& c = h->ctx;
  const int ml = h->cfg.levels;
  if (l == ml) {  // coarsest (or single level): CSLP only
    const void* src = v;
    if (dv != L.dpre) {
      CK(launch_convert(c, dv, L.dpre, v, L.rt, (size_t)nb * L.n));
      src = L.rt;
    }
    return cslp_inverse(h, l, src, xout, nullptr, nb);
  }
  Level& C = h->lv[l];
  CK(launch_defl_restrict(c, dv, C.dvec, L.nx, L.ny, v, C.b, nb, L.bc));           // line 5
  CS(coarse_solve_graph(h, l + 1, nb));                                            // lines 6-10
  CK(launch_defl_prolong_resid(c, L.opA(L.dpre), L.dpre, dv, C.x, C.nx, C.ny, v, L.t, L.rt, nb));  // 11-13
  return cslp_inverse(h, l, L.rt, xout, L.t, nb);                                  // lines 14-15
}

// One-iteration (F)GMRES cycle of a coarse level (levels 3..ml-1, and the coarsest level when it
// is treated as negative definite) with every scalar step on the device.  With m = 1 the cycle's
// result is the minimal-residual step x = (w^H b / w^H w) P b, w = A P b (Algorithm 1: v = b/||b||,
// one Arnoldi step, y from the 2 x 1 least-squares problem); no host round trip.  Iteration counts
// and breakdowns are collected at the end of the solve.  r0 = L.b, solution L.x (zero on entry).
static int cycle_m1_device(Handle* h, Level& L, int nb, const std::function<int(const void*, void*)>& prec,
                           const std::function<int(const void*, void*)>& op) {
  Ctx& c = h->ctx;
  Scalars& sc = L.sc;
  const size_t n = L.n, bn = (size_t)nb * n;
  double* d = sc.dev + sc.hA;          // b^H w and ||w||^2, stride 3
  double* coef = sc.dev + sc.ccomb;
  CS(prec(L.b, L.X));                                                     // X = P b
  CS(op(L.X, L.w));                                                       // w = A X
  CK(launch_multidot(c, L.dvec, L.b, 0, 1, L.w, n, nb, d, h->ws, 1));     // b^H w, ||w||^2
  CK(launch_m1_mr(c, d, nb, coef, L.m1cnt, L.m1cnt + nb, h->derr));
  CK(launch_combine(c, L.dx, L.X, bn, 1, coef, L.dvec, L.x, n, nb));      // x = coef X
  return HZ_OK;
}

// v_til ~ A_l^-1 b on level l >= 2 with the MADP schedule; reads lv[l-1].b, writes .x
int coarse_solve(Handle* h, int l, int nb) {
  LevelTag tag(h->ctx, l);
  Level& L = h->lv[l - 1];
  const double tol = L.tol;
  CK(cudaMemsetAsync(L.x, 0, (size_t)nb * L.n * elem_bytes(L.dvec), h->ctx.s));
  OpDesc A = L.opA(L.dvec);
  auto op = [&](const void* xin, void* wout) -> int {
    CK(launch_level_op(h->ctx, A, 0, L.dvec, L.dx, L.dvec, xin, nullptr, wout, 0.0, nb));
    return HZ_OK;
  };
  auto prec = [&](const void* vj, void* xj) -> int { return precond(h, l, vj, L.dvec, xj, nb); };
  if (L.cap == 1 && L.m1cnt) return cycle_m1_device(h, L, nb, prec, op);
  CycleOut co;
  CS(cycle(h, L.sc, L.dvec, L.dx, L.n, nb, L.V, L.X, L.w, L.cap, L.b, L.x, L.dvec, tol, nullptr, nullptr, prec, op,
           co));
  for (int q = 0; q < nb; ++q)
    if (co.its[q] > 0) {
      h->st[q].lev_it[l - 1] += co.its[q];
      h->st[q].lev_calls[l - 1] += 1;
    }
  return HZ_OK;
}

// ---------------------------------------------------------------------------------- solve
int solve(Handle* h, const void* b, void* u, int nb, double tol, unsigned flags) {
  LevelTag tag(h->ctx, 1);
  Level& L = h->lv[0];
  Ctx& c = h->ctx;
  const hz_config& cfg = h->cfg;
  const size_t n = L.n;
  for (int q = 0; q < nb; ++q) h->st[q] = RhsStats();
  Scalars& sc = h->outer_sc;
  auto norms = [&](const void* x, std::vector<double>& out) -> int {
    CK(launch_multidot(c, C128, x, 0, 1, x, n, nb, sc.dev, h->ws));
    CK(cudaMemcpyAsync(sc.host, sc.dev, sizeof(double) * 2 * nb, cudaMemcpyDeviceToHost, c.s));
    CS(wait_event(h, sc.ev));
    out.resize(nb);
    for (int q = 0; q < nb; ++q) out[q] = sc.host[2 * q] > 0 ? std::sqrt(sc.host[2 * q]) : 0.0;
    return HZ_OK;
  };
  OpDesc A = L.opA(C128);
  if (cfg.sym_rows) {  // the row-scaled system D A u = D b (same u)
    A.srow = 1;
    CK(launch_row_scale(c, L.nx, L.ny, b, h->bscaled, nb));
    b = h->bscaled;
  }
  std::vector<double> bnorm, rel(nb, 0.0);
  CS(norms(b, bnorm));
  if (flags & HZ_SOLVE_INITIAL_GUESS) {
    CK(launch_level_op(c, A, 1, C128, C128, C128, u, b, h->rres, 0.0, nb));
  } else {
    CK(cudaMemsetAsync(u, 0, (size_t)nb * n * 16, c.s));
    CK(cudaMemcpyAsync(h->rres, b, (size_t)nb * n * 16, cudaMemcpyDeviceToDevice, c.s));
  }
  std::vector<double> rn;
  CS(norms(h->rres, rn));
  std::vector<char> act(nb, 0);
  std::vector<int> total(nb, 0);
  int nact = 0;
  for (int q = 0; q < nb; ++q) {
    rel[q] = bnorm[q] > 0 ? rn[q] / bnorm[q] : 0.0;
    act[q] = bnorm[q] > 0 && rel[q] > tol;
    nact += act[q];
  }
  auto op = [&](const void* xin, void* wout) -> int {
    CK(launch_level_op(c, A, 0, C128, L.dx, C128, xin, nullptr, wout, 0.0, nb));
    return HZ_OK;
  };
  auto prec = [&](const void* vj, void* xj) -> int { return precond(h, 1, vj, C128, xj, nb); };
  while (nact) {
    int mint = cfg.max_outer;
    for (int q = 0; q < nb; ++q)
      if (act[q]) mint = std::min(mint, total[q]);
    int m = std::min(cfg.restart, cfg.max_outer - mint);
    if (m <= 0) break;
    CycleOut co;
    CS(cycle(h, L.sc, C128, L.dx, n, nb, L.V, L.X, L.w, m, h->rres, u, C128, tol, &bnorm, &act, prec, op, co));
    CK(launch_level_op(c, A, 1, C128, C128, C128, u, b, h->rres, 0.0, nb));   // true residual (FP64)
    CS(norms(h->rres, rn));
    nact = 0;
    for (int q = 0; q < nb; ++q) {
      if (!act[q]) continue;
      total[q] += co.its[q];
      h->st[q].est = bnorm[q] > 0 ? co.est[q] / bnorm[q] : 0.0;
      rel[q] = rn[q] / bnorm[q];
      if (!std::isfinite(rel[q])) {
        act[q] = 0;
        h->st[q].status = HZ_EBREAKDOWN;
      } else if (rel[q] <= tol) {
        act[q] = 0;
      } else if (total[q] >= cfg.max_outer || co.its[q] == 0) {
        act[q] = 0;
        h->st[q].status = HZ_ENOTCONV;
      } else {
        ++nact;
      }
    }
  }
  CS(collect_gmres_stats(h, nb));
  int first = HZ_OK;
  for (int q = 0; q < nb; ++q) {
    h->st[q].outer = total[q];
    h->st[q].true_rel = rel[q];
    if (h->st[q].status == HZ_OK && rel[q] > tol) h->st[q].status = HZ_ENOTCONV;
    if (!first && h->st[q].status) first = h->st[q].status;
  }
  return first;
}

}  // namespace hz
