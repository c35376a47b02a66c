// Library state behind the C ABI: level hierarchy, workspace, solver drivers.
#pragma once
#include <complex>
#include <vector>

#include "hz.h"
#include "hz_internal.h"

namespace hz {

typedef std::complex<double> cd;

struct MGLevel {
  OpDesc op;              // M on this multigrid level (level 0: the deflation level's own M_l)
  void* f = nullptr;      // right-hand side of this MG level (levels >= 1)
  void* e = nullptr;      // correction of this MG level (levels >= 1)
  void* tmp = nullptr;    // scratch for the general (nu != 1) cycle
  void* tmp2 = nullptr;
};

// Pinned host + device scalar areas of one Krylov driver (one per level and purpose).
struct Scalars {
  double* dev = nullptr;  // [hA | hB | nrm2 | coef_scale | coef_comb]
  double* host = nullptr;
  size_t hA = 0, hB = 0, nrm = 0, csc = 0, ccomb = 0, total = 0;
  cudaEvent_t ev = nullptr;
};

struct Level {
  int l = 1, nx = 0, ny = 0;
  int bc = 0;  // HZ_BC_* of the grid: Dirichlet levels hold interior unknowns only
  size_t n = 0;
  int R = 1;
  double H = 0, ks = 1;
  double m[7] = {}, L[7] = {};
  double* k_d = nullptr;
  float* k_f = nullptr;
  size_t kstride = 0;                        // per_rhs_k: n (field of rhs b at k + b n), else 0
  int dvec = C128, dpre = C128, dx = C128;   // basis, preconditioner temporaries, stored x_j
  // multigrid CSLP (l <= mg_max_level)
  std::vector<MGLevel> mg;
  double* inv = nullptr;                     // dense FP64 inverse of the coarsest MG operator
  int ninv = 0;
  size_t invstride = 0;                      // per_rhs_k: one inverse per field, ninv^2 apart
  // deflated / CSLP FGMRES of this level
  int cap = 0;                               // iteration cap per cycle
  double tol = 0.0;                          // relative tolerance of a coarse solve (0 = exactly cap iterations)
  void* V = nullptr;                         // (cap + 1) batches, dvec
  void* X = nullptr;                         // cap batches, dx
  void* w = nullptr;                         // dvec
  void* b = nullptr;                         // right-hand side on this level (l >= 2), dvec
  void* x = nullptr;                         // solution on this level (l >= 2), dvec
  void* t = nullptr;                         // Z v_til, dpre
  void* rt = nullptr;                        // r_til, dpre
  void* r = nullptr;                         // general-path scratch, dpre
  Scalars sc;
  int* m1cnt = nullptr;                      // one-iteration levels: per-rhs iterations, then calls (device)
  // GMRES CSLP inverse (l > mg_max_level)
  int capg = 0;
  void* Vg = nullptr;                        // (capg + 1) batches, dpre
  void* wg = nullptr;
  Scalars scg;
  // persistent GMRES (device_gmres): second work vector, partials, Hessenberg, control blocks
  void* wg2 = nullptr;
  double* gpartA = nullptr;
  double* gpartB = nullptr;
  int gpstride = 0;
  double* gR = nullptr;
  GmresState* gst = nullptr;                 // nbmax control blocks
  unsigned* gflag = nullptr;                 // tile-owned form: halo flag per tile
  // Bi-CGSTAB CSLP solver (cslp_solver = HZ_CSLP_BICGSTAB): r, p, v, s, t batches, scalars, partials
  void* bcg = nullptr;
  BicgState* bst = nullptr;
  double* bpart = nullptr;
  int bgrid = 0;                             // persistent Bi-CGSTAB: CTAs of its cooperative grid (0: not used)
  BicgBarrier* bbar = nullptr;               // its grid barrier
  double* bgpart = nullptr;                  // its partial sums (8 per CTA)
  int ggrid = 0;                             // CTAs of the cooperative-grid form (0: host-driven GMRES)
  int gcl = 0;                               // CTAs per cluster of the cluster form (0: not used)
  bool gseq = false;                         // batches faster one right-hand side at a time (autotune)
  int gtiles = 0, gtx = 0, gty = 0;          // tile-owned form: CTAs (= tiles) and tile shape (0: not used)
  OpDesc opA(int dt) const;
  OpDesc opM(int dt, double b1, double b2) const;
};

struct RhsStats {
  int outer = 0;
  int lev_it[HZ_MAX_LEVELS] = {}, lev_calls[HZ_MAX_LEVELS] = {}, cslp_it[HZ_MAX_LEVELS] = {};
  int cslp_reorth[HZ_MAX_LEVELS] = {};
  double est = 0, true_rel = 0;
  int status = HZ_OK;
};

struct Handle {
  hz_grid g{};
  hz_config cfg{};
  int device = -1;                           // CUDA device current at hz_setup (owns every allocation)
  Ctx ctx;
  Prof prof;
  std::vector<Level> lv;
  std::vector<void*> allocs;
  size_t bytes = 0;
  void* ws = nullptr;                        // reduction workspace
  size_t ws_bytes = 0;
  int nbmax = 1;
  std::vector<RhsStats> st;                  // per-rhs statistics of the running call
  Scalars outer_sc;                          // true-residual norms
  void* rres = nullptr;                      // level-1 true residual buffer (C128)
  void* bscaled = nullptr;                   // sym_rows: D b, the right-hand side of the scaled system
  int* derr = nullptr;                       // device breakdown flag of the device-side cycles
  // CUDA graph of the coarse solve at level graph_level (every level from there down runs on the
  // device without host decisions), one per batch size; launches it replays, for the counter
  int graph_level = 0;
  bool graph_failed = false;
  cudaStream_t capture_stream = nullptr;     // private stream the graphs are captured on
  std::vector<cudaGraphExec_t> graph_exec;   // index nb - 1
  std::vector<long long> graph_launches;
  // device-timed persistent GMRES launches per level (index l), accumulated by
  // collect_gmres_stats from the kernel's own %globaltimer stamps
  long long gdev_launches[HZ_MAX_LEVELS + 1] = {};
  double gdev_ms[HZ_MAX_LEVELS + 1] = {};
  double gdev_bytes[HZ_MAX_LEVELS + 1] = {};
};

// allocation helpers (track for hz_destroy)
int dalloc(Handle* h, void** p, size_t bytes);
int status_of(cudaError_t e, const char* where);

int setup(Handle* h, const double* k_dev);
// Loads the allocation-free residual check's module on the handle's device and looks up its
// static scratch array (noalloc.cu), so that no later call of that entry point reserves memory.
int noalloc_prepare(Handle* h);
// Keep the faster persistent GMRES form per level (tile-owned or slice-distributed).
int autotune_gmres(Handle* h);
// Keep the faster of the cluster form (16, 8 or 4 CTAs per right-hand side) and one whole-grid
// launch per right-hand side for batches of max_rhs right-hand sides.
int autotune_batch(Handle* h);
// Keep the fastest band height of the radius-1 multigrid sweeps per level shape (autotune).
int autotune_mg(Handle* h);
int gmres_grid_want(int nx, int ny);
size_t estimate_bytes(const hz_grid& g, const hz_config& cfg);
void destroy(Handle* h);

// drivers (all on nb right-hand sides in lockstep)
int vcycle(Handle* h, int l, int dt, const void* f, void* out, const void* add, int nb);
int cslp_inverse(Handle* h, int l, const void* rtil, void* out, const void* add, int nb);
int cslp_gmres(Handle* h, int l, const void* b, void* x, int nb, int* its_out);
int cslp_bicgstab(Handle* h, int l, const void* b, void* x, int nb, int* its_out);
int precond(Handle* h, int l, const void* v, int dv, void* xout, int nb);
int coarse_solve(Handle* h, int l, int nb);
int solve(Handle* h, const void* b, void* u, int nb, double tol, unsigned flags);
int wait_event(Handle* h, cudaEvent_t ev);
// Fold the persistent-GMRES iteration counters into h->st and check their error flags.
int collect_gmres_stats(Handle* h, int nb);

}  // namespace hz
