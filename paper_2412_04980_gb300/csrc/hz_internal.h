// Host-side internal interface of the library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

namespace hz {

enum Dtype { C128 = 0, C64 = 1 };

inline size_t elem_bytes(int dt) { return dt == C128 ? 16 : 8; }

// Kernel families for the per-launch event timer.
enum Family {
  F_LEVEL_OP = 0,   // level operator apply / residual / Jacobi
  F_MG_DOWN,        // fused pre-smooth + residual + full weighting
  F_MG_UP,          // fused bilinear correction + post-smooth
  F_DEFL_RESTRICT,  // Z^T
  F_DEFL_PROLONG,   // Z, and Z + A + subtract
  F_DOT,            // multi-dot products
  F_AXPY,           // basis updates / combinations / scaling
  F_REDUCE,         // second-stage reductions
  F_DENSE,          // dense coarsest multigrid solve
  F_MISC,           // conversions, copies
  F_GMRES,          // persistent whole-solve GMRES kernel
  F_BICG,           // persistent whole-solve Bi-CGSTAB kernel
  F_COUNT
};
const char* family_name(int f);

// Raise a kernel's dynamic shared-memory limit to at least `bytes`.  The limit is process-wide
// per kernel and handles on other threads may launch the same kernel with a larger size at the
// same time, so it is only ever raised (under a lock), never lowered.
cudaError_t ensure_dyn_smem(const void* func, size_t bytes);

constexpr int kProfLevels = 11;  // index 0: not inside a level; 1..10: deflation level
struct Prof {
  struct Rec { cudaEvent_t a, b; double bytes; int level; };
  bool on[F_COUNT] = {};
  std::vector<Rec> pending[F_COUNT];
  long long launches[F_COUNT] = {};
  double ms[F_COUNT] = {};
  double bytes[F_COUNT] = {};
  long long launches_lv[F_COUNT][kProfLevels] = {};
  double ms_lv[F_COUNT][kProfLevels] = {};
  double bytes_lv[F_COUNT][kProfLevels] = {};
  long long total_launches = 0;   // every kernel launch through a launcher, profiled or not
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
  void drain(int fam);   // synchronous: folds pending records into the totals
  ~Prof();
};

struct Ctx {
  cudaStream_t s = 0;
  Prof* prof = nullptr;
  int level = 0;  // deflation level whose work is being launched (profiling attribution)
};

// Sets Ctx::level for the lifetime of the object and restores the previous value.
struct LevelTag {
  Ctx& c;
  int prev;
  LevelTag(Ctx& c_, int l) : c(c_), prev(c_.level) { c.level = l; }
  ~LevelTag() { c.level = prev; }
};

// RAII-free launch timer: begin() returns an index, end() closes it.
struct ProfScope {
  Ctx& c;
  int fam;
  double bytes;
  int level;
  cudaEvent_t a = nullptr;
  ProfScope(Ctx& c_, int fam_, double bytes_);
  ~ProfScope();
};

// Host description of one grid operator (see hzd::OpP).  With kstride != 0 right-hand side b
// of a launch takes the wavenumber field k + b kstride (multi-instance batches).
struct OpDesc {
  int nx = 0, ny = 0, R = 1, bc = 0;
  int srow = 0;  // 1: Sommerfeld boundary rows scaled by 1/2 per boundary side (radius-1 rows)
  double c = 0, H = 0, ks = 1, sr = 1, si = 0;
  double m[7] = {}, l[7] = {};
  const double* k_d = nullptr;
  const float* k_f = nullptr;
  size_t kstride = 0;  // nodes between the wavenumber fields of consecutive right-hand sides (0: shared)
  size_t n() const { return (size_t)nx * ny; }
};

// ---- stencil launchers (kern_stencil.cu) --------------------------------------------
// mode: 0 y = Op x; 1 y = f - Op x; 2 y = x + omega (f - Op x) / D
// tcomp: arithmetic dtype; tx: dtype of x and f; ty: dtype of y.
cudaError_t launch_level_op(Ctx& c, const OpDesc& op, int mode, int tcomp, int tx, int ty, const void* x,
                            const void* f, void* y, double omega, int nrhs);
// y = omega f / D (Jacobi sweep from a zero initial guess), tcomp == tx == ty
cudaError_t launch_jacobi_zero(Ctx& c, const OpDesc& op, int dt, const void* f, void* y, double omega, int nrhs);
// t = Z vtil (coarse vtil, dtype tcomp), rtil = v - A t.  v has dtype tv; t, rtil dtype tcomp.
cudaError_t launch_defl_prolong_resid(Ctx& c, const OpDesc& op, int tcomp, int tv, const void* vtil,
                                      int ncx, int ncy, const void* v, void* t, void* rtil, int nrhs);
// Transfers take the grid's boundary type: vertex grids (bc 0) put coarse node I at fine node 2I,
// Dirichlet grids (bc 1, interior unknowns) at fine unknown 2I + 1.
// t = Z w (plain prolongation), same dtype.
cudaError_t launch_defl_prolong(Ctx& c, int dt, int nx, int ny, const void* w, void* t, int nrhs, int bc = 0);
// vhat = Z^T v; v dtype tin, vhat dtype tout (arithmetic in tout).
cudaError_t launch_defl_restrict(Ctx& c, int tin, int tout, int nx, int ny, const void* v, void* vhat,
                                 int nrhs, int bc = 0);
// Fused multigrid kernels, V(1,1) with zero initial guess.
// down: fc = FW(f - Op(omega f / D)) on the next coarser grid (ncx x ncy)
cudaError_t launch_mg_down(Ctx& c, const OpDesc& op, int dt, const void* f, void* fc, double omega, int nrhs);
// up: u = omega f / D + P ec; y = u + omega (f - Op u) / D (+ add if add != null, add dtype tadd)
cudaError_t launch_mg_up(Ctx& c, const OpDesc& op, int dt, const void* f, const void* ec, void* y,
                         double omega, const void* add, int tadd, void* yout2, int tout2, int nrhs);
// Band height (rows per warp) of the radius-1 strip sweeps: times both sweeps of a multigrid level
// at every candidate on the given buffers (contents are overwritten) and keeps the fastest per
// level shape and precision for the rest of the process; a no-op for other radii.
cudaError_t tune_mg_bands(Ctx& c, const OpDesc& op, int dt, const void* f, void* fc, const void* ec, void* y,
                          double omega, int nrhs);
// The tuned band height of kind 0 (restriction) / 1 (prolongation) for a shape, 0 if never tuned.
int mg_band_rows(int kind, int nx, int ny, int dt);
// General multigrid pieces: fc = FW(r); u += P ec.
cudaError_t launch_fw(Ctx& c, int dt, int nx, int ny, const void* r, void* rc, int nrhs, int bc = 0);
cudaError_t launch_prolong_add(Ctx& c, int dt, int nx, int ny, const void* ec, void* u, int nrhs, int bc = 0);

// ---- vector launchers (kern_vec.cu) -------------------------------------------------
// Dense FP64 complex matvec y = A x with dtype conversions (coarsest multigrid solve); right-hand
// side b takes the matrix A + b astride complex elements (astride 0: one matrix for the batch).
cudaError_t launch_dense(Ctx& c, const double* A, int n, int dt, const void* x, void* y, int nrhs,
                         size_t astride = 0);
// Convert between dtypes: y (ty) = x (tx), n complex elements.
cudaError_t launch_convert(Ctx& c, int tx, int ty, const void* x, void* y, size_t n);
// y (ty) = x (tx) + z (tz)  (all n elements)
cudaError_t launch_add(Ctx& c, int tx, const void* x, int tz, const void* z, int ty, void* y, size_t n);
// y = D x for HZ_C128 vectors of an nx x ny grid: D = 1/2 on boundary edges, 1/4 at corners.
cudaError_t launch_row_scale(Ctx& c, int nx, int ny, const void* x, void* y, int nb);

// Batched Krylov kernels.  nb right-hand sides; vector i of rhs b lives at base + i*ldv + b*n
// (elements), so a batch of one vector index is nb*n contiguous elements.
// Multi-dot: out[b*2nv + 2i + {0,1}] = sum_e conj(V_i^b[e]) w^b[e] (double), ws: dot_ws_bytes(nv, nb).
size_t dot_ws_bytes(int nv, int nb);
// with_norm: also out[b*(2nv+1) + 2nv] = ||w^b||^2 (the per-rhs stride becomes 2nv+1).
// skip (optional, per rhs): a non-zero entry makes the kernel return without work.
cudaError_t launch_multidot(Ctx& c, int dt, const void* V, size_t ldv, int nv, const void* w, size_t n, int nb,
                            double* out, void* ws, int with_norm = 0, const double* skip = nullptr);
// w^b (dtw) -= sum_i coef[b*ldc + 2i..] V_i^b (dtv); optionally ||w^b||^2 into nrm2[b] (device doubles).
cudaError_t launch_update(Ctx& c, int dtv, const void* V, size_t ldv, int nv, const double* coef, int ldc, int dtw,
                          void* w, size_t n, int nb, double* nrm2, void* ws, const double* skip = nullptr);
// flag[b] = 1.0 when n1[b] >= eta2 * wn[b*ldw] (second Gram-Schmidt pass not needed), else 0.0
cudaError_t launch_dgks_flag(Ctx& c, const double* wn, int ldw, const double* n1, double* flag, int nb, double eta2);
// One-iteration FGMRES on the device as a minimal-residual step: from d = (b^H w, ||w||^2) per
// right-hand side (stride 3), coef = conj(b^H w) / ||w||^2 (0 when w = 0), plus iteration / call
// counters; a non-finite value sets *err.
cudaError_t launch_m1_mr(Ctx& c, const double* d, int nb, double* coef, int* its, int* calls, int* err);
// u^b (dtu) += sum_i coef[b*2nv + 2i..] X_i^b (dtx)
cudaError_t launch_combine(Ctx& c, int dtx, const void* X, size_t ldx, int nv, const double* coef, int dtu, void* u,
                           size_t n, int nb);
// y^b = alpha_b x^b: alpha complex (2 doubles per rhs) or, with recip, 1/sqrt(alpha_b) (1 double per rhs).
cudaError_t launch_scale_dev(Ctx& c, int dt, const void* x, void* y, const double* alpha_dev, int recip, size_t n,
                             int nb);

// ---- Bi-CGSTAB CSLP solver (kern_bicgstab.cu) ---------------------------------------------
// Scalars of one right-hand side, in device memory (complex values as re, im).
struct BicgState {
  double rho[2], alpha[2], omega[2], beta[2];
  double bn2, rn2, tol2;  // ||b||^2, ||r||^2, (tol ||b||)^2
  double done;            // 0 running, 1 converged, 2 stopped by a breakdown
  double its;             // completed iterations
  double total_its;       // persistent form: iterations accumulated since the last statistics read
  double nonfinite;       // persistent form: solves that ended on a non-finite residual since then
  double pad;
};
// Grid barrier of the persistent Bi-CGSTAB kernel (device memory, zeroed; one per level).
struct BicgBarrier {
  unsigned count;  // arrivals (own 128-byte line)
  unsigned pad0[31];
  unsigned gen;    // generation, polled by the waiting CTAs (own line)
  unsigned pad1[31];
  int err;         // 1: a wait exceeded its clock budget
  int pad2[31];
};
static_assert(sizeof(BicgBarrier) == 384, "BicgBarrier is three 128-byte lines");
// Persistent form: CTAs of the cooperative grid for an nx x ny level (one tile of 32 x 16 per CTA
// and round, at most the co-resident limit), 0 if it cannot be launched.
int bicg_persist_grid(int dt, int R, int nx, int ny);
// x += BiCGSTAB(M, b) for one right-hand side in one cooperative launch of `grid` CTAs (whole
// solve, tolerance tol, at most cap iterations); work: 7 n elements of dtype dt (r, two p, two v,
// s, t); part: 8 * grid doubles; st: this right-hand side's state (its, rn2, done, and the running
// totals total_its / nonfinite); bar: the level's barrier.
cudaError_t launch_bicg_persist(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* work, double* part,
                                BicgState* st, BicgBarrier* bar, int cap, double tol, int grid);
int bicg_parts(size_t n);                  // CTAs per right-hand side of the reduction passes
size_t bicg_part_bytes(size_t n, int nb);  // partial-sum buffer
// rho = ||b||^2 and the stop test's reference (r = r_hat = b is the caller's copy)
cudaError_t launch_bicg_start(Ctx& c, int dt, const void* b, size_t n, int nb, double tol, double* part,
                              BicgState* st);
// which 0: alpha = rho / (a0^H b0) with a0 = r_hat, b0 = v; which 1: omega = a0^H b0 / a1^H b1 with
// a0 = a1 = t, b0 = s, b1 = t
cudaError_t launch_bicg_dots(Ctx& c, int dt, int which, const void* a0, const void* b0, const void* a1,
                             const void* b1, size_t n, int nb, double* part, BicgState* st);
cudaError_t launch_bicg_p(Ctx& c, int dt, const void* r, void* p, const void* v, size_t n, int nb,
                          const BicgState* st);
cudaError_t launch_bicg_s(Ctx& c, int dt, const void* r, const void* v, void* s, size_t n, int nb,
                          const BicgState* st);
// x += alpha p + omega s; r = s - omega t; then rho, ||r||, the stop test and beta
cudaError_t launch_bicg_xr(Ctx& c, int dt, void* x, const void* p, const void* s, const void* t, void* r,
                           const void* rhat, size_t n, int nb, double* part, BicgState* st);

// ---- persistent GMRES (kern_gmres.cu) ---------------------------------------------------
// Per-right-hand-side control block of the cooperative GMRES kernel (device memory, zeroed).
struct GmresState {
  unsigned count;        // grid barrier arrivals (own 128-byte line: atomics only)
  unsigned pad0[31];
  unsigned gen;          // grid barrier generation (own line: polled by waiting CTAs)
  unsigned pad1[31];
  int err;               // 1: a barrier wait exceeded its clock budget
  int its;               // iterations of the last solve
  double est;            // residual estimate of the last solve
  long long total_its;   // iterations accumulated since the last statistics read
  double total_bytes;    // algorithmic bytes (reads + writes of vectors and k) since the last read
  long long total_reorth;// second Gram-Schmidt passes since the last statistics read
  long long total_ns;    // device time of the launches since the last read (%globaltimer: entry of
                         // the first CTA to the exit of the last one)
  long long launches;    // launches since the last statistics read
  unsigned long long t_start;  // entry time of the running launch (written by CTA 0)
  unsigned done;         // CTAs of the running launch that finished
  unsigned pad3;
  long long pad2[7];
};
static_assert(sizeof(GmresState) == 384, "GmresState is three 128-byte lines");
// Largest cooperative grid for the kernel variant used on a level of n nodes (0 if it cannot be
// launched).
int gmres_max_grid(int dt, int R, int cap, size_t n);
// Tile-owned form of the persistent GMRES: tile shape (*TX, *TY) for an nx x ny level and the
// number of CTAs (one per tile), 0 if no shape gives every co-resident CTA at most one tile.
int gmres_tile_form(int dt, int R, int nx, int ny, int cap, int* TX, int* TY);
// Every fitting tile shape of the tile-owned form, most tiles first; returns the count (<= maxc).
int gmres_tile_forms(int dt, int R, int nx, int ny, int cap, int* TX, int* TY, int maxc);
// x += GMRES(M, b) for one right-hand side with the tile-owned form (grid = tiles; w0: n
// elements, the updated vector the neighbours read their halos from; nflag: one unsigned per
// tile; partA/partB: 2 (cap + 1) + 2 values per CTA; Rg, st as launch_gmres_persistent).
cudaError_t launch_gmres_tile(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* V, void* w0,
                              unsigned* nflag, double* partA, double* partB, double* Rg, GmresState* st, int cap,
                              double tol, int TX, int TY, double eta2);
// Largest thread-block cluster (16 or 8 CTAs) the cluster form can run in, 0 if none.
int gmres_cluster_size(int dt, int R, int cap);
// x += GMRES(M, b), whole solve in one launch: one right-hand side on a cooperative grid of
// `grid` CTAs, or (cluster) nrhs right-hand sides, each on its own thread-block cluster of
// `grid` <= 16 CTAs; per right-hand side q the cluster form offsets b, x, w0, w1 by q n, V by
// q (cap + 1) n, partA/partB by q grid pstride, Rg by q (2 cap (cap + 1) + 2 cap + 3 pstride)
// and st by q.
// V: (cap+1) * n, w0/w1: n (dtype dt); partA/partB: grid * pstride doubles;
// Rg: 2 * cap * (cap + 1) + 2 * cap + 3 * pstride doubles (Hessenberg, y, reduced values).
cudaError_t launch_gmres_persistent(Ctx& c, const OpDesc& M, int dt, const void* b, void* x, void* V, void* w0,
                                    void* w1, double* partA, double* partB, int pstride, double* Rg, GmresState* st,
                                    int cap, double tol, int grid, bool cluster, int nrhs, double eta2);

// ---- exact coarse stencils (stencil_gen.cpp) ----------------------------------------
// 1-D Galerkin masks of level l (1-based), length 2R+1, as exact rationals rounded once.
void galerkin_masks(int level, int* R, double m[7], double l[7]);

// ---- thread-local error message -----------------------------------------------------
void set_error(const std::string& msg);

}  // namespace hz
