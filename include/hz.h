/*
 * hz.h -- C ABI of the GB300 matrix-free multilevel deflation Helmholtz library.
 *
 * Problem (Section 2): -Laplace(u) - k(x,y)^2 u = b on a rectangle, discretised by the
 * second-order 5-point stencil on a vertex-centred grid with uniform spacing h
 * (Section 2.1, Eq. for [A_h]); Sommerfeld rows eliminate the ghost point
 * u_0 = u_2 + 2 h i k_1 u_1 (Section 2.1, Sommerfeld ghost equation).
 * Solver: FGMRES right-preconditioned by the recursive two-level deflation of
 * Algorithm 1 with the CSLP M = -Laplace - (beta1 + i beta2) k^2 (Section 3.1) and the
 * MADP schedule of Section 4.4.
 *
 * Conventions shared by every entry point:
 *  - Grids are nx * ny nodes (boundary nodes included for Sommerfeld; interior
 *    unknowns only for homogeneous Dirichlet), row-major [rhs][y][x], x fastest.
 *  - Complex vectors are interleaved (re, im): HZ_C128 = 16-byte double2 elements,
 *    HZ_C64 = 8-byte float2 elements.  Batches of nrhs vectors are contiguous.
 *  - Vector pointers are DEVICE pointers owned by the caller unless a name ends in
 *    _host.  The library never frees caller memory; it allocates its own workspace
 *    in hz_setup and frees it in hz_destroy.
 *  - All work is ordered on the stream given to hz_setup (a cudaStream_t passed as
 *    void*, 0 = legacy default stream).  Calls return after enqueueing unless the
 *    algorithm needs a scalar on the host (the Krylov solvers), in which case they
 *    synchronise that stream.
 *  - Every call returns an int status (HZ_OK = 0) and never aborts; hz_strerror()
 *    names a status and hz_last_error() gives the last detailed message of the
 *    calling thread.  A handle must not be used by two host threads at once.
 */
#ifndef HZ_H
#define HZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define HZ_OK          0
#define HZ_EINVAL      1   /* invalid argument (size, pointer, level, config value) */
#define HZ_ENOMEM      2   /* device allocation failed or memory budget exceeded */
#define HZ_ENOTCONV    3   /* iteration cap reached before the tolerance */
#define HZ_EBREAKDOWN  4   /* NaN/Inf in a residual or a zero Krylov norm without convergence */
#define HZ_ETIMEOUT    5   /* a host wait on the device exceeded the configured limit */
#define HZ_ECUDA       6   /* a CUDA runtime call failed (message in hz_last_error) */
#define HZ_ENOTSUP     7   /* valid request that this build does not support */
#define HZ_PENDING     8   /* serving: the request has not finished yet */

/* ---- enumerations ---------------------------------------------------------------- */
#define HZ_BC_SOMMERFELD 0 /* first-order Sommerfeld rows, ghost equation of Section 2.1 */
#define HZ_BC_DIRICHLET  1 /* homogeneous Dirichlet (MP-1a): nx * ny interior unknowns; coarse
                              unknown I sits at fine unknown 2I + 1, a side of n coarsens to
                              (n - 1) / 2; every level applies its stencil with zeros outside */

#define HZ_PREC_FP64   0   /* every vector and scalar in complex FP64 */
#define HZ_PREC_MIXED  1   /* preconditioner (lines 5-14 of Algorithm 1) and inner levels in
                              complex FP32; outer Arnoldi, Hessenberg least squares, true
                              residual and the multigrid coarsest solve in FP64 */

#define HZ_C128 0          /* complex double, 16 bytes per element */
#define HZ_C64  1          /* complex float, 8 bytes per element */

#define HZ_OP_A 0          /* Helmholtz operator A_l (shift 1) */
#define HZ_OP_M 1          /* CSLP operator M_l (shift beta1 + i beta2) */

#define HZ_CSLP_GMRES    0 /* CSLP inverse on Krylov levels by GMRES */
#define HZ_CSLP_BICGSTAB 1 /* CSLP inverse on Krylov levels by Bi-CGSTAB */

#define HZ_MAX_LEVELS 10

#define HZ_SOLVE_INITIAL_GUESS 1u  /* hz_solve flag: u holds the initial guess on entry */

typedef struct hz_handle_s* hz_handle;

/* Grid of the finest level (Section 2.1). */
typedef struct {
  int nx, ny;   /* nodes per side, odd and coarsenable levels-1 times (Sommerfeld: n -> (n + 1)
                   / 2, at least 5 before each step; Dirichlet: n -> (n - 1) / 2, at least 3) */
  double h;     /* uniform spacing, > 0 */
  int bc;       /* HZ_BC_* */
} hz_grid;

/* Solver configuration.  hz_config_init() fills the paper's MADP defaults; every
 * field is then taken literally. */
typedef struct {
  int levels;            /* ml >= 1 deflation levels (Algorithm 1, "predefined coarsest level") */
  int precision;         /* HZ_PREC_* */
  double beta1, beta2;   /* CSLP shift, default (1, 0.5) (Section 4.3) */
  int restart;           /* outer FGMRES restart length, default 30 */
  int max_outer;         /* cap on total outer iterations, default 300 */
  double l2_tol;         /* level-2 deflated FGMRES relative tolerance, default 0.3 (Section 4.4) */
  int l2_maxit;          /* level-2 iteration cap, default 30 */
  double cslp_tol;       /* GMRES tolerance of the CSLP inverse on levels > mg_max_level, default 0.1 */
  double c_it;           /* Krylov cap floor(c_it * N_l^(1/4)), default 6 (Section 4.2) */
  double coarsest_tol;   /* coarsest-level tolerance when indefinite, default 0.1 (Section 4.1) */
  int negdef_from_level; /* first level treated as negative definite (coarsest then runs one
                            iteration); 0 = none */
  int mg_max_level;      /* CSLP by multigrid V-cycle on levels <= this, default 2 (Section 4.4) */
  double mg_omega;       /* damped-Jacobi weight, default 0.8 */
  int mg_nu1, mg_nu2;    /* pre/post smoothing sweeps, default 1 and 1 */
  int mg_coarsest_side;  /* multigrid coarsening stops at this many nodes per side, default 20 */
  int max_rhs;           /* largest nrhs any call on this handle will pass, default 1 */
  double timeout_s;      /* limit for every host wait on the device, default 600 s */
  int device_gmres;      /* 1 (default): each GMRES CSLP solve runs as one persistent kernel with
                            on-device Givens rotations: one thread-block cluster per right-hand
                            side, all in one launch, for calls on 4 or more right-hand sides on
                            levels of at most 300,000 nodes; otherwise a cooperative grid per
                            right-hand side, with one tile per CTA where the level's tiling fits
                            the GPU (FP32) and slice-distributed vector phases elsewhere;
                            2: always the cooperative grid (tile-owned where it fits);
                            3: always clusters; 4: always the slice-distributed grid;
                            0: host-driven Arnoldi steps.  Every form runs with FP32
                            (HZ_PREC_MIXED) and FP64 vectors, except the tile-owned one
                            (FP32 only).  With cslp_solver = HZ_CSLP_BICGSTAB, any non-zero
                            value runs each Bi-CGSTAB solve as one persistent cooperative launch
                            per right-hand side; 0 keeps the launch-per-step kernels */
  double reorth_eta;     /* classical Gram-Schmidt runs a second pass when the orthogonalised
                            vector keeps less than reorth_eta of its norm ("twice is enough"
                            test), default 0.1; 1 = always two passes, 0 = one pass */
  int graphs;            /* 1 (default): the coarse solves below the first level whose whole
                            subtree runs on the device (MADP: level 3) are captured once per
                            batch size as a CUDA graph and replayed; 0: launched one by one */
  int autotune;          /* 1 (default): with device_gmres = 1, time the tile-owned GMRES form at
                            each fitting tile shape and the slice-distributed form once per
                            level shape (process-wide cache, at hz_setup) and keep the fastest;
                            0: take the tile-owned form with the most tiles wherever it fits */
  int cycle_m;           /* deflated FGMRES iterations m on each level 3 .. ml-1 that has no
                            tolerance (Algorithm 1's m on the coarser levels, Section 3.2):
                            1 (default) = V-cycle, 2 = W-cycle; >= 1 */
  double level_tol[HZ_MAX_LEVELS]; /* [l-1] for levels 3 .. ml-1: > 0 solves level l to this
                            relative residual with at most l2_maxit iterations instead of
                            cycle_m iterations (tolerances on the coarser indefinite levels,
                            Sections 4.3.3 and 4.5); default 0; entries of other levels must be 0.
                            Level 2 keeps l2_tol / l2_maxit: l2_tol = 0 runs exactly l2_maxit
                            iterations (l2_maxit = 1: MADP-v1's V-cycle, Section 4.3.1) */
  int cslp_solver;       /* Krylov solver of the CSLP inverse on levels > mg_max_level, same
                            tolerance cslp_tol and cap: HZ_CSLP_GMRES (default, Section 4.2) or
                            HZ_CSLP_BICGSTAB (the earlier multilevel work's choice, Sections 3.2
                            and 4.1) */
  int sym_rows;          /* 1: solve the row-scaled system D A_h u = D b, D = 1/2 on Sommerfeld
                            boundary edges and 1/4 at corners, whose matrix is the complex
                            symmetric one Section 2.1 refers to (same solution u; the residuals
                            and the stopping test are those of the scaled system; the
                            preconditioner is built from A_h as usual); 0 (default): the
                            ghost-eliminated rows as they are.  Sommerfeld grids only */
  int per_rhs_k;         /* 1: multi-instance batch.  k_dev of hz_setup holds max_rhs wavenumber
                            fields, [max_rhs][ny][nx], and right-hand side b of every call
                            solves (or applies) the problem with field b: same grid, spacing and
                            configuration, but its own coarse wavenumbers, multigrid coarsest
                            inverse and statistics, while every sweep stays one launch over the
                            whole batch.  Calls then take nrhs <= max_rhs and use fields
                            0 .. nrhs-1.  0 (default): one field shared by every right-hand side */
} hz_config;

/* Per-right-hand-side solve statistics. */
typedef struct {
  int status;                                  /* HZ_OK or HZ_ENOTCONV / HZ_EBREAKDOWN */
  int outer_iterations;                        /* level-1 FGMRES iterations, all cycles */
  int level_iterations[HZ_MAX_LEVELS];         /* [l-1]: deflated FGMRES iterations on level l */
  int level_calls[HZ_MAX_LEVELS];              /* [l-1]: number of level-l coarse solves */
  int cslp_gmres_iterations[HZ_MAX_LEVELS];    /* [l-1]: Krylov iterations of CSLP inverses
                                                  (GMRES, or Bi-CGSTAB with cslp_solver) */
  double true_relres;                          /* ||b - A_h u|| / ||b|| in FP64 (with sym_rows:
                                                  ||D b - D A_h u|| / ||D b||) */
  double est_relres;                           /* last Arnoldi least-squares estimate */
  double ms;                                   /* wall time of the solve in milliseconds */
  int cslp_gmres_reorth[HZ_MAX_LEVELS];        /* [l-1]: second Gram-Schmidt passes of the
                                                  persistent CSLP GMRES on level l */
} hz_stats;

/* ---- set-up ------------------------------------------------------------------------ */

/* Fill *cfg with the MADP defaults listed above (levels = 1, precision = HZ_PREC_FP64). */
int hz_config_init(hz_config* cfg);

/* Build the level hierarchy (Section 3.3): per-level sizes n_l = (n_{l-1} + 1) / 2,
 * spacing 2^(l-1) h, wavenumber injected at coincident nodes, exact Galerkin coarse
 * stencils (Section 3.3, Appendix A; 1-D recursion with p = [1,4,6,4,1]/8), multigrid
 * sub-hierarchies with an FP64 dense coarsest inverse, and all workspace for nrhs <=
 * cfg->max_rhs.  k_dev: nx*ny real FP64 wavenumbers (cfg->per_rhs_k: max_rhs such fields
 * back to back), device, read during the call only.
 * stream: cudaStream_t used by every later call on the handle.
 * (Dirichlet grids: n_l = (n_{l-1} - 1) / 2, wavenumber injected at fine unknown 2I + 1.)
 * Errors: HZ_EINVAL (sizes not coarsenable, h <= 0, non-finite or non-positive k,
 * bad config), HZ_ENOMEM, HZ_ECUDA. */
int hz_setup(const hz_grid* grid, const double* k_dev, const hz_config* cfg, void* stream,
             hz_handle* out);

/* Release every resource of the handle (synchronises its stream first). */
int hz_destroy(hz_handle h);

/* Bytes of device memory the handle holds. */
int hz_memory_bytes(hz_handle h, size_t* bytes);

/* ---- the hot-path calls -------------------------------------------------------------- */

/* y = A_h x on the finest level: Section 2.1, Eq. for [A_h] with Sommerfeld ghost rows
 * (or homogeneous Dirichlet).  x, y: nrhs * nx * ny HZ_C128, device, must not overlap. */
int hz_apply(hz_handle h, const void* x, void* y, int nrhs);

/* x = P v, the A-DEF1 preconditioner P = M^-1 (I - A Q) + Q of Section 3.1 applied by
 * Algorithm 1 lines 5-14 at level 1 (coarse system solved by the recursive schedule).
 * v, x: nrhs * nx * ny HZ_C128, device.  With levels = 1, x = M^-1 v (multigrid). */
int hz_precond(hz_handle h, const void* v, void* x, int nrhs);

/* Solve A_h u = b for each of nrhs right-hand sides by FGMRES(restart) preconditioned
 * with P, to relative residual tol in the 2-norm (Section 4: zero initial guess unless
 * flags has HZ_SOLVE_INITIAL_GUESS, confirmed by the FP64 true residual).
 * b, u: HZ_C128 device vectors; stats: nrhs host entries or NULL.
 * Returns HZ_OK when every right-hand side converged, else the first failing status. */
int hz_solve(hz_handle h, const void* b, void* u, int nrhs, double tol, unsigned flags,
             hz_stats* stats);

/* hz_solve with HOST buffers: copies b to the device, solves, copies u back (all on
 * the handle's stream).  b_host, u_host: nrhs * nx * ny complex double, host memory. */
int hz_solve_host(hz_handle h, const double* b_host, double* u_host, int nrhs, double tol,
                  unsigned flags, hz_stats* stats);

/* ---- building blocks (each one step of the hot path; used by the parity tests) ---- */

/* Grid size of deflation level l (1-based): *nx, *ny. */
int hz_level_size(hz_handle h, int level, int* nx, int* ny);

/* How a single right-hand side's CSLP GMRES runs on a level (diagnostics; no counterpart in the
 * paper): *form = 0 no GMRES on this level (multigrid CSLP) or host-driven Arnoldi steps,
 * 1 persistent slice-distributed cooperative grid, 2 persistent tile-owned cooperative grid,
 * 3 one thread-block cluster; *ctas = CTAs of that launch; *cluster = CTAs per cluster used
 * for calls on several right-hand sides (0 if the cluster form is off).  Errors: HZ_EINVAL. */
#define HZ_GMRES_NONE    0
#define HZ_GMRES_SLICE   1
#define HZ_GMRES_TILE    2
#define HZ_GMRES_CLUSTER 3
int hz_level_gmres_form(hz_handle h, int level, int* form, int* ctas, int* cluster);

/* y = A_l x (op = HZ_OP_A) or M_l x (HZ_OP_M) on deflation level l.  Level 1: the
 * 5-point rows of Section 2.1; level >= 2: the re-discretised Galerkin stencils of
 * Section 3.3 with the boundary treatment of its "Boundary" paragraph.  dtype: HZ_C128
 * or HZ_C64 for both x and y (the arithmetic follows the dtype). */
int hz_level_apply(hz_handle h, int level, int op, int dtype, const void* x, void* y, int nrhs);

/* One damped-Jacobi sweep with M_l (multigrid smoother of the CSLP inverse, Section 3.2):
 * u_out = u + omega (f - M_l u) / diag(M_l).  u, f, u_out: dtype vectors on level l. */
int hz_level_jacobi(hz_handle h, int level, int dtype, const void* u, const void* f,
                    void* u_out, int nrhs);

/* Deflation restriction v_hat = Z^T v from level l to level l+1 (Algorithm 1 line 5). */
int hz_defl_restrict(hz_handle h, int level, int dtype, const void* v, void* vhat, int nrhs);

/* Deflation prolongation t = Z w from level l+1 to level l (Algorithm 1 line 11). */
int hz_defl_prolong(hz_handle h, int level, int dtype, const void* w, void* t, int nrhs);

/* Fused Algorithm 1 lines 11-13 at level l: t = Z v_til, r_til = v - A_l t.
 * v_til on level l+1; v, t, r_til on level l; all dtype.  t may be NULL. */
int hz_defl_prolong_residual(hz_handle h, int level, int dtype, const void* vtil,
                             const void* v, void* t, void* rtil, int nrhs);

/* One multigrid V-cycle approximating M_l^-1 f on level l <= mg_max_level, zero
 * initial guess (Section 3.2, CSLP by multigrid).  f, u: dtype vectors on level l. */
int hz_mg_vcycle(hz_handle h, int level, int dtype, const void* f, void* u, int nrhs);

/* Number of multigrid levels of the level-l CSLP hierarchy and the size of MG level m. */
int hz_mg_size(hz_handle h, int level, int mg_level, int* nx, int* ny);

/* CSLP inverse by unpreconditioned GMRES on M_l to relative tolerance cfg.cslp_tol,
 * at most floor(c_it * N_l^(1/4)) iterations (Section 4.2), zero initial guess.
 * b, x: dtype vectors on level l; iterations (host, nrhs entries) may be NULL. */
int hz_cslp_gmres(hz_handle h, int level, int dtype, const void* b, void* x, int nrhs,
                  int* iterations);

/* CSLP inverse by Bi-CGSTAB (van der Vorst 1992) on M_l with the same tolerance and cap as
 * hz_cslp_gmres, zero initial guess, shadow residual b.  Needs a handle configured with
 * cslp_solver = HZ_CSLP_BICGSTAB and level > mg_max_level (else HZ_EINVAL). */
int hz_cslp_bicgstab(hz_handle h, int level, int dtype, const void* b, void* x, int nrhs,
                     int* iterations);

/* ---- allocation-free check -------------------------------------------------------- */

/* Largest nrhs accepted by hz_true_residual_noalloc. */
#define HZ_NOALLOC_MAX_RHS 64

/* relres_dev[r] = ||b_r - A_h u_r||_2 / ||b_r||_2 (||b_r - A_h u_r||_2 if b_r = 0) for
 * r < nrhs, in FP64, computed without allocating any device memory.  The paper has no
 * counterpart: this call exists for callers that cannot call cudaMalloc where they
 * check a solution (e.g. a plugin whose host application owns every device
 * allocation, or a loop that must not enter the allocator).
 * b, u: nrhs * nx * ny HZ_C128 device vectors (Sommerfeld or Dirichlet grid, as the
 * handle's); relres_dev: nrhs device doubles.  Work is ordered on the handle's stream.
 * Scratch is a static device array of 1216 * 2 * HZ_NOALLOC_MAX_RHS doubles (1.25 MB)
 * that every GPU on which a handle was set up keeps until exit.  hz_setup loads the
 * array's module and looks up its address on the handle's device, so no call of this
 * entry point (the first one included) reserves device memory.  All calls share the
 * array, so calls that overlap on the GPU (several streams, threads or handles) race and
 * must be serialised by the caller.
 * Errors: HZ_EINVAL (null pointer, nrhs < 1 or > HZ_NOALLOC_MAX_RHS, or the current device
 * is not the handle's), HZ_ECUDA (a launch failed, or a CUDA error from earlier work was
 * pending on entry: the message says which). */
int hz_true_residual_noalloc(hz_handle h, const void* b, const void* u, int nrhs, double* relres_dev);

/* ---- serving ------------------------------------------------------------------------ */
/* A server runs many independent solves (different grids, wavenumber fields, configurations)
 * on the current device at once.  Each admitted request gets its own handle and stream:
 * hierarchy and Krylov bases stay resident for the whole solve, and the work of concurrent
 * requests overlaps on the GPU.  Requests are taken in arrival order; one whose footprint
 * (hz_estimate_bytes + its device copies of k, b and u) does not fit what the running
 * requests leave of the budget waits, while later requests that fit are admitted.  A
 * request's result does not depend on what else runs: it equals hz_solve on a handle of its
 * own.  The paper solves one problem at a time; this layer is not part of its method. */
typedef struct hz_server_s* hz_server;

typedef struct {
  hz_grid grid;            /* finest grid, HZ_BC_SOMMERFELD or HZ_BC_DIRICHLET (interior unknowns) */
  hz_config config;        /* solver configuration; config.max_rhs >= nrhs */
  const double* k_host;    /* nx*ny real FP64 wavenumbers (config.per_rhs_k: config.max_rhs
                              fields back to back), host; copied by hz_submit */
  const double* b_host;    /* nrhs*nx*ny HZ_C128 right-hand sides, host; copied by hz_submit */
  double* u_host;          /* nrhs*nx*ny HZ_C128 solutions, host, caller-owned; written by the
                              server before the request is reported finished (zero initial guess) */
  hz_stats* stats_host;    /* nrhs statistics written at completion, or NULL */
  int nrhs;                /* right-hand sides solved together, >= 1 */
  double tol;              /* outer relative residual tolerance, in (0, 1) */
} hz_request;

typedef struct {
  long long completed;     /* requests that finished with HZ_OK */
  long long failed;        /* requests that finished with another status */
  long long queued;        /* requests waiting for admission */
  int active;              /* requests running now */
  double p50_ms, p99_ms;   /* latency (submit to result on the host) over completed requests */
  double solves_per_s;     /* completed requests / (last completion - first submit) */
  size_t peak_bytes;       /* largest sum of admitted footprints seen */
  size_t budget_bytes;     /* the budget given to hz_server_create */
  long long merged_solves;   /* solves that ran several requests as one batch */
  long long merged_requests; /* requests that ran in such merged solves */
} hz_server_stats;

/* Device bytes hz_setup would allocate for this grid and configuration (bytes requested
 * from cudaMalloc; an upper bound of hz_memory_bytes of the resulting handle).  Host-only.
 * Errors: HZ_EINVAL (null pointer). */
int hz_estimate_bytes(const hz_grid* grid, const hz_config* cfg, size_t* bytes);

/* Start a server on the calling thread's current device with max_active worker threads
 * (at most that many requests run at once) and a device-memory budget in bytes.
 * Errors: HZ_EINVAL (null out, max_active < 1, zero budget), HZ_ENOMEM, HZ_ECUDA. */
int hz_server_create(size_t mem_budget_bytes, int max_active, hz_server* out);

/* Merge compatible requests (same grid, tolerance and configuration apart from max_rhs and
 * per_rhs_k) that are queued when a worker takes one of them into one multi-instance solve of
 * at most max_batch_rhs right-hand sides (every right-hand side keeps its request's wavenumber
 * field: per_rhs_k), as long as the merged footprint fits the remaining budget.  Each request
 * still gets its own solution, statistics and status; they equal its solve alone up to the
 * summation order of the GMRES form the batch size selects.  0 or 1 (the default): no merging.
 * Errors: HZ_EINVAL (null server, max_batch_rhs outside [0, 1024]). */
int hz_server_set_batching(hz_server s, int max_batch_rhs);

/* Queue a request; *ticket identifies it.  k and b are copied before the call returns; u_host
 * and stats_host must stay valid until the request is reported finished.
 * Errors: HZ_EINVAL (null pointer, nrhs < 1, tol outside (0, 1), max_rhs < nrhs, Dirichlet
 * grid), HZ_ENOMEM (footprint larger than the whole budget).  Errors of the solve itself
 * (bad sizes or configuration, device failures, HZ_ENOTCONV) are the request's final status. */
int hz_submit(hz_server s, const hz_request* req, uint64_t* ticket);

/* HZ_PENDING while the request is queued or running, else its final status; *latency_ms
 * (may be NULL) receives submit-to-completion time once finished.  On a failed request
 * hz_last_error() of the calling thread then holds the request's detailed message. */
int hz_poll(hz_server s, uint64_t ticket, double* latency_ms);

/* Block up to timeout_s seconds for the request; returns like hz_poll, or HZ_ETIMEOUT. */
int hz_wait(hz_server s, uint64_t ticket, double timeout_s, double* latency_ms);

/* Counters and latency percentiles since creation. */
int hz_server_report(hz_server s, hz_server_stats* out);

/* Let running requests finish, finish queued ones with HZ_EINVAL without running them,
 * join the workers and free the server (tickets become invalid). */
int hz_server_destroy(hz_server s);

/* ---- diagnostics ------------------------------------------------------------------- */

/* Name of a status code. */
const char* hz_strerror(int status);

/* Last detailed error message of the calling thread ("" if none). */
const char* hz_last_error(void);

/* Per-kernel timing with CUDA events on the handle's stream: enable records an event
 * pair around every launch of the kernel family `family` (see hz_kernel_family_name);
 * read returns the number of launches, their summed milliseconds and their summed
 * algorithmic bytes since enable; hz_profile_read also accepts family + 256 * l to read
 * only the launches made for deflation level l (1-based).  Reading synchronises the stream. */
int hz_profile_enable(hz_handle h, int family, int enable);
int hz_profile_read(hz_handle h, int family, long long* launches, double* ms, double* bytes);
const char* hz_kernel_family_name(int family);
int hz_kernel_family_count(void);

/* Number of CUDA kernels this handle has launched since hz_setup (every launch of the
 * library's own kernels on the handle's stream, including the set-up launches). */
int hz_launch_count(hz_handle h, long long* launches);

/* Device-side timing of the persistent CSLP GMRES kernels (Section 4.2 solves on levels >= 3),
 * always on and valid inside CUDA graphs: each launch measures itself with %globaltimer, from
 * the entry of its first CTA to the exit of its last (the cluster form: per right-hand side).
 * Returns, for deflation level `level` (0 = all levels), the launches, their summed
 * milliseconds and their summed algorithmic bytes folded in by the hz_solve calls since the
 * last reset; reset != 0 clears the totals after reading.  Errors: HZ_EINVAL. */
int hz_gmres_device_time(hz_handle h, int level, int reset, long long* launches, double* ms, double* bytes);

#ifdef __cplusplus
}
#endif
#endif /* HZ_H */
