/*
 * nrmg.h -- C ABI of the GB300 (sm_103a) nonlinear-multigrid solver for the
 * regularized Hermite moment discretization of the BGK / Shakhov / ES-BGK Boltzmann
 * equation on a 2D cavity, after Hu & Li, "An efficient nonlinear multigrid
 * solver for the simulation of rarefied gas cavity flow" (arXiv 2206.13164).
 *
 * Every compute step runs in the library's own CUDA kernels on one GPU.
 *
 * Conventions shared by all calls
 * -------------------------------
 * Units are nondimensional (molecular mass 1, velocities in sqrt(R T0)).
 * Grid: nx x ny cells on [0,lx] x [0,ly], uniform unless nrmg_set_spacing
 *   gives column widths and row heights; cell (i,j) has index c = j*nx + i,
 *   i along x.  Levels are numbered as in Algorithm 2 of the
 *   paper: level 0 is the coarsest grid, level levels-1 the finest; level l
 *   has (nx >> (levels-1-l)) x (ny >> (levels-1-l)) cells, formed by merging
 *   2x2 cells (Sec. 3.2.2).
 * Cell state (Sec. 2.2, eq. truncated-dis, Grad choice): a parameter row
 *   (u1, u2, u3, theta) and the coefficients f_alpha, |alpha| <= M, in graded
 *   order (|alpha| ascending, then alpha_1 descending, then alpha_2
 *   descending), N_M = (M+1)(M+2)(M+3)/6 doubles.  States handed to the
 *   library must be in Grad form (f_0 = rho > 0, f_{e_d} = 0,
 *   sum_d f_{2e_d} = 0, theta > 0), planar (u3 = 0 and f_alpha = 0 for odd
 *   alpha_3: the symmetry of a flow with d/dx3 = 0).  Planar states stay planar
 *   exactly, so the kernels form only the coefficients with even alpha_3; the
 *   calls that take a state or a right-hand side reject non-planar input.
 * Device arrays are row-major: params [cells][4], coefficients
 *   [cells][N_M] (dense, no padding), all FP64.
 * Walls: index 0 bottom (y = 0), 1 right (x = lx), 2 top (y = ly),
 *   3 left (x = 0).  A wall may move tangentially only.
 *
 * Memory and streams: the caller owns every device buffer, including the
 * workspace handed to nrmg_create (size from nrmg_workspace_bytes); the
 * library never allocates device memory and never frees caller memory.  All
 * work is issued on the caller's stream (a cudaStream_t passed as void*).
 * Calls that return host scalars synchronize that stream; the others are
 * asynchronous.  Device-side failures (a non-physical state, a scheduler wait
 * that ran out) are recorded in a device status word and returned by the next
 * synchronizing call.  No call aborts or exits the process.  A context must
 * be used from one host thread at a time.
 */
#ifndef NRMG_H
#define NRMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NRMG_OK = 0,
  NRMG_ERR_ARG = 1,           /* invalid argument; nothing was launched */
  NRMG_ERR_CUDA = 2,          /* a CUDA call failed (launch or synchronize) */
  NRMG_ERR_OOM = 3,           /* the workspace is smaller than nrmg_workspace_bytes */
  NRMG_ERR_NONPHYSICAL = 4,   /* rho <= 0, theta <= 0 or a non-finite value appeared */
  NRMG_ERR_NOT_CONVERGED = 5, /* nrmg_solve reached max_cycles above tol */
  NRMG_ERR_TIMEOUT = 6        /* a sweep-scheduler wait ran out (about 2 s); results are invalid */
} nrmg_status;

typedef struct nrmg_ctx nrmg_ctx;

/* nx, ny must be divisible by 2^(levels-1); 1 <= levels <= 16. */
typedef struct {
  int nx, ny;
  double lx, ly;
  int levels;
} nrmg_grid;

/* Wall velocity (u[n] = 0 along the wall normal, u[2] = 0), temperature and
 * accommodation coefficient chi in [0,1] (1 = fully diffuse). */
typedef struct {
  double u[3];
  double theta;
  double chi;
} nrmg_wall;

typedef enum { NRMG_BGK = 0, NRMG_SHAKHOV = 1, NRMG_ESBGK = 2 } nrmg_model;

/* Collision frequency nu = beta sqrt(pi/2) rho theta^(1-omega) / Kn
 * (Sec. 4, eq. nu-shakhov; the paper takes beta = 1 for Shakhov and
 * beta = Pr for ES-BGK).  Pr is used by the Shakhov model (eq. Shakhov-f^E)
 * and the ES-BGK model (eq. ES-f^E, the Gaussian of covariance
 * Lambda = theta I + (1 - 1/Pr) sigma / rho, expanded in the cell's basis up
 * to degree M); either with Pr = 1 is BGK (Sec. 2.1). */
typedef struct {
  int model; /* nrmg_model */
  double Pr, omega, beta;
} nrmg_collision;

/* Scheme and cycle options.
 *   order 1: face states are cell states; order 2: linear reconstruction of
 *     eq. (moments-recon) with slope 1 (central, as printed) or 2 (van Albada
 *     limited); a cell next to a wall has zero slope along that axis.
 *   cfl: CFL number of eq. (local-CFL) (the paper uses 0.9).
 *   s1, s2: pre/post FS steps, s3: FS steps of the coarsest solver, gamma: 1
 *     V-cycle, 2 W-cycle (Algorithm 2; the paper uses 2, 2, 4, 1).
 *   precision: 0 = FP64 throughout; 1 = mixed: on every level above the
 *     coarsest, each FS^s of Algorithm 2 becomes one FP64 defect evaluation
 *     d = r - R(f), s FP32 Gauss-Seidel steps (same cell order) on a
 *     linearization L e = d for the correction e (frozen cell bases, time steps
 *     and collision frequencies; the reconstruction of the same order with the
 *     limiter's weights frozen at f), and the FP64 update f <- Grad(f + e); the
 *     residual, the transfers, the coarsest solve and the convergence test stay
 *     FP64, so the iteration converges to the same FP64 fixed point R(f) = r.
 *     Where the frozen limiter weights make the mixed cycle stall (see
 *     nrmg_solve), nrmg_solve finishes with FP64 smoothing.  nrmg_smooth always
 *     runs the FP64 Algorithm 1. */
typedef struct {
  int order, slope;
  double cfl;
  int s1, s2, s3, gamma;
  int precision;
  double dtnu; /* > 0: local time step capped at dtnu / nu, the collision frequency (0 = the
                  CFL step of eq. local-CFL alone); changes the iteration, not its fixed point */
} nrmg_opts;

/* Bytes of device workspace nrmg_create needs; 0 when the arguments are invalid. */
size_t nrmg_workspace_bytes(const nrmg_grid *grid, int M, const nrmg_opts *opts);

/* Create a solver over a caller-owned device workspace (>= 256-byte aligned,
 * ws_bytes >= nrmg_workspace_bytes).  M in [3, 16] (Shakhov's f^E needs
 * |alpha| = 3 and conservation of energy by the flux needs M >= 3).  The
 * initial state on every level is the global Maxwellian rho = 1, u = 0,
 * theta = 1.  stream: cudaStream_t (NULL = legacy default stream).
 * Errors: NRMG_ERR_ARG (bad sizes, M, Kn <= 0, theta_w <= 0, wall moving
 * along its normal, unknown model/options), NRMG_ERR_OOM, NRMG_ERR_CUDA. */
nrmg_status nrmg_create(const nrmg_grid *grid, int M, double Kn, const nrmg_wall walls[4],
                        const nrmg_collision *coll, const nrmg_opts *opts, void *dev_workspace,
                        size_t ws_bytes, void *cuda_stream, nrmg_ctx **out);

/* Release the host-side context (the workspace stays with the caller). */
nrmg_status nrmg_destroy(nrmg_ctx *ctx);

/* Copy a state (device arrays, layout above) into level `level`.  Setting
 * the finest level also resets the reference mass of the mass correction and
 * the reference residual ||R(f^0)|| of eq. (relative-residual).  Synchronizes.
 * Errors: NRMG_ERR_ARG for a non-planar state, NRMG_ERR_NONPHYSICAL for
 * rho <= 0, theta <= 0 or a non-finite value (the level is then undefined). */
nrmg_status nrmg_set_state(nrmg_ctx *ctx, int level, const double *dev_params, const double *dev_coeffs);

/* Copy level `level`'s state out to device arrays (either may be NULL). */
nrmg_status nrmg_get_state(nrmg_ctx *ctx, int level, double *dev_params, double *dev_coeffs);

/* The same two calls with HOST arrays (same dense layout: params [cells][4], coefficients
 * [cells][N_M]), for callers whose state lives in host memory.  Each array moves with one
 * cudaMemcpyAsync / cudaMemcpy2DAsync on the context's stream (the coefficient rows go
 * straight into their padded device rows); page-locked host memory makes the copies
 * asynchronous DMA.  nrmg_set_state_host then checks the state as nrmg_set_state does and
 * synchronizes; nrmg_get_state_host synchronizes before it returns (either pointer may be
 * NULL).  Errors as nrmg_set_state / nrmg_get_state. */
nrmg_status nrmg_set_state_host(nrmg_ctx *ctx, int level, const double *host_params, const double *host_coeffs);
nrmg_status nrmg_get_state_host(nrmg_ctx *ctx, int level, double *host_params, double *host_coeffs);

/* Set the right-hand side r of level `level` (the r of Algorithm 1),
 * expanded in the per-cell bases dev_rparams; NULL pointers clear it (r = 0).
 * Algorithm 2 overwrites the r of every level below the finest.  Synchronizes.
 * Errors: NRMG_ERR_ARG for a non-planar r, NRMG_ERR_NONPHYSICAL for a
 * non-finite r or a basis with theta <= 0. */
nrmg_status nrmg_set_rhs(nrmg_ctx *ctx, int level, const double *dev_rparams, const double *dev_rcoeffs);

/* `steps` fast-sweeping steps FS(f, r) (Sec. 3.1, Algorithm 1) on level
 * `level`, in place.  Each step runs the four sweeps D1..D4; every sweep
 * reproduces the serial cell order of the paper exactly (anti-diagonal
 * wavefronts with per-cell dependency counters).  Asynchronous. */
nrmg_status nrmg_smooth(nrmg_ctx *ctx, int level, int steps);

/* `steps` forward Euler steps on level `level` (Sec. 2.4, eq. euler-scheme),
 * the paper's comparison scheme (not part of the multigrid cycle): every cell
 * advances from the same old state with one step for the whole level, the
 * smallest local step of eq. (local-CFL) (eq. global-CFL; each capped at
 * dtnu / nu when dtnu > 0), then returns to Grad form.  Uses the level's
 * defect buffer.  Asynchronous. */
nrmg_status nrmg_euler(nrmg_ctx *ctx, int level, int steps);

/* Forward Euler steps on the finest level until ||R(f)|| / ||R(f^0)|| <= tol
 * (eq. relative-residual) or max_steps; *steps_out (may be NULL) = the steps
 * taken, *rel_res_out (may be NULL) = the final relative residual.
 * NRMG_ERR_NOT_CONVERGED when tol was not reached.  Synchronizes every step. */
nrmg_status nrmg_euler_solve(nrmg_ctx *ctx, double tol, int max_steps, int *steps_out, double *rel_res_out);

/* R_ij(f) - r_ij of every cell of level `level` (eq. ode-system, each row in
 * its cell's basis) into dev_R_out ([cells][N_M], may be NULL), and the
 * residual norm of eq. (relative-residual) into *norm_out (may be NULL;
 * synchronizes when non-NULL). */
nrmg_status nrmg_residual(nrmg_ctx *ctx, int level, double *dev_R_out, double *norm_out);

/* One NMG_K(f, 0) step (Algorithm 2, gamma-cycle with s1/s2/s3 FS steps,
 * restriction of eq. fH, coarse problem of eq. coarse-grid-problem, update of
 * eq. rewritten-update), then the total-mass correction of the finest level.
 * *rel_res_out (may be NULL) receives ||R(f)|| / ||R(f^0)||; synchronizes. */
nrmg_status nrmg_fas_cycle(nrmg_ctx *ctx, double *rel_res_out);

/* Cycles until ||R(f)|| / ||R(f^0)|| <= tol (eq. relative-residual) or
 * max_cycles.  NRMG_ERR_NOT_CONVERGED when tol was not reached.
 * precision 1: when the smallest relative residual seen has fallen by less than
 * a factor 0.8 over the last 8 cycles, the remaining cycles of this call smooth
 * in FP64 (nrmg_mixed_fallback then returns 1); each call starts mixed. */
nrmg_status nrmg_solve(nrmg_ctx *ctx, double tol, int max_cycles, int *cycles_out, double *rel_res_out);

/* 1 when the last nrmg_solve of a precision-1 context switched to FP64
 * smoothing because the mixed cycle stalled, else 0 (also for a NULL ctx). */
int nrmg_mixed_fallback(const nrmg_ctx *ctx);

/* Macroscopic fields of the finest level (eq. moments-relation) into
 * dev_out [cells][14]: rho, u1, u2, u3, theta, s11, s12, s13, s22, s23, s33,
 * q1, q2, q3.  Asynchronous. */
nrmg_status nrmg_fields(nrmg_ctx *ctx, double *dev_out);

/* Two-grid building blocks of Algorithm 2, for tests and custom cycles:
 * setup computes the defect of level lf, restricts state and defect to level
 * lf-1 and forms its r (eq. coarse-grid-problem); update applies
 * eq. (rewritten-update) to level lf. */
nrmg_status nrmg_two_grid_setup(nrmg_ctx *ctx, int lf);
nrmg_status nrmg_two_grid_update(nrmg_ctx *ctx, int lf);

/* Rescale the finest level to its reference total mass (the correction
 * applied after each NMG step). */
nrmg_status nrmg_mass_correct(nrmg_ctx *ctx);

/* Persistent CTAs per SM of this context's sweep launches (the FP64 sweeps and the FP32
 * correction sweeps, each capped at its kernel's occupancy); 0 restores the occupancy, the
 * default.  Fewer resident CTAs give each cell update more of its SM's FP64 rate, more give
 * the wavefront more look-ahead; the Python binding's autotuner times the choices.  The
 * iteration and its results do not depend on it.  NRMG_ERR_ARG outside [0, limit], where
 * nrmg_grid_limit returns the limit (the larger of the two kernels' occupancies). */
nrmg_status nrmg_set_grid(nrmg_ctx *ctx, int ctas_per_sm);
int nrmg_grid_limit(const nrmg_ctx *ctx);

/* Two-CTA clusters for the FP64 sweeps of small levels (the paper has no counterpart: it is a
 * schedule of the same Algorithm 1).  A level whose wavefront is shorter than the GPU is wide
 * leaves most SMs idle while one SM's FP64 pipe bounds each cell update; levels with at most
 * max_cells cells (0: none; default 16384, i.e. up to 128 x 128) then split every cell update over a cluster of two
 * CTAs on two SMs: one takes the x faces, the other the y faces, r, the collision and the
 * projection back to Grad form, the halves meeting in distributed shared memory (one
 * cluster CTA per SM on levels of at most 4096 cells, two per SM above).  The serial
 * order, and so the result up to rounding, is unchanged.  nrmg_cluster_capacity: clusters that
 * fit on the device at once (0: cluster launch unavailable, the setting is then ignored). */
nrmg_status nrmg_set_cluster(nrmg_ctx *ctx, int max_cells);

/* Non-uniform grid (Sec. 2.4: the local time step of eq. local-CFL serves non-uniform grids):
 * host_hx[nx] and host_hy[ny] are the widths of the finest level's columns and rows, positive
 * and adding up to lx and ly (to 1e-12); a coarse cell merges two columns and two rows of the
 * next finer level, whose widths add.  Each cell's flux differences are divided by its own
 * widths, its time step takes them, the second-order slopes use the distances between cell
 * centres (central: (q+ - q-) / (hm + hp); van Albada: the average of the one-sided
 * differences scaled to the cell's width, (q0 - q-) h / hm and (q+ - q0) h / hp), the norm of
 * eq. relative-residual and the mass weigh each cell by its area, and the restriction
 * averages the four children with their areas.  Call after nrmg_create and before any state
 * or right-hand side: every level returns to the global Maxwellian and the reference mass and
 * residual are reset (a batch takes the spacing its contexts have when it is created).
 * Synchronizes.  Errors: NRMG_ERR_ARG (a width <= 0 or not finite, sums off lx or ly). */
nrmg_status nrmg_set_spacing(nrmg_ctx *ctx, const double *host_hx, const double *host_hy);
int nrmg_cluster_capacity(const nrmg_ctx *ctx);

/* Fix the reference of the following cycles: the total mass the correction restores
 * (mass > 0; 0 keeps the current one) and the norm the relative residual divides by
 * (res0 > 0; 0 keeps the current one).  While a residual reference is fixed, nrmg_solve and
 * nrmg_batch_solve measure against it instead of the residual of the state they start from,
 * so a solve from a predicted start stops at the same discrete residual as one from the
 * global Maxwellian.  nrmg_set_state on the finest level clears both.  NRMG_ERR_ARG for a
 * negative or non-finite value.  The paper has no counterpart (its solves start from the
 * global Maxwellian). */
nrmg_status nrmg_set_reference(nrmg_ctx *ctx, double mass, double res0);

/* Failure-detection check (no counterpart in the paper): one FS launch on `level` whose
 * update counters are preset to a value no update ever publishes, so the first dependency
 * wait runs out after its time limit (about 2 s), every CTA leaves, and the call returns
 * NRMG_ERR_TIMEOUT.  No cell is updated; the context stays usable.  Synchronizes. */
nrmg_status nrmg_debug_stalled_sweep(nrmg_ctx *ctx, int level);

/* Synchronize the stream and return (and clear) the device status. */
nrmg_status nrmg_sync(nrmg_ctx *ctx);

/* Number of the library's kernel launches issued so far on this context. */
long long nrmg_launch_count(const nrmg_ctx *ctx);

/* Event timing of the sweep kernel (measurement aid; the paper has no counterpart).  While
 * profiling is on, every FS^steps launch is bracketed by CUDA events on the context's stream
 * (at most 65536 launches are recorded).  nrmg_fs_profile synchronizes, returns the summed
 * event time in ms, the number of timed launches, and the cell updates they performed
 * without and with a right-hand side r (any pointer may be NULL), then resets the record. */
nrmg_status nrmg_set_profiling(nrmg_ctx *ctx, int on);
/* The same record split by level (arrays of `levels` entries: summed ms, cell updates);
 * synchronizes and does not reset the record. */
nrmg_status nrmg_fs_profile_levels(nrmg_ctx *ctx, double *ms_per_level, long long *updates_per_level);
nrmg_status nrmg_fs_profile(nrmg_ctx *ctx, double *ms, long long *launches, long long *updates_no_r,
                            long long *updates_r);
/* The residual kernel's record (every mode: norms, defects, coarse right-hand sides), kept
 * while profiling is on (at most 16384 launches): summed event time in ms, timed launches,
 * and the cells evaluated without and with a right-hand side r; synchronizes, then resets. */
nrmg_status nrmg_residual_profile(nrmg_ctx *ctx, double *ms, long long *launches, long long *cells_no_r,
                                  long long *cells_r);

/* Residual without any device allocation.  The paper has no counterpart: this entry point is
 * for callers that cannot allocate device memory themselves (for example code running under
 * an allocator that forbids cudaMalloc, or a host application that only holds device pointers
 * handed to it), and so cannot provide the workspace nrmg_create needs.  It evaluates
 * R_ij(f) on the single grid `grid` (nx x ny cells; `levels` is only checked for validity)
 * with the same kernel as nrmg_residual (r = 0): the residual rows into dev_R_out
 * ([cells][N_M] dense, may be NULL) and the norm of eq. (relative-residual) into *norm_out
 * (may be NULL).  dev_params / dev_coeffs: the state, layout as above (device, read only).
 * All scratch (index tables, wall matrices, a padded copy of the state, reduction partials,
 * the status word) lives in one file-scope device array of 16 MiB
 * (NRMG_NOALLOC_SCRATCH_BYTES) that every GPU loading the library holds until exit; the call
 * makes no cudaMalloc/cudaFree and no allocating library call.  Sizes: the call fits when
 * cells * (5 + N_M rounded up to 4) * 8 bytes (params, padded coefficients and theta^(1-omega)
 * of every cell) plus at most 160 KB of index and wall tables, reduction partials and 256-byte
 * alignment fit in 16 MiB (e.g. 128x128 at M = 5, 64x64 at M = 10); larger problems return
 * NRMG_ERR_OOM before any GPU work.  Each call looks up the array's device address on the
 * current device (cudaGetSymbolAddress, with that device current; the device of the state
 * pointers must be the current one); the first call on a device loads the library's device
 * code there and should come before any stream capture.  Every call shares the
 * array and it keeps the last call's contents; calls that overlap on the GPU (other streams,
 * other host threads) race and must be serialized by the caller.  Synchronizes the stream.
 * Errors: NRMG_ERR_ARG (as nrmg_create), NRMG_ERR_OOM (too large), NRMG_ERR_NONPHYSICAL,
 * NRMG_ERR_CUDA. */
nrmg_status nrmg_residual_noalloc(const nrmg_grid *grid, int M, double Kn, const nrmg_wall walls[4],
                                  const nrmg_collision *coll, const nrmg_opts *opts, const double *dev_params,
                                  const double *dev_coeffs, double *dev_R_out, double *norm_out,
                                  void *cuda_stream);

/* Batches (the paper solves one cavity at a time; this is the batched form).  A batch runs
 * the V-cycles of several contexts in lockstep, aligned by depth below each context's finest
 * level: every FS stage of all problems (pre-smoothing at one depth together with the
 * coarsest solves reached there, or post-smoothing at one depth) is ONE persistent launch
 * whose work queue merges the problems' exact-order schedules by earliest start, so small
 * problems share the GPU.  Contexts must have the same order, slope, s1, s2, s3, model,
 * gamma = 1 and precision 0; grids, M, Kn and walls may differ (the launch sizes its shared
 * memory for the largest M, and a CTA loads the index tables of an item's M when it changes).
 * All batch work is issued on
 * the first context's stream.  The caller owns the batch workspace (>= 256-byte aligned,
 * size from nrmg_batch_workspace_bytes, 0 when the contexts are incompatible); the batch
 * keeps pointers to the contexts, which must outlive it.  Per-problem results follow
 * nrmg_fas_cycle / nrmg_solve (arrays of n entries); a problem's cycle count is the cycle at
 * which it first reached tol; nrmg_batch_solve keeps cycling until every problem has. */
typedef struct nrmg_batch nrmg_batch;
size_t nrmg_batch_workspace_bytes(nrmg_ctx *const *ctxs, int n);
nrmg_status nrmg_batch_create(nrmg_ctx *const *ctxs, int n, void *dev_workspace, size_t ws_bytes,
                              nrmg_batch **out);
nrmg_status nrmg_batch_destroy(nrmg_batch *batch);
nrmg_status nrmg_batch_fas_cycle(nrmg_batch *batch, double *rel_res_out);
nrmg_status nrmg_batch_solve(nrmg_batch *batch, double tol, int max_cycles, int *cycles_out, double *rel_res_out);
long long nrmg_batch_launch_count(const nrmg_batch *batch);
/* Persistent CTAs per SM of the batched FS launches (1 .. the kernel's occupancy; default the
 * occupancy): the knob the batch autotuner sweeps. */
nrmg_status nrmg_batch_set_grid(nrmg_batch *batch, int ctas_per_sm);
/* 1 when the batched cycle is replayed as a CUDA graph: the first nrmg_batch_fas_cycle runs
 * eagerly, the second captures the cycle's launches (on a stream other than the legacy
 * default stream) and every later one replays them; changing the grid captures again. */
int nrmg_batch_graph(const nrmg_batch *batch);

/* Human-readable name of a status, and the last error message of a context
 * (a static empty string when there is none; ctx may be NULL). */
const char *nrmg_status_str(nrmg_status s);
const char *nrmg_last_error(const nrmg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* NRMG_H */
