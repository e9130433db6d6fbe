/*
 * wl.h - C ABI of the GB300 WaterLily time-step library (libwl.so).
 *
 * One simulation ("sim") is an incompressible viscous flow on a uniform staggered
 * Cartesian grid of n_0 x n_1 [x n_2] cells (grid units: cell width 1).  One time
 * step (the paper's simstep!, Section 3 and Table 2) is:
 *   convdiff!  third-order upwind-biased finite-volume convection + viscous flux
 *              (Section 2; kappa = 1/3 face value with Koren's limiter),
 *   BDIM!      Boundary Data Immersion blend with the body's signed-distance field
 *              (Section 2, Weymouth & Yue 2011),
 *   BC!        domain boundary conditions (Table 2),
 *   project!   pressure projection with a geometric-multigrid Poisson solve on the
 *              BDIM-modified matrix (Section 2, Lauber 2022, Weymouth 2022),
 *   CFL!       adaptive time step (Section 2, Table 2),
 * arranged as a Heun predictor-corrector with a projection after each stage.
 *
 * Layout of every field that crosses this interface: interior cells only, float32,
 * x fastest: scalar index i + n_0*(j + n_1*k); a velocity is D consecutive blocks
 * of n_0*n_1*n_2 values, block c holding u_c on the LOWER c-face of each cell
 * (the staggered convention of the pressure-gradient loop of Section 2,
 * u[I,i] -= coeff[I,i]*(p[I]-p[I-del(i)])).  The upper boundary face of a
 * non-periodic direction is not stored: it always carries the boundary value U_c.
 *
 * Ownership: the library owns every device buffer of a sim.  They come from one
 * workspace: either allocated by the library (cudaMallocAsync on the sim's stream)
 * or supplied by the caller through wl_opts.workspace (size from
 * wl_workspace_bytes), in which case the caller keeps ownership and must keep it
 * alive until wl_destroy.  Callers own every dst/src pointer they pass.
 *
 * Streams: every call enqueues its work on wl_opts.stream (NULL = the legacy
 * default stream) and returns without waiting, except where a host output is
 * written (noted per call); those synchronise the stream.  A handle is not
 * thread-safe.
 *
 * Errors: every int-returning call returns WL_OK (0), a negative error or a
 * positive warning.  wl_last_error() gives a one-line message.  After
 * WL_ENONFINITE the sim is poisoned and further steps return it again.
 */
#ifndef WL_H
#define WL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WL_OK 0
#define WL_EINVAL (-1)     /* bad argument (dims, sizes, null pointers, field ids) */
#define WL_ENOMEM (-2)     /* allocation failed or supplied workspace too small */
#define WL_ECUDA (-3)      /* a CUDA runtime call failed; see wl_last_error */
#define WL_ENONFINITE (-4) /* a non-finite dt or residual was produced */
#define WL_ETIMEOUT (-5)   /* a device-side bounded wait gave up (a staged copy never arrived) */
#define WL_WNOTCONV 1      /* multigrid hit max_vcycles before tol; state stays valid */
#define WL_NODEBUG 2       /* wl_debug_bounds called on a library built without the bounds checks */

/* field ids for wl_get_field / wl_set_field */
#define WL_FIELD_U 0    /* velocity, D blocks (read/write) */
#define WL_FIELD_P 1    /* pressure p (read/write); also the multigrid unknown */
#define WL_FIELD_DIV 2  /* divergence of the current velocity, sum_c u_c[I+e_c]-u_c[I] (read) */
#define WL_FIELD_MU0 3  /* BDIM zeroth moment = Poisson face coefficient, D blocks (read) */
#define WL_FIELD_Z 4    /* right-hand side of the fine multigrid system (read/write) */
#define WL_FIELD_UPRED 5 /* projected predictor velocity u' that stage 2 reads, D blocks (read/write) */
#define WL_FIELD_USTAGE 6 /* output of the last wl_stage call, D blocks (read) */
#define WL_FIELD_EXIT 7  /* convective exit (wl_opts.exit_bc): normal velocity on the upper x face,
                            n_1 [x n_2] values, y fastest (read/write) */

/* body kinds */
#define WL_BODY_NONE 0
#define WL_BODY_SPHERE 1 /* circle in 2-D, sphere in 3-D: centre, radius */
#define WL_BODY_TORUS 2  /* 3-D: ring of radius `radius` in the y-z plane about the x axis, tube radius `radius2` */
#define WL_BODY_FIELD 3  /* any shape: its signed distance sampled at the grid's nodes (`sdf_nodes`) */

typedef struct wl_sim* wl_handle;

/* Immersed body, given by its analytic signed-distance function (Section 2: the
 * body is defined by a signed distance; its normals and kernel moments are taken
 * from it).  Positions in grid units (cell I spans [I, I+1)). */
typedef struct {
  int kind;
  double center[3];
  double radius;
  double radius2;
  /* WL_BODY_FIELD: host array of the signed distance (in cells, negative inside) at the
   * grid's nodes, positions (i, j, k) for 0 <= i <= n0 etc.: (n0+1)(n1+1)(n2+1) values in
   * 3-D, (n0+1)(n1+1) in 2-D, x fastest; copied by wl_create.  Between nodes the distance
   * is multilinear and the normal is the normalised gradient of that interpolant (exact
   * for planes; O(h^2) for smooth shapes).  Unused (may be NULL) for the other kinds. */
  const float* sdf_nodes;
} wl_body;

typedef struct {
  double tol;            /* Poisson tolerance on ||div u - A x||_inf with x = p*w*dt (default 1e-6) */
  int max_vcycles;       /* per projection (default 32) */
  int post;              /* red-black Gauss-Seidel sweeps after each coarse correction (default 4) */
  double eps;            /* BDIM kernel half-width in cells (default 1) */
  double dt_cap;         /* upper bound on dt (default 10) */
  double dt_fixed;       /* > 0: use this dt and skip the CFL rule (default 0) */
  unsigned periodic_mask;/* bit d: direction d periodic (default 0) */
  int advect;            /* 1: convection on (default); 0: diffusion only */
  int precision;         /* 1 (default): FP32 except the fine-level pressure, kept in FP64 with an FP64
                            residual (iterative refinement), so tol holds whatever the pressure's size;
                            0: all FP32 (less traffic; the residual floor ~ 6e-8*|x|*2D may exceed tol) */
  int use_graph;         /* 1: wl_step runs as a CUDA graph with device-side V-cycle loops (default) */
  void* stream;          /* cudaStream_t for all work (default NULL) */
  void* workspace;       /* optional caller-owned device buffer of wl_workspace_bytes() */
  size_t workspace_bytes;
  int exit_bc;           /* 1: convective exit on the upper x face instead of the Dirichlet value U_x: the
                            normal velocity e there is carried out at U_x, de/dt = -U_x (e - u_x[n_0-1]),
                            by the same Heun stages, then shifted so that the flux out equals the flux in;
                            tangential components keep zero gradient.  Needs x non-periodic and
                            U_x > 0; not differentiated (wl_grad_* refuse it).  Default 0. */
  int coarse_precision;  /* storage of the multigrid levels between the fine and the coarsest one:
                            WL_COARSE_FP32 (default), WL_COARSE_BF16 or WL_COARSE_FP16.  A 16-bit
                            level keeps its face coefficients, right-hand side and iterate in 16 bits
                            and does every operation in FP32; its right-hand side is stored as the
                            mean, not the sum, of its fine cells' residuals (an exact power-of-two
                            scale), so its values stay within the fine residual's range (FP16 holds
                            magnitudes up to 65504).  The fine-level residual, the pressure and the
                            FP64 coarsest solve are unchanged, so the V-cycles converge to the same
                            tolerance (iterative refinement); only their count may change. */
  int metrics;           /* 1: every step also records the kinetic energy and max |div u| of the velocity at
                            its end and the pressure force (three reductions added to the step; see
                            wl_get_metrics); 0 (default): only the scalars every step records anyway */
} wl_opts;

#define WL_COARSE_FP32 0
#define WL_COARSE_BF16 1
#define WL_COARSE_FP16 2

/* Fill *o with the defaults listed above. */
void wl_default_opts(wl_opts* o);

/* Bytes of device workspace one sim of these dimensions needs (ndim 2 or 3;
 * dims[d] >= 2) with these options (NULL = defaults).  Returns 0 on bad arguments. */
size_t wl_workspace_bytes(const int* dims, int ndim, const wl_opts* opts);

/* Create a sim (measure step of the method: evaluates the body's signed distance
 * at every face to give the BDIM moments mu0 = K0(d/eps) and the Poisson
 * coefficients L = mu0, zero on non-periodic boundary faces (Section 2); builds the
 * multigrid hierarchy).  nu: kinematic viscosity in grid units; U: D boundary /
 * free-stream velocities; body may be NULL (no body); opts NULL = defaults.
 * The velocity starts uniform U, p = 0, dt from the CFL rule.  Synchronises. */
int wl_create(const int* dims, int ndim, double nu, const double* U, const wl_body* body,
              const wl_opts* opts, wl_handle* out);

/* Initial condition.  kind 0: uniform U; kind 1: Taylor-Green vortex of amplitude
 * `amp` (u = amp sin kx cos ky cos kz, v = -amp cos kx sin ky cos kz, w = 0,
 * k = 2 pi / n_0, each component sampled at its own faces); kind 2: the velocity
 * in src (D blocks, host or device per src_is_device).  Resets p = 0 and the
 * clock, and sets dt from the CFL rule.  Synchronises. */
int wl_set_ic(wl_handle h, int kind, double amp, const float* src, int src_is_device);

/* Advance nsteps full time steps (Heun + two projections + CFL; simstep! of
 * Section 3).  Asynchronous.  Convergence and non-finite checks are recorded on
 * the device; wl_status() reads them. */
int wl_step(wl_handle h, int nsteps);

/* Advance n resident simulations together: every sim hs[i] advances nsteps time steps
 * on its own stream, the sims' work overlaps on the device, and the whole batch is
 * ordered after the work already queued on `stream` and before the work queued on it
 * next (fork and join through events), so a caller can time one batch round with two
 * events on `stream`.  Give each sim its own stream (wl_opts.stream) for the overlap.
 * Asynchronous.  Returns the first error (the other sims are still launched); a
 * poisoned sim is skipped with WL_ENONFINITE.  Serving many simulations of different
 * sizes on one device; no counterpart in the paper. */
int wl_step_batch(const wl_handle* hs, int n, int nsteps, void* stream);

/* ---- Batched steps of many small simulations (serving; no counterpart in the paper,
 * whose GMG solve is linear in cells, Section 2, so many small grids are as cheap per cell
 * as one large one once they share launches).  wl_step_batch above launches one step graph
 * per simulation; for grids of a few thousand to ~10^5 cells each launch of such a graph is
 * mostly launch latency.  A batch advances all its small simulations together: every kernel
 * of the step is launched once for all of them, each block of a launch working on one
 * simulation through a per-simulation descriptor table kept on the device (grid, field
 * pointers, level sizes and every launch's arguments, built with the same argument
 * builders as that simulation's own step), and the two projections' V-cycle loops run in
 * conditional WHILE nodes until every simulation's projection has converged (a converged
 * one skips the rest of the loop).  Each simulation computes exactly what its own step
 * computes (the same kernels on the same inputs: the same bits alone and batched).
 *
 * A simulation is batched when it has at most max_cells cells and default-like options:
 * precision 1, FP32 levels, convection on, no convective exit, metrics off, a multigrid
 * hierarchy that ends in the small-level tail (at most 8 levels above it, at most 8 sweeps
 * per level) and, in 3-D, an even n_0; up to 64 per dimension (2-D and 3-D batch
 * separately).  Other simulations step with their own graphs on their own streams, as in
 * wl_step_batch.  The batch owns its streams, graphs and a device table of 64 slots per
 * dimension (about 1 MB); it rebuilds a graph when the set of its simulations changes. */
typedef struct wl_batch_s* wl_batch;
int wl_batch_create(long long max_cells, wl_batch* out);
/* Advance the n simulations hs one time step each (the batched ones in one graph per
 * dimension, the others on their own streams), ordered after the work already queued on
 * `stream` and before the work queued on it next, and on each simulation's own stream
 * after its earlier work and before its later work.  small_done (a cudaEvent_t, may be
 * NULL) is recorded on `stream` once the batched simulations' steps are done, before the
 * others are joined: it times the small simulations' step latency.  Asynchronous.
 * Returns the first error; a poisoned simulation is skipped with WL_ENONFINITE. */
int wl_batch_step(wl_batch b, const wl_handle* hs, int n, void* stream, void* small_done);
void wl_batch_destroy(wl_batch b);
const char* wl_batch_last_error(wl_batch b);
/* Milliseconds between two recorded CUDA events (cudaEvent_t; e.g. a round's start and the
 * small_done event wl_batch_step recorded), for callers whose event wrappers do not know
 * the library recorded one of them.  WL_ECUDA if either is not complete. */
int wl_event_elapsed(void* start, void* end, float* ms);

/* One Heun stage of convdiff! + BDIM! + BC! (Table 2) with the current dt, written
 * to the stage buffer (WL_FIELD_USTAGE): stage 1 maps u0 = WL_FIELD_U to
 * mu0 f + mu1.grad f with f = u0 + dt r(u0); stage 2 maps (u0 = WL_FIELD_U,
 * u' = WL_FIELD_UPRED) to (u' + mu0 f + mu1.grad f)/2 with f = u0 + dt r(u').
 * r is the finite-volume convection-diffusion residual, mu0/mu1 the BDIM moments
 * (Section 2).  Does not change the sim's state.  Asynchronous. */
int wl_stage(wl_handle h, int stage);

/* project! (Table 2) of the current velocity with weight w (1 after stage 1, 1/2
 * after stage 2): x0 = p w dt, multigrid V-cycles until ||div u - A x||_inf <= tol
 * or max_vcycles, u_c -= L_c (x[I] - x[I-e_c]) (Section 2), p = x/(w dt).
 * Writes the V-cycles used and the final residual (x units) to the host outputs
 * (either may be NULL); synchronises.  Returns WL_WNOTCONV if not converged. */
int wl_project(wl_handle h, double w, int* vcycles_out, double* resid_out);

/* One multigrid V(0,post) cycle on the fine system A p = z held in the sim
 * (fields WL_FIELD_P and WL_FIELD_Z, p units): restrict the residual by summing
 * 2^D children, coarse faces = half the sum of the 2^(D-1) fine faces, coarsest
 * level solved in FP64, piecewise-constant prolongation, red-black Gauss-Seidel
 * smoothing (Section 2: GMG, Weymouth 2022).  Writes ||z - A p||_inf after the
 * cycle to *resid_inf_out (may be NULL); synchronises. */
int wl_gmg_vcycle(wl_handle h, double* resid_inf_out);

/* Pressure force on the body, F_d = -sum_cells (p - pbar) n_d K_eps(d), with the
 * cosine kernel K_eps = (1 + cos(pi d/eps))/(2 eps) over |d| < eps and pbar the
 * mean pressure over cells with a nonzero Poisson row; accumulated in FP64.
 * F receives D values.  Synchronises.  The paper prints no force formula: this is the
 * library's reading (and the oracle's), the pressure part of the surface force in the
 * kernel-smoothed form of the immersed-boundary method Section 2 builds on (BDIM,
 * Weymouth & Yue 2011): the surface integral of -p n becomes a sum over the cells within
 * eps of the body, weighted by the kernel of the signed distance. */
int wl_forces(wl_handle h, double* F);

/* Viscous force on the body of the current velocity, F_i = sum_cells 2 nu S_ij n_j
 * K_eps(d) over |d| < eps (the viscous part of the surface integral, kernel-weighted like
 * wl_forces; the paper states no force, so this form is this library's reading), with
 * the strain rate S = (grad u + grad u^T)/2 at cell centres: du_c/dx_c from the cell's
 * two c-faces, du_c/dx_e (e != c) by the central difference of the cell-centred u_c;
 * neighbours outside the grid follow the boundary conditions.  Accumulated in FP64 in a
 * fixed order.  F receives D values (zeros without a body).  Synchronises.
 * WL_EINVAL for a null handle or F. */
int wl_viscous_force(wl_handle h, double* F);

/* Copy a field (WL_FIELD_*) to dst (host or device).  Synchronises when dst is on
 * the host. */
int wl_get_field(wl_handle h, int which, void* dst, int dst_is_device);
/* Overwrite a writable field from src (host or device).  Synchronises. */
int wl_set_field(wl_handle h, int which, const void* src, int src_is_device);

/* Current dt (the one the next step uses), simulated time and steps taken.
 * Synchronise. */
int wl_get_dt(wl_handle h, double* dt);
int wl_set_dt(wl_handle h, double dt);
int wl_get_time(wl_handle h, double* t, long long* steps);

/* ---- Checkpoint / resume.  Long runs (and the segment recomputation of a differentiated
 * rollout, Section 1) need to stop and continue a simulation exactly; the paper has no
 * counterpart.  A saved state holds everything a step reads from the steps before it: the
 * velocity (with the exit plane of a convective exit), the fine pressure (both words of
 * the double-float pair at precision 1, which is the next projection's initial guess), dt,
 * the clock, the step count and the V-cycle bookkeeping.  Layout: a header (magic
 * "WLSTATE1", format version, grid, periodic mask, precision, exit option, nu, U, sizes)
 * followed by those fields, in host or device memory as the caller chooses; the caller
 * owns the buffer.  Loading it into a sim created with the same dims, nu, U, body,
 * periodic mask, precision and exit option makes every later step bit-identical to the
 * run that saved it (the body and the multigrid options are not recorded: they must
 * match too).  Both calls synchronise the sim's stream. */

/* Bytes of a saved state of this sim (0 for a null handle). */
size_t wl_state_bytes(wl_handle h);
/* Write the state into dst (dst_bytes >= wl_state_bytes; host or device per
 * dst_is_device).  WL_EINVAL for a null pointer or a short buffer. */
int wl_save(wl_handle h, void* dst, size_t dst_bytes, int dst_is_device);
/* Restore a state written by wl_save.  WL_EINVAL (and nothing changed) when the header
 * is not a saved state, belongs to a different setup (grid, periodic mask, precision,
 * exit option, nu, U) or src_bytes is short.  Clears a poisoned flag. */
int wl_load(wl_handle h, const void* src, size_t src_bytes, int src_is_device);

/* ---- Per-step metrics.  Every step appends one record of WL_METRIC_FIELDS doubles to a
 * device ring of the last WL_METRIC_RING steps, written on the device at the step's end
 * (no host round trip, inside the step graph): the step number, the time after it and
 * the dt it used, the V-cycles and final residual (||div u - A x||_inf, x = p w dt units)
 * of both projections (Section 2: project!), the CFL out-flux maximum of its end velocity
 * (the dt rule's numerator, Table 2: CFL!); with wl_opts.metrics also the kinetic energy
 * 0.5 sum_c sum_I u_c[I]^2 / n_cells, max |div u| and the pressure force F_d of wl_forces
 * (D values), each summed in FP64 in a fixed order; fields not measured are NaN.  The
 * paper times only these routines; it has no counterpart for the record itself. */
#define WL_METRIC_RING 1024
#define WL_METRIC_FIELDS 13
#define WL_METRIC_STEP 0
#define WL_METRIC_TIME 1
#define WL_METRIC_DT 2
#define WL_METRIC_VCYCLES1 3
#define WL_METRIC_VCYCLES2 4
#define WL_METRIC_RESID1 5
#define WL_METRIC_RESID2 6
#define WL_METRIC_CFL 7
#define WL_METRIC_KE 8
#define WL_METRIC_MAXDIV 9
#define WL_METRIC_FORCE 10 /* 10, 11, 12: F_0, F_1, F_2 */

/* Copy the last min(max_records, steps recorded, WL_METRIC_RING) records, oldest first,
 * into out (host, max_records x WL_METRIC_FIELDS doubles); *n_out (may be NULL) receives
 * their number.  Synchronises.  WL_EINVAL for a null handle, a negative count or a null
 * out with max_records > 0. */
int wl_get_metrics(wl_handle h, double* out, int max_records, int* n_out);

/* Device-recorded status: V-cycles used by the two projections of the last step, the
 * total V-cycles since wl_create (cumulative: difference two calls to count an
 * interval), and the worst final residual (x units) of the steps since the last call.
 * Returns WL_ENONFINITE / WL_WNOTCONV if any step since the last call saw that.
 * Synchronises. */
int wl_status(wl_handle h, int* last_vcycles /*[2]*/, long long* total_vcycles, double* worst_resid);

/* kernel classes of wl_profile_step */
#define WL_KCLASS_STAGE 0       /* convdiff + BDIM stage (mu0 part) */
#define WL_KCLASS_BAND 1        /* BDIM mu1 term on the body band */
#define WL_KCLASS_RESID_FINE 2  /* divergence / residual + restriction on the fine level */
#define WL_KCLASS_RESTRICT 3    /* restriction between coarse levels */
#define WL_KCLASS_SWEEP_FINE 4  /* red-black Gauss-Seidel sweep on the fine level */
#define WL_KCLASS_SWEEP_COARSE 5 /* red-black Gauss-Seidel sweeps on coarse levels */
#define WL_KCLASS_COARSEST 6    /* coarsest-level solve */
#define WL_KCLASS_CORRECT 7     /* pressure-gradient correction (+ CFL maximum) */
#define WL_KCLASS_CONTROL 8     /* one-thread control kernels (V-cycle decision, step end) */
/* the fine level's split launches, each timed on its own stream while the other runs
 * beside it (also counted, as the pair's wall time, in SWEEP_FINE / RESID_FINE): */
#define WL_KCLASS_SWEEP_FINE_UNI 9    /* fine sweep, uniform tiles */
#define WL_KCLASS_SWEEP_FINE_BANDT 10 /* fine sweep, band tiles */
#define WL_KCLASS_RESID_FINE_UNI 11   /* fine residual / divergence, uniform tiles */
#define WL_KCLASS_RESID_FINE_BANDT 12 /* fine residual / divergence, band tiles */
#define WL_KCLASS_COUNT 13

/* Advance nsteps steps through the host-driven launch sequence (the same kernels
 * as wl_step) with a pair of CUDA events on the sim's stream around every launch,
 * and return per kernel class (WL_KCLASS_*) the summed device time in ms[] and the
 * launch count in launches[] (arrays of WL_KCLASS_COUNT).  For measurement;
 * synchronises. */
int wl_profile_step(wl_handle h, int nsteps, double* ms, long long* launches);

/* Kernel launches of the step graph: *per_step = kernel nodes outside the V-cycle loops
 * (stages, divergences, corrections, controls), *per_vcycle = kernel nodes of one V-cycle
 * (counted in the graph as captured, so side-stream launches are included).  A graph step
 * with n V-cycles launches per_step + n per_vcycle kernels.  WL_EINVAL without a step graph
 * (use_graph = 0, or before the first wl_step). */
int wl_graph_kernels(wl_handle h, int* per_step, int* per_vcycle);

/* Allocation-free pressure force, for callers that cannot allocate device memory
 * (for example while capturing a CUDA graph, where cudaMalloc is not allowed, or under
 * an allocator that owns the whole device).  The paper has no counterpart; this is
 * wl_forces' computation (F_d = -sum (p - pbar) n_d K_eps(d), FP64) on fields the caller
 * already holds:
 *   dims/ndim/periodic_mask: the grid; body, eps: the immersed body and BDIM half-width;
 *   p: device pointer, n cells of FP32 pressure (x fastest).  A sim at the default
 *      precision (1) keeps its fine pressure as a double-float pair ph + pl and wl_forces
 *      sums that pair; this entry point sees only the FP32 pressure it is given (for a
 *      sim's own state, WL_FIELD_P: the pair rounded to FP32), so its result differs from
 *      wl_forces by that rounding (the low word is left out).  At precision 0 both read
 *      the same FP32 field;
 *   L: device pointer, ndim blocks of n FP32 face coefficients (WL_FIELD_MU0 layout),
 *      used to find the cells with a nonzero Poisson row for pbar;
 *   F: device pointer receiving ndim doubles; stream: cudaStream_t (NULL = default).
 * Allocates nothing: its scratch is a fixed device array (256 KiB on every GPU that
 * loads the library, kept until exit) holding one partial-sum pair per 4096 cells, so
 * grids of more than WL_NOALLOC_MAX_CELLS cells return WL_EINVAL.  The first call on
 * each device looks the array's device address up (make that first call before any
 * stream capture).  All calls share the array: calls that overlap on the GPU race.
 * Asynchronous on `stream`. */
#define WL_NOALLOC_MAX_CELLS (16384LL * 4096LL)
int wl_forces_noalloc(const int* dims, int ndim, unsigned periodic_mask, const wl_body* body, double eps,
                      const float* p, const float* L, double* F, void* stream);

/* Bounds-checked build (libwl_debug.so: the same sources compiled with WL_DEBUG_BOUNDS; a
 * substitute for a memory checker, none being available to run on the GPU).  Its kernels
 * test the index of every global store of the step and of the computed global loads
 * against the array's size; an index outside sets a bit (WL_DBG_* in the kernels' sources:
 * 1 stage, 2 band term, 4 sweep, 8 residual, 16 correction, 32 restriction, 64 a TMA copy
 * whose inner coordinate is not 16-byte aligned, 128 coarse-correction load) and the
 * access is skipped, never a trap.  Its workspace also leaves a 256-byte canary (bytes
 * 0xA5) after every array.  This call reads and clears the kernels' flags (for every sim
 * of the process) and checks this sim's canaries (bit 31: one was overwritten) into
 * *flags; 0 means no bad index and intact canaries.  Synchronises.  In the release library
 * the checks compile away: *flags = 0 and the call returns WL_NODEBUG.  No counterpart in
 * the paper. */
int wl_debug_bounds(wl_handle h, unsigned* flags);

/* Self-test of the bounded device waits.  Every kernel that waits on the device (the
 * TMA-staged sweep and residual wait for their copies on mbarriers) gives up after a
 * wall-clock limit (2 s), records the timeout in the sim's status and returns, so that
 * a wait that cannot end becomes WL_ETIMEOUT instead of a hung GPU.  This call runs
 * the same wait on an mbarrier that nothing arrives at, with the limit `seconds`
 * (0 < seconds <= 10):
 *   returns WL_ETIMEOUT when the wait gave up (the expected result), WL_OK if it
 *   completed (it cannot), WL_EINVAL for a bad limit, WL_ECUDA/WL_ENOMEM on a CUDA
 *   failure; *elapsed_ms (may be NULL) receives the kernel's duration.
 * Synchronous; allocates 4 bytes of device memory for the flag.  No counterpart in the
 * paper. */
int wl_wait_probe(double seconds, double* elapsed_ms);

/* ---- Gradients of the pressure force with respect to the body (the differentiable
 * use of the solver, Section 1; the body enters through its signed-distance function,
 * Section 2).  theta = (R, c_0, .., c_{D-1}): the radius and centre of a circle/sphere
 * body (WL_BODY_SPHERE); theta = (R, r, c_x, c_y, c_z): the ring radius (y-z plane),
 * tube radius and centre of a torus (WL_BODY_TORUS, 3-D).  The derivative is taken with
 * dt held fixed (wl_opts.dt_fixed > 0 is required: the CFL rule is a maximum over the
 * field and is not differentiated),
 * each projection differentiated as the exact projection, and, where the convection
 * scheme is not differentiable (the limiter's switch points, the upwind switch), the
 * derivative of the branch the step takes.
 *
 * Memory: (nsteps/every + 1) checkpoints of the velocity and pressure, the recorded
 * intermediates of `every` steps (2D + 2 fields each) and 6D + 2 adjoint fields, in a
 * gradient workspace of wl_grad_workspace_bytes() bytes (256-byte aligned), supplied by
 * the caller or (workspace = NULL) allocated by the library and freed by the next
 * wl_grad_forward or wl_destroy.  Long horizons fit in memory by recomputing each
 * segment of `every` steps from its checkpoint during the backward pass. */

/* Bytes of the gradient workspace for nsteps steps with a checkpoint every `every`
 * steps; 0 on bad arguments. */
size_t wl_grad_workspace_bytes(wl_handle h, int nsteps, int every);

/* Advance nsteps time steps from the current state (the step graph of wl_step, or its
 * host-driven sequence with wl_opts.use_graph = 0: the same bits), record the pressure
 * force after each step into F (host, nsteps*D doubles, F_d = -sum (p - pbar) n_d
 * K_eps(d) as wl_forces) and keep the checkpoints for wl_grad_backward.  Returns
 * WL_EINVAL unless the body is a circle/sphere or torus and dt is fixed; WL_WNOTCONV /
 * WL_ENONFINITE as wl_step; WL_ENOMEM if the supplied workspace is too small or
 * unaligned.  Synchronises once, at the end. */
int wl_grad_forward(wl_handle h, int nsteps, int every, void* workspace, size_t workspace_bytes, double* F);

/* Gradient of J = sum_n gF[n] . F_n (gF: host, nsteps*D doubles, the cotangents of the
 * forces wl_grad_forward recorded) with respect to theta into theta_bar (host; D + 1
 * doubles dJ/dR, dJ/dc_0, .. for a circle/sphere, 5 doubles dJ/d(R, r, c_x, c_y, c_z)
 * for a torus).  Recomputes every segment from its checkpoint and runs the adjoint of
 * each step backwards (adjoint Poisson solves by the same multigrid to 1e-7 relative,
 * their V-cycles in a graph WHILE node the device ends); the sim's state is the one
 * after the forward rollout again on return.  Deterministic: the same bits on every run
 * (the transposed scatters are gathers, the reductions run in a fixed order).  Returns
 * WL_WNOTCONV (theta_bar still written) if an adjoint solve hit max_vcycles,
 * WL_ENONFINITE (the sim poisoned) on a non-finite adjoint residual.  Synchronises once,
 * at the end. */
int wl_grad_backward(wl_handle h, const double* gF, double* theta_bar);

/* Levels of the multigrid hierarchy and the dims of level l (dims[3]). */
int wl_levels(wl_handle h, int* nlevels);
int wl_level_dims(wl_handle h, int l, int* dims);

/* Whether level l's staged (TMA) sweeps and residual split their tiles: tiles away from
 * the body form their face coefficients (the level's free-stream value, 0 on walls)
 * instead of loading them, the rest (the body's band) load them.  *split (may be NULL)
 * receives 1 or 0, *band_fraction (may be NULL) the fraction of the level's tiles that
 * load their coefficients (1 without a split).  For measurement: the bytes a sweep moves
 * depend on it.  No counterpart in the paper. */
int wl_level_split(wl_handle h, int l, int* split, double* band_fraction);

/* Which kernel paths the sim's step takes, as bits into *paths: WL_PATH_RESID_STAGED the
 * TMA-staged fine residual / divergence (else the index-table kernel),
 * WL_PATH_CLUSTER_TAIL the coarse levels from some level down in one thread-block
 * cluster, WL_PATH_BLOCK_TAIL the smallest levels in one block (else level by level),
 * WL_PATH_TALL_TILES the staged sweep on some level in tiles of 64 x 16 cells (else
 * 64 x 8).  The paths give the same bits; for measurement and tests.  No counterpart in
 * the paper. */
#define WL_PATH_RESID_STAGED 1
#define WL_PATH_CLUSTER_TAIL 2
#define WL_PATH_BLOCK_TAIL 4
#define WL_PATH_TALL_TILES 8
int wl_kernel_paths(wl_handle h, unsigned* paths);

void wl_destroy(wl_handle h);
const char* wl_last_error(wl_handle h);

#ifdef __cplusplus
}
#endif

#endif /* WL_H */
