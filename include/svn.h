/*
 * svn.h -- C ABI of the GB300 stress-velocity Newton (svN) solver for the
 * implicitly discretised viscous-plastic sea-ice momentum equation
 * (Shih, Mehlmann, Losch, Stadler: "Robust and efficient primal-dual Newton-
 * Krylov solvers for viscous-plastic sea-ice models", arXiv:2204.10822).
 *
 * One implicit Euler step of the momentum equation (Section 3, Eqs. "Av=F",
 * "A", "F") is the minimiser of the convex energy Phi (Eq. "energy").  svn_step
 * computes it with the paper's stress-velocity Newton method (Section 4.2):
 * the dual variable pi (Eq. "pi") lives at the quadrature points and is
 * eliminated from each linearisation (Eqs. "tautilde", "linearSVNewton"),
 * the fourth-order tensor is symmetrised and scaled (Eq. "modification"),
 * each linear system is solved by FGMRES with a multigrid preconditioner
 * (Section 5.4), and steps are damped by backtracking on Phi (Section 5.1).
 *
 * Discretisation.  Omega = (0, L)^2 split into N x N square cells, dx = L/N;
 * Q1 velocity at the (N+1)^2 nodes with v = 0 on the boundary; ice thickness
 * H (here "h") and concentration A constant per cell; 2 x 2 Gauss quadrature.
 *
 * Array layouts (all FP64, all contiguous, caller-owned):
 *   cell field   : N*N doubles, index j*N + i            (cell (i, j), j = y)
 *   node vector  : 2*(N+1)^2 doubles, index 2*(j*(N+1) + i) + k, k = 0 (x), 1 (y)
 *                  (node (i, j) at (i dx, j dx)); boundary entries are
 *                  ignored on input and written as 0 on output.
 *   dual state pi: 12*N*N doubles, index ((j*N + i)*4 + q)*3 + c, with
 *                  quadrature point q = 2*qb + qa at local coordinates
 *                  (g[qa], g[qb]), g = 1/2 -+ 1/(2 sqrt 3), and symmetric
 *                  tensor component c = 0 (xx), 1 (yy), 2 (xy).
 * Pointers are DEVICE pointers unless the function name ends in _host.  The
 * library copies what it needs; it never keeps or frees a caller pointer.
 * Every call is stream-ordered on the handle's stream; functions that return
 * host-visible numbers synchronise that stream before returning.
 *
 * Errors.  Every function returns SVN_OK (0) or a negative SVN_ERR_* code and
 * records a message readable with svn_last_error(h).  After SVN_ERR_CUDA the
 * handle should be destroyed.  No function aborts the process.
 */
#ifndef SVN_H
#define SVN_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SVN_MAX_NEWTON 200

enum svn_status {
  SVN_OK = 0,
  SVN_ERR_ARG = -1,            /* invalid argument (sizes, NULL, constants) */
  SVN_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  SVN_ERR_OOM = -3,            /* device allocation failed */
  SVN_ERR_NONFINITE = -4,      /* NaN/Inf in inputs or in the residual norm */
  SVN_ERR_NO_CONVERGENCE = -5, /* max_newton iterations without reaching tol */
  SVN_ERR_LINESEARCH = -6,     /* max_halvings halvings without decrease of Phi */
  SVN_ERR_KRYLOV = -7,         /* FGMRES breakdown or max_krylov reached */
  SVN_ERR_TIMEOUT = -8,        /* a bounded device-side wait gave up */
  SVN_ERR_STATE = -9           /* call order violated (e.g. step before forcing) */
};

enum svn_precision {
  SVN_FP64 = 0,   /* every kernel in FP64 (the plain path) */
  SVN_MIXED = 1   /* FP64 residual, energy, dual update, outer FGMRES and its
                     operator; FP32 V-cycle on FP32-stored (vcycle_fp32 = 1,
                     default) or BF16-stored stencils */
};

typedef struct svn_grid {
  int N;          /* cells per side: even, 8 <= N <= 16384 */
  double L;       /* side length [m] */
} svn_grid;

typedef struct svn_params {
  /* physics (Table "tab:params"; P* in N/m^2, f_c explicit as in Section 3) */
  double rho_ice, rho_a, rho_o, Ca, Co, f_c, Pstar, C, e, delta_min;
  /* Newton (Section 5.1) */
  int max_newton;           /* <= SVN_MAX_NEWTON */
  int max_halvings;         /* backtracking halvings before SVN_ERR_LINESEARCH */
  double ls_floor;          /* rounding floor of the Phi test, relative to sum |terms| */
  /* Krylov + multigrid (Section 5.4) */
  double krylov_rtol;       /* FGMRES stop: ||r|| <= krylov_rtol ||R(v_l)|| */
  int restart;              /* FGMRES restart length */
  int max_krylov;           /* FGMRES iteration cap per Newton step */
  int precision;            /* enum svn_precision */
  int cheb_degree;          /* Chebyshev-Jacobi smoothing steps per side (>= 1) */
  double cheb_lo;           /* lower end of the Chebyshev interval, fraction of lmax */
  int coarse_N;             /* coarsest multigrid level has coarse_N cells per side */
  int eisenstat_walker;     /* 1: adapt krylov_rtol per Newton step (timed runs) */
  int learned;              /* 1: try the learned initial guess (svn_attach_net) */
  int use_graphs;           /* 1: run each V-cycle as one captured CUDA graph */
  int reorth_always;        /* 1: always two Gram-Schmidt passes; 0: second pass only
                               when the first cancels more than half of |w|^2 */
  double ew_eta_max;        /* upper bound of the Eisenstat-Walker forcing term */
  int lmax_iters;           /* power-method steps for lambda_max(D^-1 A) per level
                               (0: Gershgorin bound) */
  double lmax_safety;       /* the estimate is multiplied by this factor */
  int learned_rule;         /* acceptance of the learned guess v_p: 0 (default) keep it if
                               ||R(v_p)|| < ||R(v_old)||; 1 if Phi(v_p) < Phi(v_old);
                               2 always; 3 blend: start from v_old + alpha (v_p - v_old)
                               with the alpha in {1, 1/2, ..., 1/64} of lowest Phi, if
                               that is below Phi(v_old) (Phi is convex, so the blend is
                               never worse than v_old in energy); 4 always, with the dual
                               state pi_0 = tau(v_old)/Delta(v_old) of the plain start */
  int method;               /* 0 (default): stress-velocity Newton (Section 4.2);
                               1: standard Newton (Section 4.1, Eq. "standardNewton"),
                               i.e. the same operator with pi = tau(v)/Delta(v) at
                               every iteration and no dual update */
  int mg_rebuild;           /* rebuild the V-cycle hierarchy (Galerkin levels, smoother
                               data) every mg_rebuild Newton iterations (1 = always);
                               the FP64 outer operator is rebuilt every iteration */
  int cheb_fuse;            /* two Chebyshev steps per pass, kernel per level: 1 (default)
                               row-streaming warps on FP32 levels with N >= 1024 and a
                               shared-memory tile with a one-node ring elsewhere; 2: the
                               shared-memory tile on every level; 3: row-streaming warps
                               on every FP32 level; 4: TMA-staged CTA tiles on FP32-stencil
                               levels with N >= 1024, tile elsewhere; 5: TMA-staged on
                               every FP32-stencil level; 0: one step per pass */
  int fused_trial;          /* 1 (default): evaluate Phi, R and pi at the unit step in one
                               fused pass; 0: separate energy / residual / dual passes */
  int vcycle_fp32;          /* mixed precision: 1 (default) stores the V-cycle stencils
                               in FP32, 0 in BF16 (BF16 rounding of the entries
                               perturbs the near-rigid modes; robust only on
                               coarse grids) */
  int cheb_degree_coarse;   /* Chebyshev degree on the coarser levels (0, default:
                               cheb_degree on every level) */
  double retry_alpha;       /* inexact-Newton safeguard (no counterpart in the paper,
                               which solves each linearisation directly): when the
                               line search fails or accepts a step length below
                               retry_alpha while the Krylov tolerance of the step is
                               above krylov_rtol, the Newton direction is recomputed
                               with a 100x tighter tolerance (at most 3 times per
                               Newton iteration).  Default 1/64; 0 disables it */
  int wait_polls;           /* bound of every mbarrier wait of the TMA-staged sweep, in
                               non-blocking polls (0: default 2^22).  A wait that runs
                               out abandons its block's work; the step then fails with
                               SVN_ERR_TIMEOUT (checked after each linearisation and
                               each Krylov solve; the counter is device-wide) */
  int q2_smooth_degree;     /* Q2 elements only: Chebyshev-block-Jacobi steps on the Q2
                               operator before and after the Q1 V-cycle of the
                               preconditioner (p-multigrid; default 3, 0: the Q1 V-cycle
                               alone) */
  double ew_tail;           /* eisenstat_walker only: the forcing term of a Newton step
                               is raised to min(ew_eta_max, ew_tail * tol * ||R_0|| /
                               ||R_k||), so that a step whose residual is already near
                               the stopping threshold is not solved far past it
                               (Kelley, Iterative Methods for Linear and Nonlinear
                               Equations, 1995, Sect. 6.3; no counterpart in the paper,
                               which solves each linearisation directly).  Default
                               0.5; 0 disables it; must be in [0, 1] */
} svn_params;

typedef struct svn_stats {
  int status;               /* same as the return code of svn_step */
  int newton_iters;
  int krylov_iters_total;
  int halvings_total;
  int learned_used;         /* the learned guess was tried */
  int learned_fallback;     /* ... and rejected (larger residual than v_old) */
  double res0;              /* ||R(v_old)||, the denominator of rel-res */
  double res_final;
  double rel_res_final;
  double seconds;           /* wall time of the step on the host */
  int krylov_per_newton[SVN_MAX_NEWTON];
  double res_hist[SVN_MAX_NEWTON + 1];
  double alpha_hist[SVN_MAX_NEWTON];
  int direction_retries;    /* Newton directions recomputed by the retry_alpha safeguard */
  double learned_alpha;     /* weight of the learned guess in the start (0: not used) */
} svn_stats;

typedef struct svn_handle svn_handle;

/* Fill *p with the paper's constants (P* = 27.5 kN/m^2, e = 2,
 * Delta_min = 2e-9 1/s, f_c = 1.46e-4 1/s) and default solver settings. */
int svn_default_params(svn_params* p);

/* Create a solver for one grid on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  Allocates all device
 * workspace (the multigrid hierarchy, FGMRES basis, quadrature state).  On
 * failure *out is still set (unless out is NULL or the handle itself could
 * not be allocated, SVN_ERR_OOM) so that svn_last_error can be read; it owns
 * no device memory and must be released with svn_destroy. */
int svn_create(const svn_grid* g, const svn_params* p, void* cuda_stream, svn_handle** out);
int svn_destroy(svn_handle* h);
const char* svn_last_error(const svn_handle* h);

/* Inputs of one implicit step (Sections 2 and 3): cell thickness h [m] and
 * concentration A at t_{n+1}, node wind v_a(t_{n+1}) and ocean v_o [m/s], and
 * the previous velocity v^n.  Checks finiteness, h > 0 and 0 <= A <= 1
 * (SVN_ERR_NONFINITE / SVN_ERR_ARG).  The step starts from v^n and
 * pi = tau(v^n)/Delta(v^n). */
int svn_set_forcing(svn_handle* h, const double* hcell, const double* A,
                    const double* wind, const double* ocean, const double* v_old);
int svn_set_forcing_host(svn_handle* h, const double* hcell, const double* A,
                         const double* wind, const double* ocean, const double* v_old);

/* One implicit step of length dt [s]: damped svN iterations until
 * ||R(v_l)|| <= tol ||R(v^n)|| (Euclidean norm of the assembled residual over
 * the free dofs).  out_v receives v^{n+1} (or the last iterate on error);
 * stats (may be NULL) is filled in every case. */
int svn_step(svn_handle* h, double dt, double tol, double* out_v, svn_stats* stats);
int svn_step_host(svn_handle* h, double dt, double tol, double* out_v, svn_stats* stats);

/* ---- Time stepping of the coupled system (Section 3) ----
 *
 * svn_transport: the explicit step for concentration and thickness
 * (Eqs. "model:A", "model:H"; Section 3; A and H cell-wise constant as in
 * Section 5.1).  Moves the handle's h and A (those of the last
 * svn_set_forcing or svn_advance) over dt [s] with its v^n by first-order
 * upwind finite volumes: face normal velocity = mean of the two end nodes,
 * node velocities on the boundary taken as 0 (v = 0 on the boundary, so no
 * flux crosses it), explicit Euler split into max(1, ceil(c)) equal
 * sub-steps where c = dt/dx * max over cells of the summed outflow normal
 * velocities, and A capped at 1 afterwards.  *substeps (may be NULL)
 * receives the number of sub-steps.  Errors: SVN_ERR_STATE before
 * svn_set_forcing, SVN_ERR_ARG for dt <= 0 or more than 10000 sub-steps,
 * SVN_ERR_NONFINITE for a non-finite velocity; SVN_ERR_ARG also if the
 * result has h <= 0 (it cannot while every input h > 0).
 *
 * svn_get_ice: copies the handle's current h and A (device, N*N each, cell
 * (i, j) at j*N + i) to caller-owned device buffers.
 *
 * svn_advance: one full time step t_n -> t_{n+1}: svn_transport with v^n,
 * then wind and ocean replaced by the given device node fields at t_{n+1}
 * (NULL keeps the current field), then the implicit momentum step from v^n
 * as in svn_step.  On success the solution becomes v^n of the next call
 * and is also written to out_v (may be NULL).  On a failed momentum step
 * v^n is left unchanged while h and A stay transported; stats and *substeps
 * as above. */
int svn_transport(svn_handle* h, double dt, int* substeps);
int svn_get_ice(svn_handle* h, double* hcell, double* A);
int svn_advance(svn_handle* h, double dt, double tol, const double* wind, const double* ocean, double* out_v,
                svn_stats* stats, int* substeps);

/* Current iterate v and dual state pi (checkpoint / warm restart). */
int svn_get_state(svn_handle* h, double* v, double* pi);
int svn_set_state(svn_handle* h, const double* v, const double* pi);

/* ---- Hot-path components, one call per step of the method.  They use the
 * forcing of the last svn_set_forcing and the given dt; all vectors are
 * device node vectors of the handle's grid unless stated. ---- */

/* Nonlinear residual R(v) = A(v, .) - F(.) (Eqs. "Av=F", "A", "F" with the
 * stress in the tau-form of Eq. "sigma"), boundary rows 0, and its Euclidean
 * norm (host double). */
int svn_residual(svn_handle* h, double dt, const double* v, double* R, double* norm);

/* Energy Phi(v + alpha_i dv) (Eq. "energy") for k <= 8 step lengths
 * (host arrays alphas[k] -> phi[k]); *scale (may be NULL) receives the sum of
 * |quadrature contributions| at alpha_0, the rounding scale of Phi. */
int svn_energy(svn_handle* h, double dt, const double* v, const double* dv,
               const double* alphas, int k, double* phi, double* scale);

/* Build the svN linearisation at (v, pi): quadrature coefficients of
 * Eq. "linearSVNewton" with Eq. "modification" and the ocean-drag derivative
 * (Eq. "standardNewton2"), the level-0 stencil and the multigrid hierarchy.
 * pi is a device dual state (layout above). */
int svn_linearize(svn_handle* h, double dt, const double* v, const double* pi);

/* y = K_level x with the operator of the last svn_linearize; level 0 is the
 * FP64 svN operator, level l >= 1 the Galerkin coarse operator on the grid
 * with N / 2^l cells (node vectors of that grid). */
int svn_apply(svn_handle* h, int level, const double* x, double* y);

/* z = M^{-1} r: one multigrid V-cycle of the last svn_linearize. */
int svn_precondition(svn_handle* h, const double* r, double* z);

/* Solve K x = b by preconditioned FGMRES to ||b - K x|| <= rtol ||b||
 * (x starts at 0); *iters receives the iteration count. */
int svn_krylov_solve(svn_handle* h, const double* b, double* x, double rtol, int* iters);

/* Dual update pi <- pi + alpha pi~(v, dv, pi) (Eq. "tautilde" with the
 * modification of Eq. "modification"), in place on the device array pi. */
int svn_dual_update(svn_handle* h, double dt, const double* v, const double* dv,
                    double alpha, double* pi);

/* ---- Allocation-free residual.  The paper has no counterpart: this entry
 * point exists for callers that cannot call cudaMalloc -- for example a host
 * model that hands the whole device to its own memory pool at start-up, or a
 * runtime that keeps its device footprint fixed after initialisation.  It
 * computes the same R(v) and ||R|| as svn_residual, without a handle:
 *   grid, prm     : grid (even N, 8 <= N <= SVN_NOALLOC_MAX_N) and constants;
 *   dt            : time step [s], > 0;
 *   hcell .. v_old: device inputs in the layouts above (as svn_set_forcing);
 *   v             : device node vector at which R is evaluated;
 *   R             : device node vector receiving R(v) (boundary entries 0);
 *   norm          : host double receiving ||R|| (may be NULL: then the call
 *                   does not synchronise the stream);
 *   cuda_stream   : cudaStream_t the work is ordered on (NULL = default).
 * It allocates nothing: every intermediate array lives in one file-scope
 * device array of about 16 MB (30 planes of the N = SVN_NOALLOC_MAX_N
 * layout), which every GPU that loads the library holds until the process
 * exits.  Every call looks up that array's address in the current device's
 * context (so a call after a device reset still finds it); make a first call
 * before any stream capture, since the module is loaded on first use.  All
 * calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU (several streams or host threads) race.
 * Returns SVN_ERR_ARG for N above the maximum, odd N or bad constants,
 * SVN_ERR_NONFINITE for a non-finite norm, SVN_ERR_CUDA on a CUDA error;
 * there is no handle, so no message is recorded. ---- */
#define SVN_NOALLOC_MAX_N 256
int svn_residual_noalloc(const svn_grid* grid, const svn_params* prm, double dt,
                         const double* hcell, const double* A, const double* wind,
                         const double* ocean, const double* v_old, const double* v,
                         double* R, double* norm, void* cuda_stream);

/* ---- Q2 velocity elements (Section 5.1: the implementation "also allows
 * higher-order discretizations"; Section 5.3 shows Problem II with quadratic
 * velocity elements).  The same implicit step, energy, svN linearisation and
 * dual update as above on biquadratic elements: N x N cells (N even,
 * 4 <= N <= 8192), each with the 9 Lagrange nodes of the tensor-product
 * quadratic basis, so the velocity lives on the (2N+1) x (2N+1) node grid of
 * spacing dx/2 (node (I, J) at (I dx/2, J dx/2), v = 0 on the boundary); H and
 * A constant per cell; 3 x 3 Gauss points per cell (R is the exact gradient
 * of the discrete energy); pi at the 9 points.
 * Layouts (device, FP64, caller-owned):
 *   cell field   : N*N, index j*N + i (as above)
 *   node vector  : 2*(2N+1)^2, index 2*(J*(2N+1) + I) + k
 *   dual state pi: 27*N*N, index ((j*N + i)*9 + q)*3 + c with point
 *                  q = 3*qb + qa at local coordinates (x[qa], x[qb]),
 *                  x = 1/2 - sqrt(3/5)/2, 1/2, 1/2 + sqrt(3/5)/2, c as above.
 * Linear systems: FGMRES on the FP64 Q2 Jacobian, preconditioned by the
 * V-cycle of the Q1 operator on the same nodes (the 2N grid, linearised at
 * the same node velocities), in the precision of params->precision.
 * svn_q2_create allocates all workspace (including a Q1 handle on the 2N
 * grid); on failure *out is still set (unless out is NULL) for
 * svn_q2_last_error and must be released with svn_q2_destroy.
 * svn_q2_set_forcing checks its inputs as svn_set_forcing does.
 * svn_q2_step: one implicit step from v^n (damped svN, Section 4.2, with the
 * backtracking of Section 5.1 and the retry_alpha safeguard); out_v and
 * stats as for svn_step.  svn_q2_residual / _energy / _linearize / _apply /
 * _dual_update: the hot-path rows on Q2 elements (svn_q2_apply multiplies by
 * the operator of the last svn_q2_linearize).  svn_q2_get_state: the last
 * iterate and its pi. ---- */
typedef struct svn_q2 svn_q2;
int svn_q2_create(const svn_grid* g, const svn_params* p, void* cuda_stream, svn_q2** out);
int svn_q2_destroy(svn_q2* h);
const char* svn_q2_last_error(const svn_q2* h);
int svn_q2_set_forcing(svn_q2* h, const double* hcell, const double* A, const double* wind,
                       const double* ocean, const double* v_old);
int svn_q2_step(svn_q2* h, double dt, double tol, double* out_v, svn_stats* stats);
int svn_q2_residual(svn_q2* h, double dt, const double* v, double* R, double* norm);
int svn_q2_energy(svn_q2* h, double dt, const double* v, const double* dv, const double* alphas, int k,
                  double* phi, double* scale);
int svn_q2_linearize(svn_q2* h, double dt, const double* v, const double* pi);
int svn_q2_apply(svn_q2* h, const double* x, double* y);
int svn_q2_dual_update(svn_q2* h, double dt, const double* v, const double* dv, double alpha, double* pi);
int svn_q2_get_state(svn_q2* h, double* v, double* pi);

/* ---- Ensembles (no counterpart in the paper: the paper solves one
 * instance at a time).  n independent instances of any grid sizes; each
 * has its own handle and private non-blocking stream, and svn_batch_step
 * advances all of them by one implicit step concurrently from host_threads
 * host threads (<= 0: 8), so that small grids share the GPU.  out_v[i] are
 * device node vectors of instance i's grid; stats (may be NULL) is an array
 * of n.  The first failing instance's code is returned, and
 * svn_batch_last_error names every failing instance (up to 8).  On a failed
 * svn_batch_create *out is still set (unless out is NULL or the batch could
 * not be allocated): svn_batch_last_error names the failing instance, and
 * svn_batch_destroy releases the instances created so far. ---- */
typedef struct svn_batch svn_batch;
int svn_batch_create(int n, const svn_grid* grids, const svn_params* p, int host_threads, svn_batch** out);
int svn_batch_destroy(svn_batch* b);
const char* svn_batch_last_error(const svn_batch* b);
int svn_batch_size(const svn_batch* b);
/* Handle of instance i (owned by the batch): use it with svn_set_forcing etc. */
svn_handle* svn_batch_instance(svn_batch* b, int i);
int svn_batch_step(svn_batch* b, double dt, double tol, double* const* out_v, svn_stats* stats);

/* ---- Autotuner (no counterpart in the paper).  Runs probe_newton Newton
 * iterations of the current forcing, then times one FGMRES solve of that
 * linearisation for every (degree, lo) pair of Chebyshev smoother settings
 * and keeps the fastest in the handle's parameters (read them back with
 * svn_get_params).  *best_ms (may be NULL) receives the winning time.  On an
 * error the handle keeps the smoother settings it had before the call. ---- */
int svn_autotune(svn_handle* h, double dt, int probe_newton, const int* degrees, int nd,
                 const double* los, int nl, double* best_ms);
/* The same search over the sweep kernels too: every cheb_fuse value in
 * cheb_fuses[nf] (each in [0, 5]: the shared-memory tile, row-streaming and
 * TMA-staged two-step kernels and their level thresholds) times every
 * (degree, lo) pair; the fastest triple is kept.  Callers that tune many
 * handles of one grid size cache the result (the Python binding keeps a JSON
 * file keyed by grid size and precision). */
int svn_autotune_kernels(svn_handle* h, double dt, int probe_newton, const int* degrees, int nd,
                         const double* los, int nl, const int* cheb_fuses, int nf, double* best_ms);
/* Set the smoother settings of a handle (as svn_params.cheb_fuse,
 * cheb_degree, cheb_lo; checked like svn_create), e.g. from a cached
 * autotuner result; they take effect at the next linearisation. */
int svn_set_smoother(svn_handle* h, int cheb_fuse, int cheb_degree, double cheb_lo);
int svn_get_params(const svn_handle* h, svn_params* p);

/* ---- Learned initial guess (no counterpart in the paper).  A U-Net on a
 * G x G cell grid (G a multiple of 64): four levels with 32/64/128/256
 * channels, two 3x3 convolutions + ReLU per level, 2x2 average pooling,
 * nearest upsampling with skip concatenation, and a 3x3 head; BF16 weights
 * and activations with FP32 accumulation (tensor-core implicit GEMMs for the
 * forward and backward-data convolutions), Adam on FP32 master weights.
 * Inputs (8 channels, block averages over N/G x N/G cells of an N-cell
 * problem): h/2, (A - 0.9)/0.1, wind/15, ocean/0.1, v_old/0.2 (m/s); output:
 * cell-centred velocity / 0.2, prolonged bilinearly to the nodes.
 * Parameters are one FP32 vector: for each of the 15 convolutions in order its
 * weights [Cout][3*ky+kx][Cin], then all biases in the same order.  All
 * pointers of svn_net_set_sample are device pointers in the layouts above;
 * v_target (may be NULL) needs N == G.  svn_net_train_step runs forward,
 * loss 0.5 mean((out - target)^2), backward and (if apply_update) one Adam
 * step on the first nb batch slots; *loss receives the loss (host).
 * svn_attach_net makes svn_step try the network's prediction as v_0 when
 * params.learned (or svn_set_learned) is on; it is used only if its residual
 * is below ||R(v_old)||, else v_old (stats.learned_used / learned_fallback).
 * The handle borrows the network (NULL detaches it): destroy the network only
 * after detaching it or destroying every handle it is attached to.  The
 * prediction runs on the handle's stream; the network must not be trained
 * concurrently on another stream. */
typedef struct svn_net svn_net;
int svn_net_create(int G, int batch, void* cuda_stream, svn_net** out);
int svn_net_destroy(svn_net* net);
const char* svn_net_last_error(const svn_net* net);
long long svn_net_num_params(const svn_net* net);
int svn_net_set_params(svn_net* net, const float* host_params, long long n);
int svn_net_get_params(svn_net* net, float* host_params, long long n);
int svn_net_get_grads(svn_net* net, float* host_grads, long long n);
int svn_net_set_sample(svn_net* net, int slot, int N, const double* hcell, const double* A,
                       const double* wind, const double* ocean, const double* v_old,
                       const double* v_target);
/* Forward on slots [0, nb); out_host (may be NULL) receives nb x G x G x 16
 * FP32 outputs (channels 0, 1 used). */
int svn_net_forward(svn_net* net, int nb, float* out_host);
int svn_net_train_step(svn_net* net, int nb, float lr, int apply_update, float* loss);
int svn_attach_net(svn_handle* h, svn_net* net);
int svn_set_learned(svn_handle* h, int on);

/* ---- Instrumentation (no counterpart in the paper): CUDA-event timing of
 * one kernel class on the handle's stream, for roofline reporting. ---- */
enum svn_kernel_class {
  SVN_K_APPLY = 0,     /* FP64 outer Jacobian apply (stencil form) */
  SVN_K_CHEB = 1,      /* finest-level Chebyshev-Jacobi sweeps (only the fused
                          two-step launches when cheb_fuse is on) */
  SVN_K_MULTIDOT = 2,  /* FGMRES multi-dot (Arnoldi projections) */
  SVN_K_UPDATE = 3,    /* FGMRES update + norm */
  SVN_K_ELEMENT = 4,   /* element matrices of the linearisation */
  SVN_K_RESIDUAL = 5,  /* nonlinear residual (cells + nodes) */
  SVN_K_ENERGY = 6,    /* energy evaluation */
  SVN_K_DUAL = 7,      /* dual update */
  SVN_K_RAP = 8,       /* Galerkin coarse operators */
  SVN_K_VCYCLE = 9,    /* one whole V-cycle (all of its kernels) */
  SVN_K_COUNT = 10
};
/* enable = 1 resets the totals and starts recording; 0 stops. */
int svn_profile(svn_handle* h, int enable);
/* Total milliseconds and number of recorded launches of one class since the
 * last svn_profile(h, 1); synchronises the handle's stream. */
int svn_profile_read(svn_handle* h, int kclass, double* ms_total, long long* launches);
/* Kernel launches issued by this library in this process so far. */
unsigned long long svn_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* SVN_H */
