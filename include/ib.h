/*
 * ib.h -- C ABI of the GB300 implicit immersed-boundary multigrid library.
 *
 * Method: Guy, Philip & Griffith, "Geometric multigrid for an implicit-time
 * immersed boundary method".  One backward-Euler IB step with lagged
 * spreading/interpolation (sec. 2.3.2, Eqs. 17-20) is reduced to a Stokes-type
 * saddle-point system on a 2-D staggered (MAC) grid by eliminating the
 * Lagrangian unknowns (Eqs. 21-22; the block system, Eq. 23, sec. 3):
 *
 *     [ mu*Lap_h - (rho/dt) I + dt * S J S^*   -grad_h ] [u]   [ -(rho/dt) u^n - S F(X^n) ]
 *     [ div_h                                   0      ] [p] = [ 0                        ]
 *
 * where S is spreading with a 4-point regularised delta (sec. 2.2), S^* its
 * adjoint (interpolation), F the spring force and J = dF/dX its Jacobian at
 * X^n.  With rho = 0 and zero rest length this is exactly the paper's system
 * with alpha S A_f S^* (alpha = gamma dt).  The system is solved by flexible
 * GMRES (sec. 3.3) right-preconditioned by one geometric V-cycle (Algorithm 1)
 * with the box / big-box smoother (secs. 5-6), re-discretised Stokes and
 * Galerkin-coarsened elasticity on coarse levels (sec. 3.2), staggered
 * transfers (sec. 3.1) and an exact solve on the N_c = max(4, box) grid
 * (sec. 6.1).  Then X^{n+1} = X^n + dt S^* u^{n+1} (Eq. 20).
 *
 * Conventions for every entry point:
 *  - Domain: periodic square of side L, N x N cells, h = L / N.
 *  - Grid vectors have layout [u | v | p], each an N x N block, row-major with
 *    x fastest (index j*N + i); u[j][i] sits at (i h, (j+1/2) h), v[j][i] at
 *    ((i+1/2) h, j h), p[j][i] at the cell centre.  Level l vectors use
 *    N_l = N / 2^l.
 *  - Lagrangian arrays X are [n_points][2] (x, y), float64.
 *  - "device" pointers are CUDA device memory on the current device; "host"
 *    pointers are ordinary host memory.  All memory passed in is owned by the
 *    caller and is only read/written for the duration of the call.
 *  - Work is issued on the CUDA stream given at set-up; calls return after
 *    their results are complete on that stream unless stated otherwise.
 *  - Every function returns an ib_status code; nothing throws across the ABI
 *    and nothing exits the process.  ib_last_error() gives a message for the
 *    last failing call on the calling thread.
 */
#ifndef IB_H_
#define IB_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IB_API __attribute__((visibility("default")))
#else
#define IB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  IB_OK = 0,
  IB_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter failed validation */
  IB_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
  IB_ERR_OOM = 3,           /* device allocation failed */
  IB_ERR_NOT_CONVERGED = 4, /* FGMRES hit max_iters above tol (results still written) */
  IB_ERR_BREAKDOWN = 5,     /* non-finite value in the Krylov recurrence */
  IB_ERR_SINGULAR = 6,      /* a zero pivot in a box or coarsest-level factorisation */
  IB_ERR_TIMEOUT = 7        /* a bounded device-side wait ran out */
} ib_status;

enum { IB_DELTA_PESKIN4 = 0, IB_DELTA_COS4 = 1 };
/* Precision of the V-cycle (FGMRES, the operator and the true residual are FP64
 * in every mode; not in the paper):
 *   IB_FP64            everything FP64.
 *   IB_FP32_PRECOND    V-cycle in FP32 (vectors, stencils, elasticity, free-box
 *                      solves); the solves of structure boxes (whose condition
 *                      number grows with the stiffness) in FP64, cast at the box.
 *   IB_MIXED_PRECOND   V-cycle in FP64 except the structure-free boxes, whose shared
 *                      inverse is applied in FP32 (the FP64 pipe is the GB300's
 *                      slowest unit and those box products are most of the
 *                      V-cycle's FLOPs). */
enum { IB_FP64 = 0, IB_FP32_PRECOND = 1, IB_MIXED_PRECOND = 2 };
enum { IB_JAC_CLAMPED = 0, IB_JAC_EXACT = 1 };

/* Boundary of the square (sec. 4):
 *   IB_WALLS_PERIODIC  the periodic unit square (the default);
 *   IB_WALLS_NOSLIP    the square with no-slip walls of the paper's tests (the lid-
 *                      driven cavity's operator): the normal velocity is zero on
 *                      each wall, and the tangential velocity of the first row of
 *                      faces sees the ghost value -u (the wall value, the mean of the
 *                      two, is zero).  In every [u | v | p] vector the faces u(0, j)
 *                      (x = 0; x = 1 has no face of its own) and v(i, 0) (y = 0) are
 *                      the walls: they are not unknowns, inputs must hold zero there,
 *                      ib_apply returns them unchanged, and right-hand sides are
 *                      zeroed there (a moving lid enters the right-hand side through
 *                      the ghost, 2 u_lid - u, as a known term the caller adds).
 *                      Coarse levels use the same ghost rule in the prolongation
 *                      (fine row next to a wall = half the coarse one).  Points must
 *                      stay at least 2h from every wall (checked at ib_setup; a
 *                      point that moves closer fails the next set-up), and the
 *                      structure's couplings must fit the assembled rows (springs
 *                      up to about 1.5 cells).  The strip form of the box kernel and
 *                      the learned stage are periodic only.  With rho = 0 only the
 *                      constant pressure is bordered out of the coarsest solve. */
enum { IB_WALLS_PERIODIC = 0, IB_WALLS_NOSLIP = 1 };

/* Time-stepping method (sec. 2.3):
 *   IB_IMPLICIT  backward Euler for the structure (sec. 2.3.2, Eqs. 17-22): the
 *                operator carries dt S J S^*, the system this library is about;
 *   IB_EXPLICIT  the explicit-time method (sec. 2.3.1): the operator is the
 *                Stokes system alone, the structure's force F(X^n) stays on the
 *                right-hand side, and X^{n+1} = X^n + dt S^* u^{n+1} as before.
 *                Stable only for gamma dt below alpha_exp (sec. 4.1); it is here to
 *                measure what the implicit method saves (sec. 7). */
enum { IB_IMPLICIT = 0, IB_EXPLICIT = 1 };

/* Problem parameters (sec. 2: grid, fluid, time step; secs. 5-6: smoother). */
typedef struct {
  int32_t N;          /* cells per side: power of two, N >= 2 * max(4, box) */
  double L;           /* domain side (> 0) */
  double rho;         /* density (>= 0); 0 gives the paper's steady Stokes system */
  double mu;          /* viscosity (> 0) */
  double dt;          /* backward-Euler step (> 0) */
  int32_t delta;      /* IB_DELTA_PESKIN4 or IB_DELTA_COS4 (sec. 2.2) */
  int32_t box;        /* box size b in {1, 2, 4, 8, 16} (sec. 6) */
  int32_t nu1, nu2;   /* pre/post smoothing sweeps, 0..8 (Algorithm 1) */
  int32_t precision;  /* IB_FP64, IB_FP32_PRECOND or IB_MIXED_PRECOND (see above) */
  int32_t jacobian;   /* IB_JAC_CLAMPED (default) or IB_JAC_EXACT spring Jacobian */
  double tol;         /* relative residual target ||b - A x|| / ||b|| (> 0) */
  int32_t max_iters;  /* FGMRES iteration cap, 1..512 (the paper stops at 100) */
  int32_t escalate;   /* IB_FP32_PRECOND only: 1 (default) = use the mixed-precision
                         V-cycle from the start when dt * max(kappa) / mu >= 3000
                         (environment variable IB_STIFF_SIGMA overrides the value), and
                         restart with it when the FP32-preconditioned FGMRES stagnates;
                         0 = FP32 throughout */
  int32_t restart;    /* FGMRES restart length m (Krylov vectors kept), 0 = max_iters;
                         workspace grows with m: (m + 1) FP64 + m preconditioner vectors */
  int32_t walls;      /* IB_WALLS_PERIODIC (default) or IB_WALLS_NOSLIP (see above) */
  double lid;         /* IB_WALLS_NOSLIP only: the top wall y = L moves with the tangential
                         velocity u(x, L) = lid * (1 - cos(2 pi x / L)) / 2, the lid of the
                         paper's cavity (sec. 4); it enters the right-hand side of ib_rhs and
                         ib_solve_step through the ghost 2 u_lid - u of the faces next to the
                         lid.  0 (default): all walls at rest. */
  int32_t time_method; /* IB_IMPLICIT (default) or IB_EXPLICIT (see above) */
} ib_params;

/* Statistics of one ib_solve_step call. */
typedef struct {
  int32_t iters;        /* FGMRES iterations (= V-cycles applied) */
  int32_t restarts;     /* restarts after a failed true-residual check */
  double rel_res_true;  /* ||b - A x|| / ||b|| recomputed in FP64 at the end */
  double rel_res_est;   /* FGMRES (Givens) estimate at the last iteration */
  double t_setup_ms;    /* hierarchy set-up time (CUDA events) */
  double t_solve_ms;    /* FGMRES time (CUDA events) */
  int32_t n_struct_boxes; /* structure boxes (with elasticity), all levels */
  int32_t status;       /* ib_status of the solve */
  int32_t escalated_at; /* iteration from which the FP64 V-cycle preconditioned (-1: never) */
  int32_t learned_used; /* iterations whose direction the learned stage improved (kept) */
} ib_stats;

typedef struct ib_problem ib_problem;  /* opaque; owned by the library */

/* Fill *p with the defaults: L=1, rho=1, mu=1, dt=1e-2, Peskin4, box 1, V(1,1),
 * FP64, clamped Jacobian, tol 1e-8, max_iters 100, escalate 1, restart 0 (no restart
 * before max_iters).  N is set to 64. */
IB_API void ib_default_params(ib_params* p);

/* Create a problem: validates the parameters, allocates all device workspace
 * (levels N, N/2, ..., N_c) and uploads the structure.
 *   X        host [n_points][2] initial point positions (any real values; periodic)
 *   springs  host [n_springs][2] point index pairs (i != j, 0 <= i, j < n_points)
 *   kappa    host [n_springs] stiffness (>= 0);  rest  host [n_springs] rest length (>= 0)
 *   stream   a cudaStream_t (NULL = legacy default stream) used by every later call
 * n_points may be 0 (no structure; then n_springs must be 0).  The spring
 * force law is F_i += kappa (1 - L0 / |d|) d with d = X_j - X_i (minimum image),
 * the discrete tension law of sec. 2.2 generalised to rest length (sec. 8).
 * On success *out receives the handle; on failure *out is NULL. */
IB_API int ib_setup(const ib_params* params, int32_t n_points, const double* X,
             int32_t n_springs, const int32_t* springs, const double* kappa,
             const double* rest, void* stream, ib_problem** out);

/* Replace the point positions by device X [n_points][2] and rebuild S, J, the
 * coarse elasticity patches and all box factors (the per-step re-forming of
 * S A_f S^* described in sec. 8). */
IB_API int ib_update_points(ib_problem* prob, const double* X_dev);

/* y = A_level w in FP64 (device pointers, 3 N_level^2 doubles each, must not
 * alias).  A_0 is the fine operator of the system above; A_l (l >= 1) is the
 * hybrid coarse operator of sec. 3.2: Stokes re-discretised with h_l plus
 * dt * R E_{l-1} P.  level in [0, n_levels). */
IB_API int ib_apply(ib_problem* prob, int32_t level, const double* w, double* y);

/* One V-cycle (Algorithm 1, nu1/nu2 sweeps, zero initial guess) on the fine
 * level: w = MGV(0, b).  device b, w: 3N^2 doubles (may not alias).  With
 * IB_FP32_PRECOND the cycle runs in FP32 and b, w are converted at entry and
 * exit; with IB_MIXED_PRECOND the free-box solves apply an FP32 inverse. */
IB_API int ib_vcycle(ib_problem* prob, const double* b, double* w);

/* b = [-(rho/dt) u^n - S F(X); 0] for the current points (device, 3N^2
 * doubles).  u_n: device [2][N][N] doubles or NULL for a fluid at rest.  With
 * IB_WALLS_NOSLIP the wall faces are zero and the moving lid (params.lid) adds
 * -2 mu u_lid(x_i) / h^2 to the u rows next to it. */
IB_API int ib_rhs(ib_problem* prob, const double* u_n, double* b);

/* One implicit IB step (sec. 2.3):
 *   u_n    device [2][N][N] velocity at t^n, or NULL (fluid at rest)
 *   up     device [3][N][N] output: u, v, p at t^{n+1}, pressure with zero mean
 *   X      device [n_points][2]: in X^n, out X^{n+1} = X^n + dt S^*(X^n) u^{n+1}
 *   stats  host, may be NULL
 * Re-forms S, J and the hierarchy from X^n, solves with MG-preconditioned
 * FGMRES to params.tol, then moves the points.  Returns IB_ERR_NOT_CONVERGED
 * if max_iters was reached (the best iterate is still written and X moved),
 * IB_ERR_TIMEOUT if a bulk copy of the Krylov basis did not land within the wait
 * limit: 1 s, or the number of nanoseconds in the environment variable
 * IB_WAIT_LIMIT_NS when it is set at ib_setup (0 makes every wait that does not
 * find its copies already landed time out, which exercises this path; the
 * iterate is then meaningless).
 * FGMRES orthogonalises by classical Gram-Schmidt applied twice, in three
 * passes over the basis; the environment variable IB_CGS_FUSED=0 (read at
 * ib_setup) splits the middle pass in two, the form otherwise taken only when a
 * 64-element slice of the whole basis does not fit in shared memory.  Bases of up
 * to 16 vectors take a register form of the middle pass; IB_CGS_REG=0 (read at
 * ib_setup) keeps them on the bulk-copy form.
 * Reproducibility: with the assembled elasticity rows (the default), the same
 * inputs give bit-identical results from run to run: the right-hand side's
 * spread, the operator's spread and the level-0 row assembly gather through
 * per-row point lists in a fixed order, and every reduction sums in a fixed
 * order.  IB_ROW_LISTS=0 (read at ib_setup) takes the scatter forms with FP64
 * atomic additions instead (about 1 ms less set-up on a 1024^2 grid with 32 768
 * points; results then vary at the rounding level).
 * With IB_FP32_PRECOND, a step below the stiffness threshold (IB_STIFF_SIGMA)
 * eliminates its structure boxes in FP32, the inverses kept and applied in FP64
 * as before; a solve that escalates to the mixed V-cycle re-forms and
 * inverts them in FP64 first.  IB_INV32=0 (read at ib_setup) always inverts in
 * FP64; IB_INV32=2 (read at every set-up) eliminates in FP32 for every step of
 * the FP32 and mixed V-cycles, stiff ones included, without the FP64
 * re-forming.  IB_POISON=1 (read at the
 * library's first allocation) fills every new device allocation with all-ones
 * bytes (NaN), a test aid that makes reads of unwritten memory show. */
IB_API int ib_solve_step(ib_problem* prob, const double* u_n, double* up, double* X,
                  ib_stats* stats);

/* One implicit step with the spring force taken at the new positions: the
 * backward-Euler step whose force is F(X^{n+1}) rather than its linearisation
 * about X^n, solved by Newton's method (sec. 8 names Newton's method for nonlinear
 * force laws; each iteration is a linearised system of the form ib_solve_step
 * solves).  S and S^* stay at X^n (lagged, sec. 2.3); iteration k evaluates the
 * springs' force and Jacobian at X^k = X^n + dt S^* u^k (u^0 = 0) and solves
 *   [mu Lap - (rho/dt) + dt S J(X^k) S^*] u - G p = -(rho/dt) u^n - S [F(X^k) - J(X^k)(X^k - X^n)],
 *   D u = 0
 * with the MG-preconditioned FGMRES of ib_solve_step; the first iterate is
 * ib_solve_step's result.  Iterates until max |X^{k+1} - X^k| <= tol_newton * h
 * (after at least two solves) or max_newton solves.  The converged step does not
 * depend on the Jacobian variant (IB_JAC_EXACT converges quadratically, the
 * clamped one linearly).  Arguments as for ib_solve_step (device pointers, X
 * updated in place to X^{n+1}); stats: iters summed over the solves, t_setup_ms
 * and t_solve_ms summed, the other fields from the last solve.  newton (host
 * memory, two doubles, may be NULL): newton[0] = solves done, newton[1] = the last
 * max |X^{k+1} - X^k| / h.  Errors: IB_ERR_INVALID_ARG (max_newton < 1,
 * tol_newton < 0, the explicit-time method, NULL X with points) and those of
 * ib_solve_step; IB_ERR_NOT_CONVERGED if a linear solve stops at max_iters (the
 * iteration ends there). */
IB_API int ib_solve_step_newton(ib_problem* prob, const double* u_n, double* up, double* X,
                                int32_t max_newton, double tol_newton, ib_stats* stats, double* newton);

/* Solve A_0 x = b for a given right-hand side with the current hierarchy (the
 * points of ib_setup or the last ib_update_points / ib_solve_step), by the same
 * MG-preconditioned FGMRES from x = 0 (sec. 3.3):
 *   b      device [3][N][N] doubles (with no-slip walls its wall faces are zeroed)
 *   x      device [3][N][N] output, pressure with zero mean (may not alias b)
 *   stats  host, may be NULL (t_setup_ms = 0)
 * The points do not move.  Returns as ib_solve_step. */
IB_API int ib_solve(ib_problem* prob, const double* b, double* x, ib_stats* stats);

/* Number of levels in the hierarchy and the grid size of a level. */
IB_API int ib_num_levels(const ib_problem* prob);
IB_API int ib_level_size(const ib_problem* prob, int32_t level);

/* Grid size of the finest level run by the coarse-level ("tail") kernel in the
 * V-cycle of the given precision (IB_FP32_PRECOND for the FP32 V-cycle, IB_FP64 or
 * IB_MIXED_PRECOND for the one on FP64 vectors), 0 if that V-cycle does not exist.
 * The tail runs every sweep, transfer and the coarsest solve of its levels in
 * one launch, on one CTA (arrays in shared memory) or on one thread-block
 * cluster (arrays in global memory, levels up to 128^2).  The split and the form
 * are timed at set-up unless the environment variable IB_TAIL_NMAX (the largest
 * grid size for the tail) pins them; IB_TAIL_CLUSTER=1 then asks for the cluster
 * form and IB_TAIL_CLUSTER=0 excludes it from the timing as well. */
IB_API int ib_tail_grid(const ib_problem* prob, int32_t precision);

/* CTAs of the thread-block cluster that runs the tail kernel of the V-cycle of the
 * given precision, 0 for the single-CTA form or if that V-cycle does not exist. */
IB_API int ib_tail_cluster(const ib_problem* prob, int32_t precision);

/* Levels with at least IB_BOX_GEMM_MIN boxes per colour (environment variable,
 * default 2048) solve their n x n boxes (n = 2, 4) with a register-blocked kernel
 * that treats the free boxes of a CTA as one small matrix product; levels with at
 * most IB_BOX_ONE_MAX (default 512) give each box its own CTA with its inverse in
 * shared memory; the levels between use one thread per box row, several boxes per
 * CTA.  Both read at ib_setup. */

/* Form of the n x n box kernel (n = 2, 4) on a smoothing level of the V-cycle of the given
 * precision, as the set-up autotuner chose it by timing one colour phase of each form
 * on the problem's own hierarchy: 1 one box per CTA, 2 a thread per box row (several
 * boxes per CTA), 3 the register-blocked product, 4 / 5 / 6 the strip kernel with 8 /
 * 16 / 32 boxes per strip, 7 eight boxes per 64-thread CTA, each thread one row of
 * all eight (FP32 V-cycle, 4 x 4 boxes); 0 when no form was timed (the size rule above applies: 1 x 1
 * or 8 x 8 boxes, IB_BOX_TUNE=0, or an IB_BOX_* variable set); -1 for an invalid
 * argument.  The environment variable IB_BOX_FORMS (comma-separated codes, finest
 * level first, read at ib_setup) gives the forms instead of timing them (a form that
 * does not apply to its level falls back to the size rule). */
IB_API int ib_box_form(const ib_problem* prob, int32_t precision, int32_t level);

/* Number of structure boxes (boxes whose block includes elasticity) on a level,
 * as found by the last set-up. */
IB_API int ib_num_struct_boxes(const ib_problem* prob, int32_t level);

/* ---- Batches of independent problems (not in the paper) ----
 *
 * A batch holds nprob independent problems of any grid sizes and parameters.
 * Each problem gets its own CUDA stream (highest priority for problems with
 * dt * max(kappa) / mu >= 3000, which set the batch's makespan) and its own
 * captured V-cycle graph, and
 * a pool of host threads (up to 16; the environment variable IB_BATCH_THREADS
 * overrides the count) drives the problems' FGMRES iterations at the same time,
 * so the small, latency-bound launches of different problems overlap on the GPU.
 * ib_solve_step_batch takes the problems longest first by the estimate
 * N^2 min(1 + sigma / 1000, max_iters / 8), sigma = dt * max(kappa) / mu, on the
 * fewest threads whose longest-first schedule of these estimates ends within 5 %
 * of the costliest problem (a few stiff problems and many cheap ones: the cheap
 * ones run one after another beside the stiff ones instead of all at once).
 *   params   host [nprob]
 *   pt_off   host [nprob + 1] point offsets (pt_off[0] = 0); sp_off likewise for springs
 *   X, springs, kappa, rest   host, concatenated per problem; spring indices are
 *            local to their problem
 *   stream   the caller's stream: ib_solve_step_batch starts after the work already
 *            queued on it and the caller's stream waits for the whole batch
 * Storage of the batched vectors: problem k's block of up_all starts at
 * sum_{i<k} 3 N_i^2 doubles, of u_n_all at sum_{i<k} 2 N_i^2, of X_all at
 * 2 pt_off[k]. */
typedef struct ib_batch ib_batch;
IB_API int ib_setup_batch(int32_t nprob, const ib_params* params, const int32_t* pt_off, const double* X,
                          const int32_t* sp_off, const int32_t* springs, const double* kappa,
                          const double* rest, void* stream, ib_batch** out);
/* One implicit step of every problem (see ib_solve_step).  u_n_all device or NULL;
 * up_all, X_all device; stats host [nprob] or NULL.  Returns the worst status over
 * the problems (IB_ERR_NOT_CONVERGED only if every other problem succeeded). */
IB_API int ib_solve_step_batch(ib_batch* batch, const double* u_n_all, double* up_all, double* X_all,
                               ib_stats* stats);
IB_API int ib_batch_size(const ib_batch* batch);
/* The k-th problem of the batch (owned by the batch; do not destroy it). */
IB_API ib_problem* ib_batch_problem(ib_batch* batch, int32_t k);
IB_API void ib_destroy_batch(ib_batch* batch);

/* ---- Learned preconditioner stage (not in the paper) ----
 *
 * A 3-level convolutional U-Net (16/32/64 channels, 3x3 circular convolutions,
 * GELU, 2x2 average pooling, nearest upsampling with skip concatenation, a 1x1
 * head; BF16 weights with FP32 master copies, FP32 accumulation) that maps the
 * residual left by a V-cycle to an estimate of the remaining error.  The residual
 * is first brought to velocity-error units, rs = (h^2/mu r_u, h^2/mu r_v, h r_p).
 * Input channels: rs / ||rs||, and a structure channel
 * log(1 + dt/(mu h^2) sum_k Kbar_k phi phi) (Kbar_k = summed stiffness of the
 * springs at point k).  Output: the error estimate divided by ||rs|| (the pressure
 * channel further divided by mu/h).
 * Parameters are one FP32 vector of ib_unet_num_params() values in layer order
 * [W_0 b_0 W_1 b_1 ...], W_l in [c_out][c_in][k][k].  All arrays device FP32
 * [C][N][N] unless stated; N a power of two in 64..4096. */
typedef struct ib_unet ib_unet;
IB_API int64_t ib_unet_num_params(void);
/* params: host FP32 initial parameters (NULL = zeros); stream as for ib_setup. */
IB_API int ib_unet_create(int32_t N, const float* params, void* stream, ib_unet** out);
IB_API int ib_unet_set_params(ib_unet* net, const float* params /* host */);
IB_API int ib_unet_get_params(ib_unet* net, float* params /* host */);
/* y [3][N][N] = net(x [4][N][N]) */
IB_API int ib_unet_forward(ib_unet* net, const float* x, float* y);
/* loss = ||net(x) - t||^2 / ||t||^2 and its gradient (host, num_params values; may be NULL) */
IB_API int ib_unet_loss_grad(ib_unet* net, const float* x, const float* t, double* loss, float* grad);
/* one Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr on that loss */
IB_API int ib_unet_train_step(ib_unet* net, const float* x, const float* t, float lr, double* loss);
IB_API void ib_unet_destroy(ib_unet* net);
/* Attach (net != NULL) or detach the learned stage of a problem (same N; the problem
 * does not own the network).  With a stage attached each FGMRES direction z = MG(v)
 * becomes z + alpha d, d the network's correction for r = v - A z and alpha the
 * exact minimiser of ||r - alpha A d||, when alpha > 0 and the residual drops by at
 * least 0.1 %; otherwise the V-cycle direction is kept.  After 3 consecutive
 * rejections the stage is not evaluated again in that solve. */
IB_API int ib_set_learned_stage(ib_problem* prob, ib_unet* net);
/* A training pair from the method itself: b = A x, z = MG(b) (one V-cycle of the
 * problem's precision), r = b - A z, e = x - z; writes the network input for r to
 * in4 [4][N][N] and the scaled error (as the network's output is defined) to target
 * [3][N][N].  x: device 3N^2 doubles. */
IB_API int ib_learned_pair(ib_problem* prob, const double* x, float* in4, float* target);
/* One step of multigrid as a stand-alone solver (sec. 5) on an error: with e = x* - x_k
 * (device, 3N^2 doubles, updated in place to e - MG(A e) = x* - x_{k+1}) writes the
 * pair of ib_learned_pair for x = e, i.e. the network input for the residual
 * r_{k+1} = A e_{k+1} left after the V-cycle and the scaled error e_{k+1}.  Repeated
 * from e = x* (x_0 = 0) it yields the residual -> error pairs the method produces
 * while it solves. */
IB_API int ib_learned_chain(ib_problem* prob, double* e, float* in4, float* target);

/* Kernel classes for launch counting and event timing. */
enum {
  IB_KC_STOKES = 0,   /* level Stokes residual / apply */
  IB_KC_BOX = 1,      /* box-smoother solves of one colour */
  IB_KC_INTERP = 2,   /* interpolation S^*_l w of the elasticity term */
  IB_KC_SPREAD = 3,   /* J U and spreading S_l (elasticity term) */
  IB_KC_TRANSFER = 4, /* restriction, prolongation and correction */
  IB_KC_COARSE = 5,   /* exact coarsest solve */
  IB_KC_KRYLOV = 6,   /* FGMRES vector kernels and scalar updates */
  IB_KC_SETUP = 7,    /* patches, springs, box assembly and inverses */
  IB_KC_OTHER = 8,    /* fills, casts, right-hand side, point update */
  IB_KC_COUNT = 9
};

/* Kernel launches issued by this problem since set-up (all classes, or one class
 * when kclass is in [0, IB_KC_COUNT)); -1 for a NULL handle. */
IB_API int64_t ib_launch_count(const ib_problem* prob, int32_t kclass);

/* enable = 1: from now on bracket every kernel launch with CUDA events on the
 * problem's stream (adds event records between launches; use it in a separate
 * measurement pass).  enable = 0: stop.  Either call resets the accumulators. */
IB_API int ib_profile(ib_problem* prob, int32_t enable);

/* Synchronise the stream and return, for one kernel class, the number of timed
 * launches, their summed device time (ms) and their summed algorithmic bytes
 * (the bytes the operation must move: unique reads plus writes, as defined per
 * class in the design notes).  Output pointers may be NULL. */
IB_API int ib_profile_read(ib_problem* prob, int32_t kclass, int64_t* launches, double* ms,
                           double* bytes);

/* enable = 1: from now on record an event pair on the problem's stream around every
 * V-cycle replayed from its CUDA graph (the form FGMRES and ib_vcycle run; the
 * kernels themselves are unchanged, unlike ib_profile's per-launch brackets);
 * enable = 0: stop.  Either call resets the counts. */
IB_API int ib_vcycle_timer(ib_problem* prob, int32_t enable);

/* Synchronise the stream and return the number of V-cycles timed since
 * ib_vcycle_timer and their summed device time (ms), for the V-cycle of the given
 * precision: IB_FP32_PRECOND for the FP32 V-cycle, IB_FP64 or IB_MIXED_PRECOND for
 * the one on FP64 vectors.  Output pointers may be NULL. */
IB_API int ib_vcycle_timer_read(ib_problem* prob, int32_t precision, int64_t* count, double* ms);

/* ---- Allocation-free operator apply (the paper has no counterpart) ----
 *
 * y = A_0 w on the fine grid, the same operator as ib_apply(prob, 0, w, y),
 * computed without a problem handle and without allocating any device memory.
 * It is meant for callers that cannot allocate device memory: code that must not
 * stall on cudaMalloc's implicit device synchronisation in the middle of a time
 * step, or a host framework that owns all device memory through its own pool and
 * does not let libraries allocate.
 *   params   host; uses N, L, rho, mu, dt, delta and jacobian (periodic square only:
 *            walls must be IB_WALLS_PERIODIC)
 *   X        device [n_points][2];  springs device int32 [n_springs][2];
 *   kappa, rest  device [n_springs];  w, y  device 3 N^2 doubles (must not alias)
 *   stream   cudaStream_t (NULL = legacy default stream)
 * The one scratch array it needs (the velocity interpolated to the points) is a
 * fixed static device array of 2 * IB_NOALLOC_MAX_POINTS doubles (1 MiB) that
 * every GPU which loads the library holds until the process exits; calls with
 * n_points > IB_NOALLOC_MAX_POINTS return IB_ERR_INVALID_ARG.  All calls on a
 * device share that array and it keeps the previous call's contents, so calls
 * that overlap on the GPU (other streams or threads) race and must be serialised
 * by the caller.  The first call on each device looks up the array's address
 * with cudaGetSymbolAddress while that device is current; make that first call
 * before any stream capture.  The call waits for its stream to finish (it reads
 * back a device error word) and returns IB_ERR_INVALID_ARG for out-of-range or
 * coincident spring end points. */
#define IB_NOALLOC_MAX_POINTS 65536
IB_API int ib_apply_noalloc(const ib_params* params, int32_t n_points, const double* X,
                            int32_t n_springs, const int32_t* springs, const double* kappa,
                            const double* rest, const double* w, double* y, void* stream);

/* Release all device memory of the problem.  NULL is ignored. */
IB_API void ib_destroy(ib_problem* prob);

/* Message for the last failing call on this thread ("" if none). */
IB_API const char* ib_last_error(void);

/* Library version string. */
IB_API const char* ib_version(void);

#ifdef __cplusplus
}
#endif
#endif /* IB_H_ */
