/*
 * ptp.h -- C ABI of the GB300 time-periodic parabolic solver.
 *
 * The library solves the implicit-Euler, time-periodic problem of Problem 1
 * (Section 2, eq. disc1-disc2):
 *
 *     M (u^n - u^{n-1}) / tau + K(u^n) = f^n,   n = 1..N,   u^0 = u^N,
 *
 * for P1 finite elements on triangles (Section 4), with
 *     K(u)_i = sum_T nu(|grad u|_T) |T| grad(u)_T . grad(phi_i),
 *     nu(s)  = nu_min + (nu_max - nu_min) s^2 / (s^2 + s_sat^2) on iron
 *              elements and nu_linear elsewhere,
 *     M      = sigma-weighted consistent P1 mass (degenerate where sigma = 0),
 *     f^n_i  = sum_c amp_c sin(2 pi t^n / T + phase_c) int(chi_c phi_i),
 *              t^n = n tau, tau = T / N,
 * by the fixed-point iteration of eq. (iter1)-(iter2) with
 * K_hat = L = nu_max * (unit-coefficient stiffness), in correction form
 *     (M + tau L) d^n - M d^{n-1} = tau (f^n - A(U)^n),  U <- U + d,
 * each periodic linear system being solved by multigrid in time
 * (Remark on parallel solvers, Section 3; method (M1), Section 4).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: PTP_OK (0) or a negative PTP_E* code.  No C++ exception
 *    crosses this boundary.  ptp_last_error() gives a message.
 *  - Space-time vectors ("[n_free][N]") hold the free (non-Dirichlet) nodes
 *    in ascending node id, node-major with the time index fastest:
 *    X[i * N + (n - 1)] is the value at free node i and time step n.
 *  - Functions without suffix take HOST pointers; the library copies in and
 *    out on its stream and returns after the result is on the host.
 *    Functions with suffix _dev take DEVICE pointers (on the context's
 *    device), enqueue on the context's stream and return without waiting
 *    unless stated otherwise.
 *  - The caller owns every buffer it passes; the library owns its internal
 *    device state, which lives until ptp_destroy().
 *  - A context is not thread-safe; use one context per host thread.
 */
#ifndef PTP_H
#define PTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PTP_OK        0
#define PTP_EINVAL   -1   /* invalid argument or inconsistent sizes        */
#define PTP_ECUDA    -2   /* a CUDA runtime call failed                    */
#define PTP_ENOTCONV -3   /* max iterations reached; outputs hold the last
                             iterate and the statistics are filled          */
#define PTP_ENAN     -4   /* a non-finite residual norm was detected        */
#define PTP_ESTATE   -5   /* call order violated (e.g. solve before setup)  */
#define PTP_ENOMEM   -6   /* device allocation failed                       */

/* ---- precision of the inner (linear) solve --------------------------- */
#define PTP_FP64  0       /* every kernel in double                         */
#define PTP_MIXED 1       /* multigrid-in-time, smoother, PCG and SpMM in
                             float with float accumulation; outer residual,
                             update and coarsest periodic solve in double   */

/* ---- spatial preconditioner of the batched PCG ----------------------- */
#define PTP_PREC_JACOBI 0 /* diagonal scaling                               */
#define PTP_PREC_GMG    1 /* geometric multigrid V-cycle on the nested
                             structured grids (needs ptp_set_structured)    */

/* ---- exact periodic solve of the last multigrid-in-time level --------- */
#define PTP_COARSE_VCYCLES 0 /* N_c = 1: tau_c L x = b; N_c = 2: sum and
                                difference split (both SPD, PCG in double);
                                a truncated hierarchy: coarse_cycles V-cycles
                                of the levels below                          */
#define PTP_COARSE_DFT     1 /* discrete Fourier transform in time (Remark on
                                parallel solvers, Section 3): mode k solves
                                ((1 - e^{-2 pi i k/N_l}) M + tau_l L) x_k = b_k,
                                k = 0..N_l/2 (conjugate symmetry), by
                                conjugate-orthogonal CG in double with the
                                tau_l L multigrid V-cycle as preconditioner;
                                time_levels = 1 makes it the whole inner solve */

typedef struct ptp_ctx ptp_ctx;

/* Solver options; ptp_default_opts() fills sensible defaults. */
typedef struct ptp_opts {
    double tol;          /* stop when ||F - A(U^k)||_2 <= tol ||F - A(U^0)||_2
                            (stopping rule of Section 4)                     */
    int    max_outer;    /* maximum fixed-point iterations                   */
    int    precision;    /* PTP_FP64 or PTP_MIXED                            */
    int    time_levels;  /* multigrid-in-time levels used by the V-cycle;
                            0 = all (coarsen by 2 while N_l is even and
                            N_l > coarse_steps); see coarse_cycles           */
    int    coarse_steps; /* N_c of the coarsest level: 1 or 2 (exact solve)  */
    int    vcycles;      /* multigrid-in-time V-cycles per outer step        */
    int    pre_smooth;   /* damped block-Jacobi sweeps before coarsening
                            (default 1)                                      */
    int    post_smooth;  /* ... and after; < 0 (default): chosen with
                            omega_t, see below                               */
    double omega_t;      /* block-Jacobi damping; <= 0 (default): chosen per
                            problem.  On a spatial mode with eigenvalue
                            lambda of L x = lambda M x the periodic system of
                            level l is (1 + kappa_l) x^n - x^{n-1} with
                            kappa_l = tau_l lambda; the V(pre, post) cycle
                            with omega near 1 contracts fast for kappa >= 1
                            but amplifies slow modes with kappa -> 0.  Set-up
                            estimates lambda_min by inverse iteration and
                            takes the cheapest (post, omega) whose cycle has
                            a model spectral radius <= 0.6 for every
                            kappa >= 0.9 tau_0 lambda_min (ptp_stats reports
                            the choice)                                      */
    int    pcg_iters;    /* PCG iterations per block-Jacobi spatial solve    */
    int    spatial_prec; /* PTP_PREC_JACOBI or PTP_PREC_GMG                  */
    int    gmg_smooth;   /* damped-Jacobi sweeps per GMG level (pre = post)  */
    double gmg_omega;    /* damping of those sweeps (default 0.7)            */
    double coarse_tol;   /* relative tolerance of the coarsest-level PCG     */
    int    coarse_max_it;/* iteration cap of the coarsest-level PCG          */
    int    use_graph;    /* capture one outer step in a CUDA graph           */
    int    check_every;  /* host reads the residual every this many steps    */
    int    coarse_cycles;/* when time_levels stops above the 1- or 2-step
                            bottom, the periodic problem of its last level is
                            solved "exactly" by this many V-cycles of the
                            remaining hierarchy (two-level method: time_levels
                            = 2)                                             */
    int    coarse_solver;/* exact periodic solve of the last level used:
                            PTP_COARSE_VCYCLES (the 1- or 2-step split at the
                            bottom, coarse_cycles V-cycles above it) or
                            PTP_COARSE_DFT (time DFT, one complex shifted
                            spatial solve per mode; any N_l <= 1022)          */
    int    dft_max_it;   /* iteration cap of each DFT mode solve (COCG)      */
    double init_tol;     /* tolerance of the static initialisation (0: tol) */
    int    init_static;  /* 1: a solve without U0 starts from the static
                            solutions (initialisation of Section 4)         */
    double newton_eta;   /* Newton: relative tolerance of each linear solve
                            (default 1e-2)                                   */
    int    krylov_dim;   /* Newton: flexible GMRES iterations per linear
                            solve (1..31, no restart; default 20)            */
    int    stencil;      /* structured grids, PTP_MIXED, GMG: 1 = the float
                            inner solve runs the shared-memory stencil
                            kernels (fused residual + restriction,
                            interpolation + sweep + dot products; default),
                            0 = the padded-ELL row kernels                   */
    int    k1_fused;     /* structured grids, saturating law: 1 = the outer
                            residual in one fused pass (shared-memory element
                            fluxes), 0 = element pass + node pass (default)  */
    int    coarse_direct;/* 1 (default): on a uniform structured grid with
                            K_hat = nu_max * stiffness and (nx - 1), (ny - 1)
                            powers of two, the tau_c L solve of the coarsest
                            time level is direct (sine transforms, exact up
                            to rounding) instead of coarse_tol PCG; 0 = PCG */
    int    fuse_coarse;  /* 1: in PTP_MIXED fixed-point solves on the
                            stencil path, the multigrid-in-time work of the
                            time levels with at most 16 steps runs as one
                            cooperative kernel with a grid-wide barrier
                            between its passes (same results bit for bit,
                            half the launches).  0 (default): separate
                            launches, which measured faster on a GB300       */
    int    fuse_update;  /* 1 (default): fewer passes over the iterates of
                            the time levels, with the same results bit for
                            bit.  On the stencil path a pre-sweep from zero
                            with one PCG iteration leaves its update
                            x = omega_t alpha p to the time restriction that
                            follows, which forms x on the fly and stores it;
                            and in a V(pre, 0) cycle (one per outer step)
                            the prolongations of every level and the update
                            of U run as one pass.  0 = separate kernels     */
} ptp_opts;

/* Statistics of the last solve. */
typedef struct ptp_stats {
    int    outer_iterations;  /* fixed-point steps taken                     */
    int    converged;         /* 1 if the stopping rule was met              */
    double res0;              /* ||F - A(U^0)||_2                            */
    double res_final;         /* ||F - A(U^k)||_2 at the returned iterate    */
    double setup_ms;          /* operator/hierarchy set-up time              */
    double solve_ms;          /* wall time of the solve call                 */
    double residual_ms;       /* device time of the last residual evaluation */
    int64_t kernel_launches;  /* kernels launched by the solve (graph nodes
                                 counted once per replay)                    */
    int    time_levels;       /* levels actually used                        */
    int    spatial_levels;    /* GMG levels actually used (1 = none)         */
    double init_ms;           /* wall time of the static initialisation      */
    int    init_iterations;   /* its fixed-point steps (0: not run)          */
    int    inner_iterations;  /* Newton: Krylov iterations of all steps      */
    double omega_t;           /* time smoother used: damping ...             */
    int    post_smooth;       /* ... and post-smoothing sweeps               */
    double kappa_min;         /* tau_0 lambda_min(L, M) behind an automatic
                                 choice (0 if none was made)                 */
} ptp_stats;

void        ptp_default_opts(ptp_opts* opts);

/* Host-only model of the multigrid-in-time cycle (no GPU is used).  On the
   scalar periodic system (1 + kappa_l) x^n - x^{n-1} = b^n of each level
   (N_l = Nl[l] steps, Nl[l] = 2 Nl[l+1], the last level solved exactly,
   kappa_l = kappa0 Nl[0] / Nl[l]): damped Jacobi (omega), pair-sum
   restriction, injection.  ptp_time_cycle_rho writes the spectral radius of
   the V(pre, post) cycle's error propagation (power iteration);
   ptp_choose_time_smoother the choice that the automatic omega_t and
   post_smooth make for kappa >= kappa_min (post < 0 / omega <= 0: free).
   Both return PTP_EINVAL for bad sizes or a hierarchy that does not halve. */
int ptp_time_cycle_rho(const int* Nl, int levels, double kappa0, int pre, int post, double omega, double* rho);
int ptp_choose_time_smoother(const int* Nl, int levels, double kappa_min, int pre, int post, double omega,
                             int* post_out, double* omega_out, double* rho_out);
const char* ptp_version(void);
/* sizeof(ptp_opts) and sizeof(ptp_stats) as compiled into the library, so a
   binding can check its own struct layouts.  Either pointer may be NULL. */
void        ptp_abi_sizes(size_t* opts_bytes, size_t* stats_bytes);

/* Create a context for CUDA device `device` (>= 0).  No CUDA call is made
   here: the device is first used by ptp_setup or ptp_set_stream, which also
   create the context's own non-blocking stream.  The set_* calls below only
   record host data and work without a GPU. */
int  ptp_create(ptp_ctx** out, int device);
/* Free all device memory and the context.  Accepts NULL. */
void ptp_destroy(ptp_ctx* ctx);
/* Message of the last failing call on this context ("" if none). */
const char* ptp_last_error(const ptp_ctx* ctx);
/* Use an external CUDA stream (cudaStream_t passed as void*; NULL = the
   context's own stream).  The caller keeps the stream alive. */
int  ptp_set_stream(ptp_ctx* ctx, void* stream);

/* ---- problem definition (host pointers, copied) ---------------------- */

/* Triangle mesh: xy[2*n_nodes] coordinates, tri[3*n_tri] counter-clockwise
   vertex ids (0-based), dirichlet[n_nodes] = 1 for homogeneous Dirichlet
   nodes (u = 0, Section 4).  Returns PTP_EINVAL for vertex ids out of range
   or non-finite coordinates; clockwise or degenerate triangles make
   ptp_setup return PTP_EINVAL. */
int ptp_set_mesh(ptp_ctx* ctx, int n_nodes, const double* xy, int n_tri,
                 const int32_t* tri, const uint8_t* dirichlet);

/* Declare that the mesh is the uniform nx-by-ny grid on [x0,x1]x[y0,y1]
   with node (i,j) = j*nx+i, cells split along (i,j)-(i+1,j+1), boundary
   Dirichlet, and build exactly that mesh (replacing any previous mesh).
   Enables the geometric-multigrid preconditioner when nx-1 and ny-1 are
   divisible by 2 on at least one coarsening.  PTP_EINVAL unless nx, ny >= 2,
   nx * ny <= 2^28 and the bounds are finite with x0 < x1, y0 < y1. */
int ptp_set_structured(ptp_ctx* ctx, int nx, int ny, double x0, double y0,
                       double x1, double y1);

/* Materials per element (Section 4, "Test problem"): conductivity sigma_e
   (finite, >= 0), nonlinear_e = 1 for the iron law, else nu_linear; both
   arrays hold n_tri entries of the mesh set last.  PTP_EINVAL unless
   0 < nu_min <= nu_max, 0 < nu_linear (both finite) and
   1e-15 <= s_sat <= 1e15. */
int ptp_set_materials(ptp_ctx* ctx, const double* sigma_e,
                      const uint8_t* nonlinear_e, double nu_min,
                      double nu_max, double s_sat, double nu_linear);

/* Reluctivity law of the paper's transformer (Section 4, "Test problem") on
   the nonlinear elements instead of the saturating law:
       nu(s) = a min(exp(b s^2), c) + d,
   abcd[4 * n_tri] = (a, b, c, d) per element, read on nonlinear elements
   only (a >= 0, b > 0, c >= 1, d > 0).  NULL restores the saturating law.
   Call after ptp_set_materials.  The adjoint and Newton entry points reject
   this law. */
int ptp_set_law_exp(ptp_ctx* ctx, const double* abcd);

/* Per-element weights of the linear operator of the fixed-point iteration,
   K_hat = sum_T khat_e[T] A_T (A_T the unit-coefficient element stiffness;
   eq. iter1, Theorem 3 allows any linear symmetric elliptic K_hat).  khat_e:
   n_tri positive doubles; NULL restores K_hat = nu_max A. */
int ptp_set_khat(ptp_ctx* ctx, const double* khat_e);

/* Coils: coil_of_elem[n_tri] in [-1, n_coils), amplitude and phase per
   coil (finite); the current density on coil c is amp_c sin(2 pi t/T +
   phase_c).  n_coils = 0 removes every source (the arrays may then be NULL).
   Every entry is checked before the context changes: a call that returns
   PTP_EINVAL leaves the previous sources in place. */
int ptp_set_sources(ptp_ctx* ctx, int n_coils, const int32_t* coil_of_elem,
                    const double* amp, const double* phase);

/* Period T > 0 (finite) and number of implicit-Euler steps N >= 1
   (tau = T/N). */
int ptp_set_time(ptp_ctx* ctx, double T, int N);

/* Assemble every operator and hierarchy on the device for `opts`
   (time levels, precision and preconditioner are fixed here).  Must be
   called after the set_* calls and again after any of them. */
int ptp_setup(ptp_ctx* ctx, const ptp_opts* opts);

/* Sizes after ptp_setup: free nodes, time steps, triangles, time levels. */
int ptp_sizes(const ptp_ctx* ctx, int* n_free, int* N, int* n_tri,
              int* time_levels);

/* Structure counts after ptp_setup, for roofline arithmetic.  counts[k] is
   written for k < n (n <= PTP_INFO_COUNT); returns the number written.
     0 free nodes   1 time steps N     2 triangles       3 iron triangles
     4 iron element-node incidences    5 nonzeros of the linear-element
     stiffness      6 nonzeros of the mass (M/tau) rows  7 nonzeros of the
     level-0 spatial operator M + tau L                  8 spatial levels
     9 time levels  10 coils  11 threads per block of the row kernels
    12 largest time tile of the stencil kernels   13 their blocks per SM     */
#define PTP_INFO_COUNT 14
int ptp_info(const ptp_ctx* ctx, int64_t* counts, int n);

/* Launch-schedule autotuner of this context.  Times the level-0 SpMM with
   128, 256 and 512 threads per block (rows per block = threads / (N /
   vector width)) and keeps the fastest for every row kernel; on structured
   grids with the stencil kernels (PTP_MIXED) it also times whole outer
   steps of the fixed point (from zero, stopping rule off; the iterate is
   left undefined) for time tiles of up to 8, 16, 32 and 64 columns and row
   strips aiming at 2, 3, 4 and 6 blocks per SM, and keeps the fastest pair
   (ptp_info entries 12 and 13).  *block_threads and *best_us (per launch of
   the SpMM) may be NULL.  Synchronises. */
int ptp_autotune(ptp_ctx* ctx, int* block_threads, double* best_us);

/* ---- batched independent instances ----------------------------------- */

/* A batch advances many set-up contexts (uneven meshes and N allowed) with
   one CUDA-graph launch per fixed-point step.  In PTP_BATCH_MERGED mode (the
   default) the outer step of every instance is recorded and the recordings
   are merged: launches of the same kernel kind at aligned positions of the
   instances' steps become one launch over a work-list of (instance, its
   blocks), so the kernels per step do not grow with the number of
   instances.  An instance whose step has work without a batched form (the
   exponential law, the ELL kernels of unstructured meshes, the DFT time
   solver, the fused K1 option) runs as a parallel branch of the same graph;
   PTP_BATCH_BRANCHES runs every instance that way.  The batch does not own
   the contexts; they must stay alive and set up while the batch is used.
   Same device only. */
#define PTP_BATCH_MERGED   0
#define PTP_BATCH_BRANCHES 1
#define PTP_BATCH_AUTO     2   /* default: the faster of the two, timed */
typedef struct ptp_batch ptp_batch;
int  ptp_batch_create(ptp_batch** out, int device);
void ptp_batch_destroy(ptp_batch* batch);
const char* ptp_batch_last_error(const ptp_batch* batch);
int  ptp_batch_add(ptp_batch* batch, ptp_ctx* ctx);
int  ptp_batch_size(const ptp_batch* batch);
/* Solves every instance from zero to opts->tol (tolerance, iteration cap and
   check interval from opts; precision and hierarchy from each context's
   ptp_setup).  stats: array of ptp_batch_size entries (may be NULL);
   *n_converged (may be NULL) counts instances that met the stopping rule.
   Each instance's iterate stays in its context (read with ptp_residual_dev
   or a later ptp_solve); results are bitwise identical to solving the
   instance alone (each instance's blocks compute what its own launch would,
   in the same order).  The stats of every instance count the kernels of
   the whole batch.  Returns PTP_OK if all converged, else PTP_ENOTCONV or PTP_ENAN. */
int  ptp_batch_solve(ptp_batch* batch, const ptp_opts* opts, ptp_stats* stats, int* n_converged);
/* Copies instance i's current iterate (device U, [n_free][N]). */
int  ptp_batch_result_dev(ptp_batch* batch, int i, double* U);
/* PTP_BATCH_MERGED, PTP_BATCH_BRANCHES or PTP_BATCH_AUTO (takes effect at
   the next solve).  AUTO (the default) times a few steps of one branch per
   instance, one merged program and four merged groups when the step is
   captured, keeps the fastest, and restarts every instance from zero: merged
   launches win when the instances are small (launch-bound steps), separate
   branches when they are large enough to fill the GPU alone. */
int  ptp_batch_set_mode(ptp_batch* batch, int mode);
/* Merged mode: the instances are split into `groups` (1..64, default 4)
   groups of about equal space-time size, each merged into its own program;
   the programs run concurrently as branches of the step's graph, so kernels
   of different kinds (the double K1 of one group, the float stencil passes
   of another) overlap.  Kernels per step stay bounded by the groups, not the
   instances.  Takes effect at the next solve. */
int  ptp_batch_set_groups(ptp_batch* batch, int groups);
/* The captured step of the last ptp_batch_solve: kernels per step (merged
   launches plus those of branch instances), instances merged, merged
   launches.  Pointers may be NULL; PTP_ESTATE before the first solve. */
int  ptp_batch_plan_info(const ptp_batch* batch, int64_t* launches_per_step, int* merged_instances,
                         int* merged_launches);

/* ---- the hot path ---------------------------------------------------- */

/* Source F = (f^1..f^N), [n_free][N] (Problem 1 data, Section 4 source). */
int ptp_source(ptp_ctx* ctx, double* F);
int ptp_source_dev(ptp_ctx* ctx, double* F);

/* Outer residual R = F - A(U), A(U)^n = M (u^n - u^{n-1})/tau + K(u^n),
   u^0 = u^N (proof of Theorem 2), all [n_free][N] in double, and its
   Euclidean norm (stopping rule of Section 4).  `norm` may be NULL.
   The _dev form writes the norm to host memory after synchronising; its R
   must not be U (PTP_EINVAL). */
int ptp_residual(ptp_ctx* ctx, const double* U, double* R, double* norm);
int ptp_residual_dev(ptp_ctx* ctx, const double* U, double* R, double* norm);

/* Y = (M + tau_l L) X for the N_l = N / 2^l columns of time level l
   (the diagonal blocks of the periodic system at level l), double.  X and Y
   are different buffers (PTP_EINVAL if equal). */
int ptp_apply_shifted_dev(ptp_ctx* ctx, int level, const double* X, double* Y);
/* Same in float (the operator values rounded to float), for PTP_MIXED. */
int ptp_apply_shifted_f32_dev(ptp_ctx* ctx, int level, const float* X, float* Y);

/* R = F - A(U) and ||R|| like ptp_residual_dev, for callers that cannot let
   the library allocate device memory while they run (a framework whose own
   pool owns the device, a hard memory budget, or a loop that cannot afford
   the synchronisation of cudaMalloc/cudaFree).  The paper has no counterpart:
   this is an interface variant, not part of the method.
   U, R (may be NULL) and norm (may be NULL) are DEVICE pointers; the norm is
   written to device memory, nothing is synchronised.  The call allocates
   nothing: its scratch is a fixed 4 MiB array compiled into the library,
   held by every GPU that loads it until the process exits.  Limit: the iron
   element fluxes must fit, 2 * n_iron * N <= 522232 doubles (PTP_EINVAL with
   a message otherwise; ptp_info gives n_iron).  R must not be U, and norm
   must be neither (PTP_EINVAL).  The first call in a CUDA context looks up
   the array's device address and keeps it for that context; make that first
   call before any stream capture begins.  All calls share the array and it
   keeps the last call's contents, so calls that overlap on the GPU race. */
int ptp_residual_noalloc_dev(ptp_ctx* ctx, const double* U, double* R, double* norm);

/* Periodic operator of level l: Y^n = (M + tau_l L) X^n - M X^{n-1},
   X^0 = X^{N_l} (eq. iter1 multiplied by tau_l), double.  X and Y are
   different buffers (PTP_EINVAL if equal). */
int ptp_periodic_apply_dev(ptp_ctx* ctx, int level, const double* X, double* Y);
/* Periodic residual of level l in float, the block-Jacobi smoother's pass:
   R^n = B^n - [(M + tau_l L) X^n - M X^{n-1}], X^0 = X^{N_l}, operator
   values rounded to float.  On structured grids with the stencil path this
   is the 7-point stencil kernel of the inner solve, else the ELL kernel.
   R differs from X and B (PTP_EINVAL otherwise); PTP_MIXED contexts only. */
int ptp_periodic_residual_f32_dev(ptp_ctx* ctx, int level, const float* X, const float* B, float* R);

/* Batched PCG: solve (M + tau_l L) X = B column by column (N_l columns),
   starting from X = 0, with the preconditioner chosen at setup, until every
   column's residual is <= tol * ||b_col|| or max_it iterations.  *iters
   receives the iterations run (may be NULL).  B and X are different buffers
   (PTP_EINVAL if equal).  Synchronises. */
int ptp_spatial_solve_dev(ptp_ctx* ctx, int level, const double* B, double* X,
                          double tol, int max_it, int* iters);
int ptp_spatial_solve_f32_dev(ptp_ctx* ctx, int level, const float* B, float* X,
                              double tol, int max_it, int* iters);

/* Multigrid in time for the periodic linear system of level 0,
   (M + tau L) x^n - M x^{n-1} = b^n, x^0 = x^N: `cycles` V-cycles from
   x = 0 in the precision chosen at setup (inputs/outputs double); with
   coarse_solver = PTP_COARSE_DFT and time_levels = 1 one cycle is the DFT
   solve itself.  *relres receives ||b - P x|| / ||b|| (may be NULL).  B and X
   are different buffers (PTP_EINVAL if equal).  Synchronises. */
int ptp_periodic_solve_dev(ptp_ctx* ctx, const ptp_opts* opts, const double* B,
                           double* X, int cycles, double* relres);

/* Initialisation of Section 4: the decoupled nonlinear static problems
   K(u^n) = f^n, n = 1..N (sigma = 0, so the mass term drops), solved for all
   N steps at once by eq. (iter1) with M = 0:  L d^n = f^n - K(u^n),
   u^n <- u^n + d^n, each spatial solve a batched multigrid-preconditioned PCG
   (opts->pcg_iters iterations), from U = 0 until
   ||F - K(U)||_2 <= init_tol ||F||_2 (init_tol 0: opts->tol).  U: [n_free][N]
   doubles, host (ptp_static_solve) or device (ptp_static_solve_dev, which
   synchronises).  Returns PTP_ENOTCONV after max_outer steps.  `stats` may be
   NULL; its outer_iterations and res0/res_final describe this solve. */
int ptp_static_solve(ptp_ctx* ctx, const ptp_opts* opts, double* U, ptp_stats* stats);
int ptp_static_solve_dev(ptp_ctx* ctx, const ptp_opts* opts, double* U, ptp_stats* stats);

/* Newton's method for Problem 1 (method (M2) of Section 4): J(U) d = F - A(U)
   with the Jacobian blocks M/tau + DK(u^n) and -M/tau (cyclic), solved by
   flexible GMRES (at most krylov_dim iterations, relative tolerance
   newton_eta) preconditioned by the inner periodic solve of the fixed point
   (opts->vcycles V-cycles of multigrid in time); then U += t d with Armijo
   back-tracking t = 1, 1/2, ... on ||F - A(U)||.  Stops when
   ||F - A(U)|| <= tol ||F - A(U^0)|| or after max_outer Newton steps.  U0:
   NULL = zero start (or the static solutions with init_static).  Saturating
   law only (PTP_EINVAL for the exponential law).  Host (ptp_newton_solve) or
   device pointers (ptp_newton_solve_dev, which synchronises).  stats:
   outer_iterations = Newton steps, inner_iterations = Krylov iterations. */
int ptp_newton_solve(ptp_ctx* ctx, const ptp_opts* opts, const double* U0, double* U,
                     ptp_stats* stats);
int ptp_newton_solve_dev(ptp_ctx* ctx, const ptp_opts* opts, const double* U0,
                         double* U, ptp_stats* stats);

/* Y = J(U) V, the Jacobian of A at U applied to V (all device pointers,
   [n_free][N] doubles; Y is neither U nor V; synchronises).  Saturating law
   only. */
int ptp_jacobian_apply_dev(ptp_ctx* ctx, const double* U, const double* V, double* Y);

/* Fixed-point solve of Problem 1 (eq. iter1-iter2 in correction form) from
   U0 (NULL = zero start) to opts->tol; U receives the last iterate.
   Returns PTP_ENOTCONV if max_outer was reached, PTP_ENAN on a non-finite
   residual.  `stats` may be NULL.  The host form copies U0 in and U out
   inside the call; the _dev form synchronises before returning. */
int ptp_solve(ptp_ctx* ctx, const ptp_opts* opts, const double* U0, double* U,
              ptp_stats* stats);
int ptp_solve_dev(ptp_ctx* ctx, const ptp_opts* opts, const double* U0,
                  double* U, ptp_stats* stats);

/* ---- adjoint of the period-averaged eddy-current loss --------------- */

/* J(U) = (1/N) sum_n sum_{iron e} sigma_e (d_tau u^n)_e^T M1_e (d_tau u^n)_e,
   the eddy-current loss averaged over the period (M1_e: unit-conductivity
   consistent element mass, d_tau u^n = (u^n - u^{n-1})/tau, u^0 = u^N).
   U is a device [n_free][N] array; J is written to host memory.
   Synchronises. */
int ptp_loss_dev(ptp_ctx* ctx, const double* U, double* J);

/* Gradient of J at the solution U of Problem 1 with respect to the coil
   amplitudes (dJ_damp[n_coils]), the iron law parameters
   (dJ_dnu[3] = d/d(nu_min, nu_max, s_sat)) and the conductivity of every
   element (dJ_dsigma[n_tri]).  Implicit-function adjoint: solves the
   transposed space-time Jacobian system (backward and periodic in time,
   blocks M/tau + DK(u^n) with DK's element block
   |T| grad(phi)^T [nu I + 2 nu'(s^2) g g^T] grad(phi)) by the same fixed
   point and multigrid in time as ptp_solve, to opts->tol, then reduces
   dJ/dp = dJ/dp|_U - lambda^T d(A - F)/dp.  nu_max enters the iron law only
   (K_hat does not change the solution); nu_linear is not a parameter.
   At most 8 coils.  J, dJ_damp and dJ_dnu are host pointers (may be NULL).
   _dev: U and dJ_dsigma are device pointers; host form: host pointers.
   Returns PTP_ENOTCONV (gradients still written) if the adjoint fixed point
   did not reach opts->tol. */
int ptp_adjoint_gradient_dev(ptp_ctx* ctx, const ptp_opts* opts, const double* U, double* J,
                             double* dJ_damp, double* dJ_dnu, double* dJ_dsigma, ptp_stats* stats);
int ptp_adjoint_gradient(ptp_ctx* ctx, const ptp_opts* opts, const double* U, double* J,
                         double* dJ_damp, double* dJ_dnu, double* dJ_dsigma, ptp_stats* stats);

/* ---- measurement probes ---------------------------------------------- */

/* Measured fused multiply-add rate of the device, in TFLOP/s (2 flops per
   FMA): independent FMA chains in every thread of one full wave of blocks on
   every SM (8 and 16 chains per thread), the loop sized to about 40 ms, best
   of 3 launches of each timed with CUDA events.  fp64 != 0: double FMAs, else float.  The paper has no
   counterpart: this measures the arithmetic roofline of the double kernels
   (the outer residual, the coarsest level), which the device's copy
   bandwidth does not bound.  Allocates and frees a small buffer; host
   output; synchronises.  PTP_ECUDA if a CUDA call failed. */
int ptp_probe_fma(int device, int fp64, double* tflops);

/* out[i] = 1/d[i] by the Newton reciprocal of the outer residual kernels
   (two Newton-Raphson steps from the float reciprocal), for testing it
   against the device's double division.  Valid for d in [2^-126, 2^127].
   d and out are DEVICE arrays of n doubles (not the same buffer); stream
   may be NULL (the default stream); synchronises.  The paper has no
   counterpart. */
int ptp_probe_recip_dev(int device, const double* d, double* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PTP_H */
