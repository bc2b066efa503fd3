/*
 * expd.h -- C ABI of the GB300 Exp-ParaDiag library (libexpd.so).
 *
 * Exp-ParaDiag (Garai & Chamakuri, arXiv 2603.04350) solves the all-at-once
 * system of an exponential BDF-s time integrator for u_t = L u + N(u),
 * L = a*Lap - c, on Nt time steps at once:
 *
 *     R_s v = f_s,   R_s = I - sum_{j=1..s} a_j C_{j-1} (x) A^j,  A = exp(dt L_h)
 *
 * (Sec. 3 Eq. (3.1), Sec. 4 Eq. (4.2), Sec. 5 Eqs. (5.2)-(5.8)), with the
 * alpha-circulant preconditioner R_s^alpha (Eq. (3.2), Eq. (4.4)) applied by
 * the three steps of Eq. (3.3) / Eq. (4.5): an alpha-scaled DFT over the time
 * slices, Ns independent shifted spatial solves, and the inverse scaled DFT.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Grids.  1D: n[0] points.  2D: n[0] rows (slow axis) x n[1] columns (fast
 *    axis).  Periodic grids (spectral Laplacian, x_j = j*L/n) need power-of-two
 *    sizes 8..4096; Dirichlet grids (3-/5-point Laplacian on n interior
 *    points, x_j = j*L/(n+1)) accept 2..4096 points per axis.
 *  - Time.  u_0 is the initial value; u_1..u_Nt are the time slices.  For
 *    order s the unknowns are v = (u_s, ..., u_Nt): Ns = Nt - s + 1 slices.
 *    u_1..u_{s-1} are either produced by the ramp (u_j by BDF-j, j < s) or
 *    supplied by the caller (EXPD_STARTUP_GIVEN).
 *  - Arrays.  All arrays are float64, C order, slice-major: a space-time
 *    array is [slices][n0] (1D) or [slices][n0][n1] (2D).  u0 is one slice.
 *    U arguments hold u_1..u_Nt ([Nt] slices); residual and preconditioner
 *    arguments hold the Ns unknown rows ([Ns] slices, row i is time s+i).
 *  - Pointers may be device pointers (cudaMalloc / torch CUDA tensors) or
 *    host pointers; the library detects which with cudaPointerGetAttributes.
 *    Host buffers are staged through plan-owned device buffers with the
 *    copies enqueued on the call's stream, so a call with host buffers
 *    includes its own host<->device traffic.  Device buffers that are not
 *    16-byte aligned (a view starting at an odd element) are staged the same
 *    way, by device-to-device copies, and such a call returns once its
 *    results are in the caller's buffer, as a host-pointer call does.  The caller owns every buffer it
 *    passes; the library never keeps a pointer past the call.
 *  - Streams.  `stream` is a cudaStream_t (NULL = the legacy default
 *    stream).  Device-pointer calls are asynchronous except that solvers
 *    synchronise the stream to read convergence norms; host-pointer calls
 *    return after their results are in host memory.  One call per plan may
 *    be in flight at a time.
 *  - Errors.  Every entry point returns an expd_status; nothing is thrown
 *    across the ABI.  expd_last_error() gives a thread-local message for the
 *    last failure.  Different plans may be used from different host threads
 *    at the same time (plan memory is stream-ordered; kernel launch limits are
 *    set once per process and never lowered).  EXPD_ERR_CUDA means a CUDA call failed (the message names
 *    it); the plan stays valid unless the CUDA context itself is lost.
 */
#ifndef EXPD_H
#define EXPD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EXPD_OK = 0,
    EXPD_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range        */
    EXPD_ERR_OOM = 2,           /* device allocation failed                             */
    EXPD_ERR_NOT_CONVERGED = 3, /* max_iter reached; the last iterate is returned       */
    EXPD_ERR_DIVERGED = 4,      /* update non-finite or 1e3 times the first update      */
    EXPD_ERR_CUDA = 5,          /* a CUDA runtime call failed                           */
    EXPD_ERR_UNSUPPORTED = 6,   /* valid request that this build does not implement     */
    EXPD_ERR_TIMEOUT = 7,       /* the scheme's time limit ran out, or a pipeline wait  */
                                /* inside a kernel gave up (the GPU stays usable)       */
    EXPD_ERR_CANCELLED = 8      /* expd_plan_cancel stopped the call                    */
} expd_status;

/* Boundary conditions and the eigenbasis of L_h they give (Sec. 2 after
 * Eq. (2.7); the Neumann Allen-Cahn experiment of Sec. 7):
 *  PERIODIC   n points x_j = j L/n, spectral Laplacian, the DFT;
 *  DIRICHLET  n interior points x_j = j L/(n+1), 3/5-point Laplacian, the DST-I;
 *  NEUMANN    n cell centres x_j = (j - 1/2) L/n, 3/5-point Laplacian with
 *             mirrored ghost values (zero normal derivative), the DCT-II. */
enum { EXPD_BC_PERIODIC = 0, EXPD_BC_DIRICHLET = 1, EXPD_BC_NEUMANN = 2 };
enum { EXPD_NL_NONE = 0, EXPD_NL_ALLEN_CAHN = 1 };      /* N(u) = 0 or u - u^3          */
enum { EXPD_PREC_FP64 = 0, EXPD_PREC_MIXED = 1 };
enum { EXPD_STARTUP_RAMP = 0, EXPD_STARTUP_GIVEN = 1 };

/* Spatial grid.  ndim is 1 or 2; n[1]/length[1] are ignored for 1D. */
typedef struct {
    int ndim;
    int n[2];
    double length[2];
    int bc;                     /* EXPD_BC_*                                           */
} expd_grid;

/* L = a*Lap - b.grad - c (Sec. 1, Eq. (1.2); the advection term as in the
 * advection-diffusion experiments of Sec. 7 and Remark 3.7) and the
 * nonlinearity N.  b[d] is the velocity along grid axis d (the axis of n[d]);
 * advection needs a periodic grid: its spectral first derivative gives the
 * complex symbol -a|k|^2 - i b.k - c (the Nyquist wavenumber's first-derivative
 * symbol is 0, so real fields stay real).  b = {0, 0} for pure diffusion.
 *
 * Complex states (the Schrodinger equation of Sec. 7: a = i, c = 2i or 200i):
 * with complex_state = 1 the coefficients are a + i a_im and c + i c_im, and
 * every state array of the calls below (u0, f, U, R, S) holds complex values,
 * interleaved (re, im) doubles -- the layout of C99 double _Complex and of
 * complex128 tensors -- so an array of k slices holds 2 k M doubles.  A complex
 * state needs nonlin = EXPD_NL_NONE and the float64 precision (other cases
 * return EXPD_ERR_UNSUPPORTED); GMRES then runs in complex arithmetic
 * (Hermitian inner product, complex Givens rotations).  With complex_state = 0,
 * a_im and c_im must be 0. */
typedef struct {
    double a;
    double c;
    int nonlin;                 /* EXPD_NL_*                                           */
    double b[2];
    double a_im;                /* imaginary part of a (complex_state only)            */
    double c_im;                /* imaginary part of c (complex_state only)            */
    int complex_state;          /* 0: real arrays, 1: complex (interleaved) arrays     */
} expd_operator;

/* Scheme and solver controls.
 *  order      s in 1..6: exponential BDF-s (Eq. (2.2), Eq. (4.1), Sec. 5)
 *  precision  EXPD_PREC_FP64: every transform, the preconditioner and the
 *             residual in float64.  EXPD_PREC_MIXED:
 *             - the fixed point first sweeps entirely in float32 (iterate,
 *               residual, N and its FFTs, preconditioner) until its error
 *               estimate reaches tol or the float32 floor stalls it, then
 *               sweeps with an accurate iterate, residual and N (double-float
 *               on periodic grids, float64 on Dirichlet grids) and the float32
 *               preconditioner, which converge to the float64 fixed point
 *               (Dirichlet grids with a nonlinearity skip the float32 sweeps);
 *             - GMRES and BiCGStab run on the float32 preconditioner too, with
 *               iterative refinement: every time the Krylov recurrence has
 *               reduced its residual by 1e-3, or claims convergence, the
 *               residual f_s - R_s v is recomputed in float64 and
 *               preconditioned, and the method restarts from it; convergence
 *               is declared on that recomputed residual only;
 *             - start-up, right-hand side and output transforms use
 *               double-float arithmetic on periodic grids and float64 on
 *               Dirichlet grids, except that on 2D Dirichlet grids whose sizes
 *               are multiples of 128 up to 1024 (n + 1 not a power of two) the
 *               sine transforms (Sec. 3.1, the eigenbasis of L_h) run on the
 *               tensor cores as split-bf16 products: every row cut into k
 *               7-bit digits, the digit products summed exactly in float32,
 *               the pairs in double-float, k = ceil((3 - log2 tol) / 7) in
 *               3..7, relative error about 2^(-7k).  A pipeline wait of that
 *               kernel that gives up (after 2 s, or at once when the plan is
 *               cancelled) makes the call return EXPD_ERR_TIMEOUT, or
 *               EXPD_ERR_CANCELLED after expd_plan_cancel.
 *  max_iter   iteration cap of the iterative solvers
 *  tol        target L^inf(0,T;L^2) relative error (Sec. 7's norm).  The
 *             fixed point stops when rho/(1-rho) * max_n||s_n|| / max_n||v_n||
 *             <= tol (s the update, rho the observed contraction); GMRES and
 *             BiCGStab stop when sqrt(Ns) times the relative preconditioned
 *             residual is <= tol
 *  gmres_restart  GMRES restart length m (1..64)
 *  startup    EXPD_STARTUP_RAMP or EXPD_STARTUP_GIVEN (u_1..u_{s-1} read
 *             from the first s-1 slices of the U argument of the solvers)
 *  jacobian   EXPD_JAC_LAGGED: the fixed point preconditions with R_s^alpha
 *             (N lagged, Eqs. (7.3)-(7.4)).  EXPD_JAC_MEAN_U0: inexact Newton
 *             steps with the Jacobian at the initial value (proposed after
 *             Eq. (6.5)) averaged over space, i.e. R_s^alpha - beta_s dt nbar I,
 *             nbar = mean of N'(u_0); Step (b) stays diagonal and the fixed
 *             point is unchanged.  Ignored for linear problems.
 *  guess      the fixed point's initial iterate.  EXPD_GUESS_LINEAR (0, the
 *             default): u_n = A^(n-s+1) u_{s-1}, the scheme's own solution
 *             when N = 0 and f = 0 (the BDF coefficients sum to one; Eq. (2.2),
 *             Eq. (4.1)) -- one sweep of the zero start produces it up to the
 *             alpha perturbation, so the iteration needs one sweep fewer.
 *             EXPD_GUESS_ZERO (1): u_n = 0.  The paper runs several initial
 *             guesses (Sec. 7) without fixing one.  GMRES and BiCGStab start
 *             from zero under both.  EXPD_GUESS_GIVEN (2, every solver but the
 *             sequential one): the initial iterate is read from slices
 *             s-1..Nt-1 of the U argument (u_s..u_Nt) -- resuming from a
 *             checkpoint, e.g. the last iterate a call that returned
 *             EXPD_ERR_NOT_CONVERGED, EXPD_ERR_TIMEOUT or EXPD_ERR_CANCELLED
 *             left in U (copied to host memory and back in between, or not).
 *             The stopping tests are the fresh solve's: GMRES and BiCGStab
 *             measure residuals against the zero start's P^{-1} f_s.  No
 *             counterpart in the paper.
 *  kernel_flags  interchangeable kernel variants (each pair computes the same
 *             result; the autotuner chooses among them): EXPD_KF_TIME_SMEM
 *             takes the shared-memory time kernel where the register kernel
 *             would run, EXPD_KF_FFT_RADIX4 the radix-4 shared-memory FFTs
 *             instead of the four-step register FFTs, EXPD_KF_DST_FP64 the
 *             float64 sine-transform products instead of the tensor cores,
 *             EXPD_KF_DST_N64 tensor-core sine-transform tiles of 128 x 64
 *             outputs instead of 128 x 128 (twice the tiles: small grids).
 *             The environment variables EXPD_TIME_KERNEL=smem,
 *             EXPD_FFT_KERNEL=radix4 and EXPD_DST_TC=0, read at plan
 *             creation, set the same flags.  0 = the default kernels.
 *  nl_form    how the nonlinear term enters the scheme: EXPD_NLF_IF (0, the
 *             paper's integrating-factor form, Eq. (6.1), Eq. (7.3)) or
 *             EXPD_NLF_ETD1 (first-order exponential time differencing,
 *             u_n = A u_{n-1} + dt phi_1(dt L) N(u_{n-1}),
 *             phi_1(z) = (e^z - 1)/z, the ETD alternative named at the start
 *             of Sec. 6; order 1 only).  Ignored for linear problems.
 *  time_limit_ms  wall-clock limit of one solver call in milliseconds, checked
 *             between iterations (EXPD_ERR_TIMEOUT when exceeded; the last
 *             iterate is returned); 0 = none.                              */
enum { EXPD_JAC_LAGGED = 0, EXPD_JAC_MEAN_U0 = 1 };
enum { EXPD_GUESS_LINEAR = 0, EXPD_GUESS_ZERO = 1, EXPD_GUESS_GIVEN = 2 };
enum { EXPD_KF_TIME_SMEM = 1, EXPD_KF_FFT_RADIX4 = 2, EXPD_KF_DST_FP64 = 4, EXPD_KF_DST_N64 = 8 };
enum { EXPD_NLF_IF = 0, EXPD_NLF_ETD1 = 1 };
typedef struct {
    int order;
    int precision;
    int max_iter;
    double tol;
    int gmres_restart;
    int startup;
    int jacobian;               /* EXPD_JAC_*                                          */
    int guess;                  /* EXPD_GUESS_*                                        */
    int kernel_flags;           /* EXPD_KF_* bits                                      */
    int nl_form;                /* EXPD_NLF_*                                          */
    double time_limit_ms;       /* 0 = no limit                                        */
} expd_scheme;

#define EXPD_MAX_HISTORY 128

/* Per-solve report.  history[k] is the convergence measure after iteration
 * k+1: the estimated relative error (fixed point) or the relative
 * preconditioned residual (GMRES, BiCGStab; with the mixed precision's
 * refinement, the Krylov recurrence's value, while final_measure is the
 * recomputed one).  The phase times are device times between CUDA events
 * recorded on the call's stream: ms_setup from the start of the call to the
 * start of the first iteration (host-buffer staging, start-up values and their
 * transforms, the right-hand side f_s), ms_iterate for the iterations,
 * ms_output for the inverse transforms and staging of the result; reading them
 * makes the call wait for its stream once more at the end.  A NULL info skips
 * them. */
typedef struct {
    int iterations;
    int fp32_iterations;        /* fixed-point sweeps that evaluated N with float32 FFTs */
    double final_measure;
    double contraction;         /* last observed ratio of successive update norms    */
    double history[EXPD_MAX_HISTORY];
    int refinements;            /* mixed Krylov: residuals recomputed in float64     */
    double ms_setup;
    double ms_iterate;
    double ms_output;
} expd_info;

typedef struct expd_plan_s* expd_plan;

/* Create a plan: validates the problem, allocates all device workspace for it
 * (see expd_plan_workspace_bytes) and builds the spectral tables (the
 * eigenvalues of L_h, exp(dt mu), the alpha-circulant eigenvalues
 * lambda_n = alpha^(1/Ns) e^{2 pi i n/Ns} and Gamma_alpha of Sec. 2, BDF
 * coefficients).  Requires 0 < alpha < 1, dt > 0, order + 1 <= Nt and
 * Nt - order + 1 <= 512 (EXPD_ERR_UNSUPPORTED above: a time column of 8 modes
 * must fit one CTA's shared memory), beta_s*dt < 1 for nonlinear problems.
 * `stream` orders the table uploads.
 * On failure *out is NULL and nothing stays allocated. */
expd_status expd_plan_create(const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                             double alpha, const expd_scheme* scheme, void* stream,
                             expd_plan* out);

/* Device bytes the plan holds (for admission by memory footprint). */
expd_status expd_plan_workspace_bytes(expd_plan plan, size_t* bytes);

/* Device bytes expd_plan_create would allocate for these arguments, computed
 * without allocating anything (admission control before creating a plan).
 * flags adds the buffers a plan allocates on first use: EXPD_FOOTPRINT_SOURCE
 * (a source f is passed), EXPD_FOOTPRINT_HOST (host pointers, or device
 * pointers that are not 16-byte aligned, are passed),
 * EXPD_FOOTPRINT_GMRES (expd_solve_gmres or expd_solve_bicgstab is called). */
enum { EXPD_FOOTPRINT_SOURCE = 1, EXPD_FOOTPRINT_HOST = 2, EXPD_FOOTPRINT_GMRES = 4 };
expd_status expd_plan_footprint_bytes(const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                                      double alpha, const expd_scheme* scheme, int flags, size_t* bytes);

/* Residual of the all-at-once system (Eq. (3.2) right-hand side; for the
 * lagged nonlinear form Eqs. (7.3)-(7.4)):
 *     R = f_s + beta_s dt N(v) - R_s v,
 * where v = U[s-1..Nt-1] (u_s..u_Nt), the startup values are u0 and
 * U[0..s-2], and f_s holds the startup terms and beta_s dt f(t_n).
 *   u0  [1 slice]   f  [Nt slices] or NULL (no source)   U  [Nt slices]
 *   R   [Ns slices] (output)
 * Everything is evaluated in float64. */
expd_status expd_residual(expd_plan plan, const double* u0, const double* f, const double* U,
                          double* R, void* stream);

/* S = (R_s^alpha)^{-1} R by the three steps of Eq. (3.3) / Eq. (4.5):
 * (a) S_a = (F (x) I)(Gamma_alpha (x) I) R, F the unitary DFT with
 * omega = e^{2 pi i/Ns}; (b) per slice S_b,n = (I - sum_j a_j lambda_n^j A^j)^{-1} S_a,n
 * in L_h's eigenbasis; (c) S = (Gamma_alpha^{-1} (x) I)(F^* (x) I) S_b.
 *   R, S  [Ns slices]; R and S may alias.
 * Steps (a)-(c) run in the plan's preconditioner precision (float32 for
 * EXPD_PREC_MIXED); the spatial transforms around them are float64. */
expd_status expd_precond_apply(expd_plan plan, const double* R, double* S, void* stream);

/* Preconditioned fixed-point (Richardson) iteration v^{k+1} = v^k +
 * (R_s^alpha)^{-1}(f_s + beta_s dt N(v^k) - R_s v^k) (Eq. (3.2), Eq. (4.4);
 * lagged N as in Eqs. (7.3)-(7.4)) from the initial iterate the scheme's
 * `guess` selects: by default (EXPD_GUESS_LINEAR) v^0_n = A^(n-s+1) u_{s-1},
 * with EXPD_GUESS_ZERO v^0 = 0, with EXPD_GUESS_GIVEN the iterate in U.
 *   u0 [1 slice]; f [Nt slices] or NULL; U [Nt slices] output u_1..u_Nt
 *   (input for its first s-1 slices when startup = EXPD_STARTUP_GIVEN, for
 *   the others when guess = EXPD_GUESS_GIVEN)
 *   info may be NULL.
 * Returns EXPD_ERR_NOT_CONVERGED (U holds the last iterate) when max_iter
 * sweeps do not reach tol, EXPD_ERR_DIVERGED when an update is non-finite or
 * exceeds 1e3 times the first one (the iteration matrix's spectral radius
 * exceeds 1, e.g. alpha/(1 - alpha) > 1 for slowly decaying modes),
 * EXPD_ERR_TIMEOUT / EXPD_ERR_CANCELLED (U holds the last iterate) when the
 * scheme's time limit ran out or expd_plan_cancel was called. */
expd_status expd_solve_fp(expd_plan plan, const double* u0, const double* f, double* U,
                          expd_info* info, void* stream);

/* Left-preconditioned restarted GMRES(m) on (R_s^alpha)^{-1} R_s v =
 * (R_s^alpha)^{-1} f_s (Sec. 3.2, Theorem 3.3), v^0 = 0, float64 vectors.
 * EXPD_PREC_FP64: classical Gram-Schmidt with one re-orthogonalisation, the
 * float64 preconditioner, restarts every m iterations.  EXPD_PREC_MIXED: the
 * float32 preconditioner, one Gram-Schmidt pass, and a restart from the
 * residual recomputed in float64 whenever a cycle has reduced its residual by
 * 1e-3 or claims convergence (iterative refinement; the float32
 * preconditioner's rounding, about eps32/alpha relative, then limits only how
 * fast the restarts contract, never the accuracy).  Linear problems only
 * (EXPD_ERR_INVALID_ARG otherwise).  Arguments and the time-limit and cancel
 * statuses as expd_solve_fp. */
expd_status expd_solve_gmres(expd_plan plan, const double* u0, const double* f, double* U,
                             expd_info* info, void* stream);

/* Left-preconditioned BiCGStab (van der Vorst's recurrences) on
 * (R_s^alpha)^{-1} R_s v = (R_s^alpha)^{-1} f_s, v^0 = 0, float64 vectors: the
 * short-recurrence alternative to GMRES that Sec. 7 (Table 2) times beside it
 * (two preconditioned operator applications and three reductions per
 * iteration, seven vectors of storage whatever the iteration count).  Stops
 * like expd_solve_gmres; restarts its shadow residual on a breakdown; returns
 * EXPD_ERR_DIVERGED when the residual turns non-finite.  EXPD_PREC_MIXED runs
 * the float32 preconditioner and replaces the recurrence's residual by the one
 * recomputed in float64 (restarting the recurrences) under the same rule as
 * GMRES.  Linear problems only.  Arguments as expd_solve_fp;
 * info->history[k] is the relative preconditioned residual after k
 * iterations. */
expd_status expd_solve_bicgstab(expd_plan plan, const double* u0, const double* f, double* U,
                                expd_info* info, void* stream);

/* Sequential time stepping of the same scheme: u_n = sum_j a_j A^j u_{n-j} +
 * beta_s dt f(t_n) for n = s..Nt, with u_n - beta_s dt N(u_n) solved pointwise
 * by Newton when N is nonzero (Eq. (2.2), Eq. (4.1), Eq. (7.3); with
 * EXPD_NLF_ETD1, u_n = A u_{n-1} + dt phi_1(dt L) N(u_{n-1}) explicitly), in
 * float64, one step after the other on the GPU.  Its result is the exact
 * solution of the all-at-once system that expd_solve_fp and expd_solve_gmres
 * iterate towards (the system is block lower-triangular), so it is both a
 * reference and the time-stepping baseline the parallel-in-time solve is
 * measured against.  Arguments as expd_solve_fp (no info; the plan's
 * precision, tol and max_iter are ignored).  Uses the plan's workspace: not
 * concurrently with another call on the same plan. */
expd_status expd_solve_sequential(expd_plan plan, const double* u0, const double* f, double* U, void* stream);

/* Ask the solver call in flight on this plan -- or, when none is, the plan's
 * next solver call -- to stop at its next iteration boundary (and a
 * tensor-core sine-transform launch in flight to give up its pipeline waits):
 * that call returns EXPD_ERR_CANCELLED with the last iterate in U, and the
 * request is consumed.  Thread-safe: meant to be called from another host
 * thread than the one running the solve. */
expd_status expd_plan_cancel(expd_plan plan);

/* ---- allocation-free preconditioner solve ---------------------------------
 * The paper has no counterpart to this entry point; it is a deployment variant
 * of expd_precond_apply for callers that must not allocate device memory --
 * callers whose device memory is owned by an allocator of their own (a serving
 * engine that reserves the free HBM at start-up, a framework memory pool), or
 * that run where an allocation could fail or stall in the middle of their
 * work.  It takes the plan parameters directly instead of a plan (creating a
 * plan calls cudaMalloc) and computes S = (R_s^alpha)^{-1} R exactly as
 * expd_precond_apply does, with every table and intermediate kept in one
 * fixed device array of EXPD_NOALLOC_SCRATCH_BYTES bytes that each GPU loading
 * the library holds until the process exits.  It calls no cudaMalloc, no
 * cudaFree and no allocating library routine.
 *   R, S   16-byte-aligned device pointers, [Ns slices] as for
 *          expd_precond_apply (may alias); other pointers get
 *          EXPD_ERR_INVALID_ARG (staging them would need memory)
 * Limits: at most 512 unknown slices, and the tables, the eigen-space copy of
 * R, the spatial scratch and the norm partials must fit the array (about
 * 2 Ns M complex values plus the DST matrices on Dirichlet grids); larger
 * problems get EXPD_ERR_INVALID_ARG with the byte count in expd_last_error();
 * an operator with advection (b != 0) gets EXPD_ERR_UNSUPPORTED.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and leave their contents in it: calls that
 * overlap on the GPU (different streams or host threads) race. */
#define EXPD_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
expd_status expd_precond_apply_noalloc(const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                                       double alpha, const expd_scheme* scheme, const double* R, double* S,
                                       void* stream);

/* ---- per-kernel timing -------------------------------------------------------
 * With timing enabled, every libexpd kernel launch of the plan is bracketed by
 * two CUDA events recorded on the stream it is launched on; expd_timing_read
 * waits for those events and reports, per kernel class, the number of timed
 * launches, the summed device time, and the summed algorithmic DRAM bytes and
 * flops the launches are defined to move / perform (the roofline numerators:
 * one read of every input element and one write of every output element).
 * `launches` counts all kernels launched by the plan since the last reset,
 * timed or not.  Timing adds two event records per launch. */
enum {
    EXPD_K_TIME = 0,      /* time kernel, float64 iterate: residual + alpha-scaled DFT +      */
                          /* shifted solves + inverse DFT + update                            */
    EXPD_K_FFT_COL = 1,   /* float64 spatial FFT along the strided axis                       */
    EXPD_K_FFT_ROW = 2,   /* float64 real FFT along the contiguous axis (incl. fused N(u))    */
    EXPD_K_DST = 3,       /* Dirichlet DST-I as a dense matrix product                        */
    EXPD_K_GMRES = 4,     /* GMRES dot products and vector updates                            */
    EXPD_K_POINTWISE = 5, /* pointwise solves, eigen-space combinations, f_s assembly         */
    EXPD_K_REDUCE = 6,    /* per-slice norm reduction                                         */
    EXPD_K_TIME32 = 7,    /* time kernel, float32 iterate (the mixed path's float32 sweeps)   */
    EXPD_K_FFT_COL32 = 8, /* float32 spatial FFT along the strided axis                       */
    EXPD_K_FFT_ROW32 = 9, /* float32 real FFT along the contiguous axis (incl. fused N(u))    */
    EXPD_K_TIMEDD = 10,   /* time kernel, double-float iterate (the mixed path's last sweeps) */
    EXPD_K_FFT_COLDD = 11, /* double-float spatial FFT along the strided axis                */
    EXPD_K_FFT_ROWDD = 12, /* double-float real FFT along the contiguous axis                */
    EXPD_K_DST_TC = 13,   /* Dirichlet DST-I on the tensor cores: split-BF16 digit products   */
    EXPD_K_DST_SPLIT = 14, /* Dirichlet DST-I on the tensor cores: rows cut into bf16 digits  */
    EXPD_K_TIME_TC = 15,  /* time kernel on the tensor cores (real columns, float32           */
                          /* preconditioner, float64 iterate; Steps (a), (c) as products)     */
    EXPD_NUM_KCLASS = 16
};

typedef struct {
    long long launches;
    int count[EXPD_NUM_KCLASS];
    double ms[EXPD_NUM_KCLASS];
    double bytes[EXPD_NUM_KCLASS];
    double flops[EXPD_NUM_KCLASS];
} expd_timing;

/* Turn per-launch event timing on (1) or off (0) for the plan. */
expd_status expd_timing_enable(expd_plan plan, int enable);

/* Report the accumulated timing; reset = 1 clears it afterwards. */
expd_status expd_timing_read(expd_plan plan, expd_timing* out, int reset);

/* Release the plan and all its device memory.  NULL is accepted. */
expd_status expd_destroy(expd_plan plan);

/* Static text for a status code. */
const char* expd_status_string(expd_status s);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* expd_last_error(void);

/* Library ABI version (major*10000 + minor*100 + patch). */
int expd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EXPD_H */
