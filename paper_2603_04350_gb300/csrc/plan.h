// Internal plan object and the host-side launchers shared by the .cu files.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <atomic>
#include <chrono>
#include <string>
#include <utility>
#include <vector>

#include "expd.h"

// Largest supported sizes (shared memory per warp-FFT column).
#define EXPD_MAX_PERIODIC_N 4096
#define EXPD_MAX_DIRICHLET_N 4096
// Unknown slices per plan: a time column (Ns values, or the Bluestein length
// L <= 1024 for Ns <= 512) of 8 modes sits in one CTA's shared memory in float64
#define EXPD_MAX_NS 512
#define EXPD_TIME_COLS 8  // time-direction columns (spatial modes) per CTA

expd_status expd_cuda_fail(cudaError_t e, const char* what, const char* file, int line);
expd_status expd_fail(expd_status s, const std::string& msg);
// Clears this thread's expd_last_error() message (at the start of an entry point).
void expd_clear_error();
struct expd_plan_s;
// Validate the problem and fill the plan's scalar fields (no allocation).
expd_status plan_init_fields(expd_plan_s* p, const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                             double alpha, const expd_scheme* scheme);
bool expd_is_device_ptr(const void* ptr);

// Time-direction tables in one precision (t64: double, t32: float).
struct TimeTables {
    int L = 0, log2L = 0, bluestein = 0;
    void* gam = nullptr;      // [Ns]   Gamma_alpha: alpha^(n/Ns)
    void* osc = nullptr;      // [Ns]   output scale 1/(Ns alpha^(n/Ns)), times 1/L^2 for Bluestein
    void* lam = nullptr;      // [Ns]   lambda_n = alpha^(1/Ns) e^{2 pi i n/Ns}
    void* tw = nullptr;       // [L/2]  e^{-2 pi i k/L}
    void* chirp = nullptr;    // [Ns]   e^{+pi i n^2/Ns}           (Bluestein)
    void* bplus = nullptr;    // [L]    FFT_L of conj-chirp kernel, bit-reversed order
    void* bminus = nullptr;   // [L]    FFT_L of chirp kernel, bit-reversed order
};

// State of the device-controlled fixed point (the stopping test of the
// host loop, run by one warp after every sweep); read back once per solve.
struct LoopCtl {
    int it, it32, result, phys_valid;
    int pad[4];
    double prev, rho, rho_phase, measure, s_first, last_rel;
    double history[EXPD_MAX_HISTORY];
};
constexpr size_t EXPD_CTL_DOUBLES = sizeof(LoopCtl) / sizeof(double);
static_assert(sizeof(LoopCtl) % sizeof(double) == 0, "loop state in whole doubles");

struct expd_plan_s {
    // ---- problem ----------------------------------------------------------
    int ndim = 1, NX = 1, NY = 1;  // NX fast axis, NY slow axis (1 for 1D)
    int bc = EXPD_BC_PERIODIC;
    double LX = 1, LY = 1;
    double a = 0, c = 0;
    double a_im = 0, c_im = 0;  // imaginary parts of a and c (complex states)
    int cplx = 0;           // complex state: interleaved complex physical slices, full spectrum
    double bx = 0, by = 0;  // advection velocity along NX / NY
    int adv = 0;            // complex symbol (advection, or imaginary a or c): complex E and coefficient tables
    int nonlin = EXPD_NL_NONE;
    double dt = 0;
    int Nt = 0, order = 1, Ns = 0;
    double alpha = 0;
    int precision = EXPD_PREC_FP64, max_iter = 50, restart = 20, startup = EXPD_STARTUP_RAMP;
    double tol = 1e-8;
    int kernel_flags = 0;     // EXPD_KF_* (from the scheme and the environment)
    int nl_form = EXPD_NLF_IF;
    double time_limit_ms = 0; // 0: no limit
    double acoef[7][7] = {};  // acoef[q][j]: a_j of BDF-q, j = 1..q
    double beta[7] = {};      // beta_q

    // ---- layout -------------------------------------------------------------
    long long M = 0;     // physical points per slice
    long long Mp = 0;    // doubles per physical slice: M, or 2 M for a complex state
    int KX = 0;          // periodic: NX/2+1 complex per row; Dirichlet or complex state: NX per row
    long long Mcol = 0;  // time columns per slice (complex modes or real modes)
    int realcol = 0;     // 1 for Dirichlet grids with a real state (real eigen-coefficients)
    size_t esz = 16;     // bytes per eigen element (16 complex, 8 real)

    // ---- tables ---------------------------------------------------------------
    double* E = nullptr;       // [Mcol] exp(dt mu_m)
    double* PHI64 = nullptr;   // ETD1: [Mcol] dt phi_1(dt mu_m), phi_1(z) = (e^z - 1)/z
    float* PHI32 = nullptr;    // the same in float32
    void* PHIdd = nullptr;     // the same as double-float (mixed periodic plans)
    double* C64 = nullptr;     // [order][Mcol] a_j exp(j dt mu_m), j = 1..order (time-kernel coefficients)
    float* C32 = nullptr;      // the same in float32
    double2* Wx64 = nullptr;   // [NX/2+1] e^{-2 pi i k/NX}
    float2* Wx32 = nullptr;
    double2* Wy64 = nullptr;   // [NY/2]   e^{-2 pi i k/NY}
    float2* Wy32 = nullptr;
    void* Wxdd = nullptr;      // double-float copies of Wx / Wy (dd2)
    void* Wydd = nullptr;
    void* Cdd = nullptr;       // [order][Mcol] double-float coefficients (dd)
    void* gamdd = nullptr;     // [Ns] Gamma_alpha as double-float
    void* oscdd = nullptr;     // [Ns] output scale as double-float
    double* Sx = nullptr;      // Dirichlet: [NX][NX] orthonormal DST-I matrix (dense path)
    double* Sy = nullptr;      // Dirichlet: [NY][NY]
    double* SxT = nullptr;     // Neumann: [NX][NX] inverse-transform operand (Sx is the forward one)
    double* SyT = nullptr;     // Neumann: [NY][NY]
    int fast_dst = 0;          // Dirichlet with n + 1 a power of two: FFT-based sine transforms
    double2* Dtx = nullptr;    // fast DST twiddles exp(-2 pi i k / (2 (NX + 1))), k <= NX
    double2* Dty = nullptr;    // the same for NY
    // Dirichlet dense sizes on the mixed path: split-BF16 tensor-core products
    int tc_dst = 0;            // the dense DST runs on the tensor cores (dst_tc.cu)
    int tc_nsl = 0;            // 7-bit digits per value
    int tc_fold = 0;           // products over the symmetric half of S (S[j][n-1-k] = (-1)^j S[j][k])
    int tc_chunk = 0;          // slices transformed per pass
    int tc_eSx = 0, tc_eSy = 0;  // exponents of the S_x and S_y digits (|S| < 2^e)
    uint16_t* tc_S = nullptr;  // packed digit slices of S_x then S_y
    uint16_t* tc_pack = nullptr;  // packed digit slices of the rows being transformed
    int* tc_ex = nullptr;      // row exponents: [NX + NY] unused, rows [tc_chunk * max(NX, NY)]
    int* tc_err = nullptr;     // set by the kernel when a pipeline wait gave up
    TimeTables t64, t32;

    // ---- state --------------------------------------------------------------
    void* Uh = nullptr;        // [Ns][Mcol] iterate in L_h's eigenbasis
    void* Fh = nullptr;        // [Ns][Mcol] known right-hand side f_s
    void* Sh = nullptr;        // [order][Mcol] startup values u_0..u_{s-1}
    void* fh = nullptr;        // [Nt][Mcol] transformed source (lazy)
    void* NL64 = nullptr;      // [Ns][Mcol] N(v) transformed, float64
    void* NL32 = nullptr;      // [Ns][Mcol] N(v) transformed, float32 (mixed)
    void* work64 = nullptr;    // [Ns][NY][KX] double2 / physical scratch
    void* work32 = nullptr;    // [Ns][NY][KX] float2 (mixed nonlinear)
    void* U32 = nullptr;       // [Ns][Mcol] float32 iterate of the mixed path's float32 sweeps
    void* F32 = nullptr;       // [Ns][Mcol] float32 copy of Fh
    double* startphys = nullptr;  // [order][M] physical u_0..u_{s-1}
    double2* partial = nullptr;   // [Ns][time grid] per-slice norm partials
    double* redout = nullptr;     // [8 + 2 Ns]: per-slice totals (||res_n||^2, ||X_n||^2) from [8] (device)
    double* redhost = nullptr;    // [2 Ns] pinned host copy of the per-slice totals
    cudaStream_t stream = nullptr; // stream of the most recent call: allocations and frees are ordered on it
    int pooled = 0;               // device supports stream-ordered allocation
    int time_grid = 0;            // CTAs of the time kernel (multiple of SM count)
    int partial_cap = 0;          // CTAs the partial-norm buffer has room for
    int time_grid_used = 0;       // CTAs of the last time-kernel launch (for the reduction)
    int dots_fused = 0;           // the last time-kernel launch produced the requested Krylov partials
    int jacobian = 0;             // EXPD_JAC_*
    int guess = 0;                // EXPD_GUESS_*: the fixed point's initial iterate
    int f_slices = 0;             // leading slices of the right-hand side Fh / F32 that can be nonzero
    // One sweep of the fixed point (N evaluation, time kernel, per-slice
    // reduction) per phase, captured as a CUDA graph on first use and relaunched
    // every iteration; keyed by the per-call values the launches bake in.
    struct SweepGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key_ptr = nullptr;
        double key_shift = 0;
        int key_fs = 0;  // right-hand side slices baked into the time kernel's launch
        long long launches = 0;
        int eager = 0;  // sweeps launched directly (the first one sets kernel attributes)
    } sweep_graph[5];             // [0..2] fixed-point phases, [3] sequential stepping,
                                  // [4] double-float sweeps after the first
    // The whole fixed point as one graph: initialisation, a device-controlled
    // loop over float32 sweeps, the conversion, a loop over accurate sweeps
    // (conditional while-nodes; the stopping test runs on the GPU).
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        const void* key_ptr = nullptr;
        double key_shift = 0;
        int key_fs = 0, two = 0;
        long long l_init = 0, l_body1 = 0, l_between = 0, l_body2 = 0;
    } loop_graph;
    int no_device_loop = 1;       // 0: stopping test on the GPU (EXPD_DEVICE_LOOP=1)
    double** phys_slot = nullptr; // device: destination of the physical iterate (in the norms buffer)
    double* phys_slot_value = nullptr;  // what phys_slot holds (rewritten only when it changes)
    double* redhost_dev = nullptr;      // redhost as the GPU addresses it (mapped pinned memory)
    long long fp_solves = 0;      // fixed-point solves run on this plan
    int no_graphs = 0;            // 1: launch kernel by kernel (EXPD_GRAPHS=0)
    int poison = 0;               // 1: fill every new device buffer with NaN bytes (EXPD_POISON=1)
    int canary = 0;               // 1: guard words after every workspace buffer, checked after each call (EXPD_CANARY=1)
    std::vector<std::pair<void*, size_t>> canaries;  // (buffer, its usable bytes) of the guarded buffers
    unsigned long long nvtx_phase = 0;  // the open NVTX range of a solver call's phase (0: none)
    int no_cplx_time = 0;         // 1: complex columns take the generic time kernel (EXPD_TIME_CPLX=0)
    int no_reg_time = 0;          // 1 forces the shared-memory time kernel (tests)
    int no_real_time = 0;         // 1: real columns take the generic kernel (EXPD_TIME_REAL=0, tests)
    int no_tc_time = 0;           // 1: real columns keep the FFT time kernels (EXPD_TIME_TC=0)
    void* tt_tab = nullptr;       // tensor-core time kernel: DFT matrices as fp16 digits and tables (time_tc.cu)
    int* tt_err = nullptr;        // its error word (a wait on an MMA gave up)
    int no_fft4 = 0;              // 1 forces the radix-4 shared-memory row / column FFTs (tests)
    // mixed Krylov refinement: a cycle ends once its residual fell by this factor
    double krylov_eta = 1e-3;
    // ---- cancellation and time limit (expd_plan_cancel, expd_scheme.time_limit_ms) ----
    std::atomic<int> cancel_req{0};  // set by expd_plan_cancel, consumed by the call it stops
    volatile int* cancel_host = nullptr;  // mapped pinned word the tensor-core kernel polls
    const int* cancel_dev = nullptr;      // the same word as the GPU addresses it
    int call_cancelled = 0;       // the running call consumed a cancel request
    std::chrono::steady_clock::time_point call_t0;
    // ---- per-phase device times of a solver call (expd_info.ms_*) ----
    cudaEvent_t phase_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // host-pointer staging (lazy)
    double* stage = nullptr;      // [(2*Nt + 1) * M]
    size_t stage_elems = 0;
    // GMRES basis (lazy)
    void* gm = nullptr;           // Krylov vectors (GMRES basis or BiCGStab vectors) + dot partials
    int gm_vecs = 0;              // vectors of length eigen_elems the block holds

    size_t bytes = 0;             // device bytes held
    int sm_count = 0;

    // ---- per-kernel timing (expd_timing_enable / expd_timing_read) ----
    int timing = 0;
    long long launches = 0;
    struct KRec {
        int cls, e0;
        double bytes, flops;
    };
    std::vector<cudaEvent_t> events;
    std::vector<KRec> recs;
    size_t ev_used = 0;
};

// Brackets one kernel launch: counts it and, with timing on, records events
// around it on the launch stream.
// Device memory of a plan: stream-ordered (cudaMallocAsync / cudaFreeAsync on
// the plan's stream), so creating and destroying plans while other streams
// compute does not synchronise the device.  plan_malloc returns once the
// allocation is usable from any stream.
cudaError_t plan_malloc(expd_plan p, void** ptr, size_t bytes);
void plan_free(expd_plan p, void* ptr);
// Makes s the plan's stream; work still queued on the previous one finishes first.
cudaError_t plan_bind_stream(expd_plan p, cudaStream_t s);

// Raises a kernel's dynamic shared-memory limit to the device's opt-in
// maximum, once per kernel and never lowering it: plans used from several host
// threads launch the same kernels with different sizes, and a per-launch limit
// set by one thread would undercut another thread's launch.  Fails for
// requests above the device maximum.
cudaError_t smem_allow(const void* kern, size_t smem);

// Debug aid (EXPD_CANARY=1): reports EXPD_ERR_CUDA when a guard word after a
// workspace buffer was overwritten (a write past the buffer's end).
expd_status canary_check(expd_plan p, cudaStream_t s);

struct KProf {
    expd_plan p;
    cudaStream_t s;
    int cls, e0 = -1;
    double bytes, flops;
    KProf(expd_plan p_, cudaStream_t s_, int cls_, double bytes_, double flops_ = 0.0);
    ~KProf();
};

// ---- spatial transforms (spatial.cu) ----------------------------------------
// physical [nslices][NY][NX] float64 <-> eigen [nslices][Mcol], float64.
expd_status spatial_forward64(expd_plan p, const double* phys, void* eig, int nslices, cudaStream_t s);
expd_status spatial_inverse64(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s);
// the same with double-float arithmetic (periodic grids with double-float
// tables; otherwise the float64 transforms)
expd_status spatial_forward_dd64(expd_plan p, const double* phys, void* eig, int nslices, cudaStream_t s);
expd_status spatial_inverse_dd64(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s);
// out = transform of N(inverse transform of Uh) for the Ns unknown slices, in
// float32 (f32 = 1, out is float2/float) or float64; Uh is float32 when in32.
expd_status nonlinear_eval(expd_plan p, const void* Uh, void* out, int f32, cudaStream_t s, int in32 = 0);
// elementwise precision conversion of n values (double <-> float)
expd_status convert_f64_to_f32(expd_plan p, const double* in, float* out, long long n, cudaStream_t s);
expd_status convert_f32_to_f64(expd_plan p, const float* in, double* out, long long n, cudaStream_t s);
// double-float ("dd", float hi + float lo) helpers of the mixed path's accurate phase
expd_status convert_f64_to_dd_inplace(expd_plan p, double* a, long long n, cudaStream_t s);
expd_status convert_f32_to_dd(expd_plan p, const float* in, void* out, long long n, cudaStream_t s);
// phys_slot (optional): device memory holding where the physical rows before
// N go (float64 [Ns][NY][NX]); the pointer is read by the kernel, so a captured
// sweep serves any destination
// The fixed point's initial iterate X (float32 when x32, else float64, eigen
// layout): X_k = E^(k+1) S_{s-1}, the last start-up slice propagated by A.
expd_status linear_guess(expd_plan p, void* X, int x32, cudaStream_t s);
// x32: Uh is the float32 iterate (exact in double-float)
expd_status nonlinear_eval_dd(expd_plan p, const void* Uh, void* out, cudaStream_t s, double* const* phys_slot = nullptr,
                              int x32 = 0);
// phys += inverse transform of a float32 half-spectrum [Ns][NY][KX] (float32
// four-step kernels; periodic grids with NX in 32..2048, NY in 16..1024)
bool inverse32_accum_supported(expd_plan p);
expd_status spatial_inverse32_accum(expd_plan p, const void* eig, double* phys, cudaStream_t s);
expd_status spatial_inverse_dd(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s);
// u = solution of u - bdt N(u) = w, pointwise (float64 physical).
expd_status pointwise_solve(expd_plan p, const double* w, double* u, long long n, double bdt, cudaStream_t s);
// out[m] = sum_{j=1..q} coef[j] E_m^j in[j][m] + g * src[m]   (eigen arrays)
expd_status eigen_combine(expd_plan p, void* out, const void* const* in, const double* coef, int q,
                          const void* src, double g, cudaStream_t s);
// f_s: Fh[i] = bdt f^(s+i) + sum_{j: s+i-j<s} a_j E^j Sh[s+i-j]
// *out_dev = sum of x[i]^2 (deterministic); scratch holds 64 doubles
expd_status sum_squares(expd_plan p, const double* x, long long n, double* out_dev, double* scratch, cudaStream_t s);
// F32 (optional): also the float32 copy; fh_dd: Fh stored as double-float pairs;
// nl0 (ETD1): N(u_0) in the eigenbasis, whose phi-scaled value row 0 gains
expd_status assemble_rhs(expd_plan p, const void* fh, cudaStream_t s, float* F32 = nullptr, int fh_dd = 0,
                         const void* nl0 = nullptr);
// ETD1: NL_n <- dt phi_1(dt mu) NL_{n-1}, NL_0 <- 0, in place (kind 0 float64,
// 1 float32, 2 double-float storage)
expd_status etd_shift(expd_plan p, void* NL, int kind, cudaStream_t s);
// ETD1 step: out = E prev + dt phi_1(dt mu) nl (float64 eigen slices)
expd_status etd_step(expd_plan p, void* out, const void* prev, const void* nl, cudaStream_t s);
// out = N(u) pointwise (physical float64)
expd_status nonlinearity_eval_phys(expd_plan p, const double* u, double* out, long long n, cudaStream_t s);

// ---- tensor-core DST (dst_tc.cu) ----------------------------------------------
// The mixed path on a 2D Dirichlet grid with both sizes multiples of 128 up to
// 1024 (and n + 1 not a power of two) transforms with split-BF16 products on
// the tensor cores; EXPD_DST_TC=0 keeps the float64 products.
bool dst_tc_eligible(expd_plan p);
void dst_tc_layout(expd_plan p);     // digit count (from tol) and slices per pass
size_t dst_tc_bytes(expd_plan p);    // device bytes dst_tc_setup allocates
expd_status dst_tc_setup(expd_plan p, cudaStream_t s);  // needs Sx, Sy on the device
// Y[s] = S_y X[s] S_x, ns slices; tmp holds tc_chunk slices of M doubles
expd_status dst2_tc(expd_plan p, const double* X, double* Y, int ns, double* tmp, cudaStream_t s);
expd_status dst_tc_check(expd_plan p, cudaStream_t s);

// ---- time direction (time_kernel.cu) -----------------------------------------
struct TimeOp {
    const void* X = nullptr;   // state / operand in the eigenbasis (may be null)
    const void* F = nullptr;   // additive right-hand side (may be null)
    const void* NL = nullptr;  // transformed nonlinearity (may be null)
    void* sout = nullptr;      // optional copy of the update s in float32 (accum mode)
    double dshift = 0;         // Step (b) solves with (1 - dshift) I - sum_j a_j (lambda A)^j
    int f_slices = -1;         // F is zero beyond its first f_slices slices (-1: all may be nonzero)
    int nl_f32 = 0;
    double bdt = 0;            // coefficient of NL
    double sigR = -1;          // coefficient of R_s X
    int precond = 1;           // apply (R_s^alpha)^{-1} to the combination
    int accum = 0;             // X += result (X must be writable) instead of out = result
    void* out = nullptr;
    int f32 = 0;               // preconditioner precision (steps (a)-(c))
    int st32 = 0;              // X, F, NL, out and the residual arithmetic in float32
    int stdd = 0;              // X, F, NL, out and the residual arithmetic in double-float
    const void* X32 = nullptr; // double-float accumulation: read the iterate from this float32 array
                               // (exact in double-float) and write X + s to X (register kernel)
    int dots = 0;              // Krylov: per-slice partials (||out||^2, <X, out>) for time_reduce,
                               // where the kernel taken supports them (p->dots_fused tells)
};
expd_status time_apply(expd_plan p, const TimeOp& op, cudaStream_t s);
// Tensor-core time kernel (time_tc.cu): real columns, float32 preconditioner on
// float64 storage, Ns <= 128.  Eligibility, the device bytes of its tables,
// their construction (at plan creation) and the launch.
bool time_tc_eligible(expd_plan p);
size_t time_tc_bytes(expd_plan p);
expd_status time_tc_setup(expd_plan p, cudaStream_t s);
// The register time kernel serves this plan's window (Ns in {16, 32, 64}).
bool time_reg_usable(expd_plan p);
// per-slice totals of the time kernel's CTA partials into redout[8..]:
// (||res_n||^2, ||X_n||^2) per slice n (weighted eigen norms), fixed order.
expd_status time_reduce(expd_plan p, cudaStream_t s);
expd_status time_tables_build(expd_plan p, cudaStream_t s);
// CTAs of the time kernel: SM count x resident CTAs, at most the tile count (no allocation)
expd_status time_grid_for(expd_plan p, int* grid);
void time_tables_free(expd_plan p);

// ---- GMRES vector kernels (gmres.cu) ---------------------------------------------
// weighted dot products h[i] = <V_i, w> for i < k (V_i = basis column i), deterministic
expd_status gm_dots(expd_plan p, const double* V, long long ld, int k, const double* w, double* h_dev,
                    cudaStream_t s);
// w -= sum_i h[i] V_i
expd_status gm_update(expd_plan p, const double* V, long long ld, int k, const double* h_dev, double* w,
                      cudaStream_t s);
// w = scale (w - sum_i c[i] V_i) and h_dev[0] = the weighted ||w||^2 of the result, in one pass
expd_status gm_update_norm(expd_plan p, const double* V, long long ld, int k, const double* c_dev, double scale,
                           double* w, double* h_dev, cudaStream_t s);
// y = a*x + b*y  (plain elementwise)
expd_status gm_axpby(expd_plan p, long long n, double a, const double* x, double b, double* y, cudaStream_t s);
// complex states: Hermitian dot products (re, im pairs) and complex multi-axpy
expd_status gm_cdots(expd_plan p, const double* V, long long ld, int k, const double* w, double* h_dev,
                     cudaStream_t s);
expd_status gm_cupdate(expd_plan p, const double* V, long long ld, int k, const double* h_dev, double* x,
                       cudaStream_t s);
long long eigen_elems(expd_plan p);  // doubles per space-time eigen vector
