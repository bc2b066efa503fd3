// C ABI of libexpd: plans, the fixed-point and GMRES solvers, and the residual
// and preconditioner entry points (declared and documented in include/expd.h).
//
// A solve runs entirely in L_h's eigenbasis:
//   1. u0 (and the source f) go to the eigenbasis; the startup values
//      u_1..u_{s-1} come from the ramp (BDF-j, j < s) or from the caller;
//   2. the known right-hand side f_s is assembled (startup terms a_j A^j u_{n-j}
//      with n-j < s, plus beta_s dt f(t_n));
//   3. Richardson sweeps (Eq. (3.2) / Eq. (4.4)) or GMRES (Sec. 3.2) run on the
//      Ns unknown slices; a nonlinear sweep first evaluates N at the iterate
//      through the spatial FFTs (lagged form, Eqs. (7.3)-(7.4));
//   4. the unknown slices return to physical space.
#include <math.h>
#include <math_constants.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <complex>
#include <mutex>
#include <cstdint>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "plan.h"
#include "time_column.cuh"

namespace {

thread_local std::string g_err;

const int64_t kMaxSlices = 1 << 20;

struct Rational {
    int64_t n, d;
};
int64_t gcd64(int64_t a, int64_t b) {
    if (a < 0) a = -a;
    if (b < 0) b = -b;
    while (b) {
        int64_t t = a % b;
        a = b;
        b = t;
    }
    return a ? a : 1;
}
Rational rnorm(int64_t n, int64_t d) {
    if (d < 0) {
        n = -n;
        d = -d;
    }
    const int64_t g = gcd64(n, d);
    return {n / g, d / g};
}
Rational radd(Rational a, Rational b) { return rnorm(a.n * b.d + b.n * a.d, a.d * b.d); }
Rational rdiv(Rational a, Rational b) { return rnorm(a.n * b.d, a.d * b.n); }

// BDF-q: sum_{i=1..q} (1/i) (1 - z)^i = sum_j c_j z^j, normalised to
// u_n - sum_j a_j u_{n-j} = beta dt f_n (Eq. (4.1), Eqs. (5.1)-(5.7)).
void bdf(int q, double* a, double* beta) {
    Rational c[7];
    for (int j = 0; j < 7; ++j) c[j] = {0, 1};
    for (int i = 1; i <= q; ++i) {
        int64_t binom = 1;
        for (int j = 0; j <= i; ++j) {
            c[j] = radd(c[j], rnorm((j % 2 ? -1 : 1) * binom, i));
            binom = binom * (i - j) / (j + 1);
        }
    }
    *beta = (double)c[0].d / (double)c[0].n;
    a[0] = 0.0;
    for (int j = 1; j <= q; ++j) {
        const Rational r = rdiv(c[j], c[0]);
        a[j] = -(double)r.n / (double)r.d;
    }
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Whether a caller's buffer goes through the plan's staging buffers: host
// memory, and device memory that is not 16-byte aligned (a view starting at
// an odd element: the kernels read 16-byte vectors and copy 16-byte-aligned
// rows in bulk, so they see only aligned buffers)
bool needs_stage(const void* ptr) {
    return !is_device_ptr(ptr) || (reinterpret_cast<uintptr_t>(ptr) & 15u) != 0;
}

// Pinned host words for the per-sweep norm read-back, handed out from one
// process-wide arena (freeing pinned memory would synchronise the device).
std::mutex g_pin_mu;

// Blocks of 2^c doubles (c >= 3), carved from pinned chunks that are never
// freed; released blocks return to their size class's free list.
std::vector<double*> g_pin_class[24];

double* pinned_acquire(size_t ndoubles) {
    int c = 3;
    while (((size_t)1 << c) < ndoubles) ++c;
    if (c >= 24) return nullptr;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    std::vector<double*>& fl = g_pin_class[c];
    if (fl.empty()) {
        const size_t block = (size_t)1 << c;
        const size_t count = std::max<size_t>(1, ((size_t)64 << 10) / (block * sizeof(double)));
        double* chunk = nullptr;
        if (cudaMallocHost(&chunk, count * block * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (size_t i = count; i-- > 0;) fl.push_back(chunk + i * block);
    }
    double* r = fl.back();
    fl.pop_back();
    return r;
}

// pinned words of a plan: per-slice norm totals, the device loop's state, one
// spare, and the cancel flag
size_t pinned_words(const expd_plan_s* p) { return 2 * (size_t)p->Ns + EXPD_CTL_DOUBLES + 2; }

// Spatial-transform scratch: one complex value per mode and slice; a complex
// state on a Dirichlet grid splits chunks of max(1, Ns/4) slices into real
// and imaginary parts and needs 8 M doubles per slice of a chunk.
// Eigenvalue of the 3-point (1D) / 5-point (2D) Laplacian on mode (kx, ky):
// Dirichlet -(4/h^2) sin^2(pi (k+1) h/(2L)) with h = L/(n+1) (sine modes
// k + 1 = 1..n); Neumann -(4/h^2) sin^2(pi k/(2n)) with h = L/n (cosine modes
// k = 0..n-1 on the cell centres).
double fd_laplacian_symbol(const expd_plan_s* p, int kx, int ky) {
    auto one = [&](int k, int n, double L) {
        if (p->bc == EXPD_BC_NEUMANN) {
            const double h = L / n, sn = sin(M_PI * k / (2.0 * n));
            return -(4.0 / (h * h)) * sn * sn;
        }
        const double h = L / (n + 1), sn = sin(M_PI * (k + 1) * h / (2.0 * L));
        return -(4.0 / (h * h)) * sn * sn;
    };
    double lap = one(kx, p->NX, p->LX);
    if (p->ndim == 2) lap += one(ky, p->NY, p->LY);
    return lap;
}

size_t work64_bytes(const expd_plan_s* p) {
    const size_t slices = (p->cplx && p->bc != EXPD_BC_PERIODIC) ? (size_t)std::max(p->Ns, 4) : (size_t)p->Ns;
    return slices * p->NY * p->KX * sizeof(double2);
}

void pinned_release(double* q, size_t ndoubles) {
    if (!q) return;
    int c = 3;
    while (((size_t)1 << c) < ndoubles) ++c;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_class[c].push_back(q);
}

// guard words after a buffer (EXPD_CANARY=1): 256 bytes of this pattern
constexpr size_t CANARY_BYTES = 256;
constexpr unsigned char CANARY_BYTE = 0xA5;

expd_status dalloc(expd_plan p, void** ptr, size_t bytes, const char* what) {
    *ptr = nullptr;
    if (bytes == 0) return EXPD_OK;
    cudaError_t e = plan_malloc(p, ptr, bytes + (p->canary ? CANARY_BYTES : 0));
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return expd_fail(EXPD_ERR_OOM, std::string("cudaMalloc failed for ") + what + " (" +
                                            std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
    p->bytes += bytes;
    if (p->canary) {
        e = cudaMemsetAsync(static_cast<char*>(*ptr) + bytes, CANARY_BYTE, CANARY_BYTES, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMemsetAsync(canary)", __FILE__, __LINE__);
        p->canaries.emplace_back(*ptr, bytes);
    }
    // debugging aid: all-ones bytes are a NaN in every floating type, so a
    // read of a buffer before it is written turns the result non-finite
    if (p->poison) {
        e = cudaMemsetAsync(*ptr, 0xFF, bytes, p->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMemsetAsync(poison)", __FILE__, __LINE__);
    }
    return EXPD_OK;
}

// the kernel classes of expd_timing, for the NVTX range of each launch
const char* kclass_name(int c) {
    static const char* names[EXPD_NUM_KCLASS] = {"time", "fft_col", "fft_row", "dst", "gmres",
                                                 "pointwise", "reduce", "time32", "fft_col32", "fft_row32",
                                                 "timedd", "fft_coldd", "fft_rowdd", "dst_tc", "dst_split", "time_tc"};
    return c >= 0 && c < EXPD_NUM_KCLASS ? names[c] : "expd";
}

// NVTX ranges of a solver call's phases (set-up, iterations, output): one
// open range per plan, ended when the next phase starts or the call ends
void nvtx_phase(expd_plan p, const char* name) {
    if (p->nvtx_phase) nvtxRangeEnd((nvtxRangeId_t)p->nvtx_phase);
    p->nvtx_phase = name ? (unsigned long long)nvtxRangeStartA(name) : 0ull;
}

template <typename T>
expd_status upload_vec(expd_plan p, T** dptr, const std::vector<T>& h, const char* what, cudaStream_t s) {
    expd_status st = dalloc(p, reinterpret_cast<void**>(dptr), h.size() * sizeof(T), what);
    if (st != EXPD_OK) return st;
    EXPD_CUDA_TRY(cudaMemcpyAsync(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    return EXPD_OK;
}

void free_plan(expd_plan p) {
    if (!p) return;
    void* bufs[] = {p->E,    p->PHI64, p->PHI32, p->PHIdd, p->C64,  p->C32, p->Cdd, p->Wxdd, p->Wydd, p->gamdd, p->oscdd, p->Wx64, p->Wx32,   p->Wy64,    p->Wy32,    p->Sx,        p->Sy, p->SxT, p->SyT, p->Dtx, p->Dty,
                    p->Uh,   p->Fh,   p->Sh,     p->fh,      p->NL64,    p->NL32,      p->work64,
                    p->work32, p->startphys, p->partial, p->redout, p->stage, p->gm, p->U32, p->F32,
                    p->tc_S, p->tc_pack, p->tc_ex, p->tt_tab};
    for (void* b : bufs) plan_free(p, b);
    for (auto& g : p->sweep_graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (p->loop_graph.exec) cudaGraphExecDestroy(p->loop_graph.exec);
    pinned_release(p->redhost, pinned_words(p));
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    for (cudaEvent_t e : p->phase_ev)
        if (e) cudaEventDestroy(e);
    time_tables_free(p);
    delete p;
}

// ---- staging of host pointers ------------------------------------------------
struct Staging {
    const double* u0 = nullptr;
    const double* f = nullptr;
    double* U = nullptr;        // device view of the U argument
    double* U_host = nullptr;   // non-null when U is host memory
    size_t U_slices = 0;
};

expd_status ensure_stage(expd_plan p) {
    if (p->stage) return EXPD_OK;
    p->stage_elems = (size_t)(2 * p->Nt + 1) * p->Mp;
    return dalloc(p, reinterpret_cast<void**>(&p->stage), p->stage_elems * sizeof(double), "staging");
}

// Resolve u0/f (inputs, [1]/[Nt] slices) and U ([U_slices], in/out) to device memory.
expd_status stage_in(expd_plan p, const double* u0, const double* f, double* U, size_t U_slices, bool U_is_input,
                     Staging& st, cudaStream_t s) {
    const bool hu0 = u0 && needs_stage(u0);
    const bool hf = f && needs_stage(f);
    const bool hU = U && needs_stage(U);
    if (hu0 || hf || hU) {
        expd_status r = ensure_stage(p);
        if (r != EXPD_OK) return r;
    }
    const size_t M = (size_t)p->Mp;
    st.u0 = u0;
    st.f = f;
    st.U = U;
    st.U_slices = U_slices;
    if (hu0) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(p->stage, u0, M * sizeof(double), cudaMemcpyDefault, s));
        st.u0 = p->stage;
    }
    if (hf) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(p->stage + M, f, (size_t)p->Nt * M * sizeof(double), cudaMemcpyDefault, s));
        st.f = p->stage + M;
    }
    if (hU) {
        st.U_host = U;
        st.U = p->stage + (size_t)(p->Nt + 1) * M;
        if (U_is_input)
            EXPD_CUDA_TRY(cudaMemcpyAsync(st.U, U, U_slices * M * sizeof(double), cudaMemcpyDefault, s));
    }
    return EXPD_OK;
}

expd_status stage_out(expd_plan p, const Staging& st, cudaStream_t s) {
    if (st.U_host)
        EXPD_CUDA_TRY(cudaMemcpyAsync(st.U_host, st.U, st.U_slices * (size_t)p->Mp * sizeof(double),
                                      cudaMemcpyDefault, s));
    if (st.U_host) EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    return EXPD_OK;
}

// The solvers read U when it carries start-up values or the initial iterate.
bool u_is_input(expd_plan p) { return p->startup == EXPD_STARTUP_GIVEN || p->guess == EXPD_GUESS_GIVEN; }

// EXPD_GUESS_GIVEN: the caller's iterate (U's unknown slices u_s..u_Nt,
// physical) in the eigenbasis, float64, into dst
expd_status load_guess(expd_plan p, const double* U, void* dst, cudaStream_t s) {
    return spatial_forward64(p, U + (size_t)(p->order - 1) * p->Mp, dst, p->Ns, s);
}

void* eig_slice(expd_plan p, void* base, long long n) {
    return static_cast<char*>(base) + (size_t)n * p->Mcol * p->esz;
}

// ---- startup values and f_s ----------------------------------------------------
// Sh[n] (eigen) and startphys[n] (physical) for n = 0..s-1, fh (eigen source)
// when f is given, and the assembled right-hand side Fh.
expd_status setup_start(expd_plan p, const double* u0, const double* f, const double* Ugiven, cudaStream_t s,
                        float* F32 = nullptr, int fh_dd = 0) {
    const size_t M = (size_t)p->Mp;
    const int so = p->order;
    // the mixed path transforms its data with double-float arithmetic (2^-48
    // roundoff, far below any tolerance it is run at) on the float32 pipes
    const bool ddt = p->precision == EXPD_PREC_MIXED;
    auto fwd = [&](const double* x, void* y, int n) {
        return ddt ? spatial_forward_dd64(p, x, y, n, s) : spatial_forward64(p, x, y, n, s);
    };
    auto inv = [&](const void* y, double* x, int n) {
        return ddt ? spatial_inverse_dd64(p, y, x, n, s) : spatial_inverse64(p, y, x, n, s);
    };
    EXPD_CUDA_TRY(cudaMemcpyAsync(p->startphys, u0, M * sizeof(double), cudaMemcpyDeviceToDevice, s));
    expd_status st = fwd(p->startphys, p->Sh, 1);
    if (st != EXPD_OK) return st;
    if (f) {
        if (!p->fh) {
            st = dalloc(p, &p->fh, (size_t)p->Nt * p->Mcol * p->esz, "source (eigen)");
            if (st != EXPD_OK) return st;
        }
        st = fwd(f, p->fh, p->Nt);
        if (st != EXPD_OK) return st;
    }
    void* tmp = p->Fh;  // slice 0 of Fh is free until assemble_rhs
    for (int n = 1; n < so; ++n) {
        double* phys_n = p->startphys + (size_t)n * M;
        void* eig_n = eig_slice(p, p->Sh, n);
        if (p->startup == EXPD_STARTUP_GIVEN) {
            EXPD_CUDA_TRY(cudaMemcpyAsync(phys_n, Ugiven + (size_t)(n - 1) * M, M * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
            st = fwd(phys_n, eig_n, 1);
            if (st != EXPD_OK) return st;
            continue;
        }
        // ramp: BDF-n step  w = sum_j a_j A^j u_{n-j} + beta_n dt f(t_n)
        const void* in[6];
        double coef[6];
        for (int j = 1; j <= n; ++j) {
            in[j - 1] = eig_slice(p, p->Sh, n - j);
            coef[j - 1] = p->acoef[n][j];
        }
        const void* src = f ? eig_slice(p, p->fh, n - 1) : nullptr;
        const double bdt = p->beta[n] * p->dt;
        if (p->nonlin == EXPD_NL_NONE) {
            st = eigen_combine(p, eig_n, in, coef, n, src, bdt, s);
            if (st == EXPD_OK) st = inv(eig_n, phys_n, 1);
        } else {
            st = eigen_combine(p, tmp, in, coef, n, src, bdt, s);
            if (st == EXPD_OK) st = inv(tmp, phys_n, 1);
            if (st == EXPD_OK) st = pointwise_solve(p, phys_n, phys_n, (long long)M, bdt, s);
            if (st == EXPD_OK) st = fwd(phys_n, eig_n, 1);
        }
        if (st != EXPD_OK) return st;
    }
    // ETD1: row 0 of f_s gains dt phi_1(dt L) N(u_0); N(u_0) goes through slice
    // 1 of the N buffer (physical scratch) into its slice 0 (eigen)
    const void* nl0 = nullptr;
    if (p->nl_form == EXPD_NLF_ETD1) {
        double* phys = static_cast<double*>(eig_slice(p, p->NL64, 1));
        st = nonlinearity_eval_phys(p, p->startphys, phys, (long long)M, s);
        if (st == EXPD_OK) st = fwd(phys, p->NL64, 1);
        if (st != EXPD_OK) return st;
        nl0 = p->NL64;
    }
    return assemble_rhs(p, f ? p->fh : nullptr, s, F32, fh_dd, nl0);
}

// out = {sqrt(max_n ||s_n||^2), sqrt(max_n ||x_n||^2), sum_n ||s_n||^2, sum_n ||x_n||^2}
// from the per-slice totals, in slice order; the max propagates NaN (fmax
// would drop it and hide a diverged iterate)
expd_status read_reduced_norms(expd_plan p, cudaStream_t s, double out[4]) {
    // the reduction kernel wrote the per-slice totals into mapped host memory
    EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    auto nanmax = [](double a, double b) { return (a != a || b != b) ? NAN : std::max(a, b); };
    double m0 = 0, m1 = 0, s0 = 0, s1 = 0;
    for (int n = 0; n < p->Ns; ++n) {
        const double a = p->redhost[2 * n], b = p->redhost[2 * n + 1];
        m0 = nanmax(m0, a);
        m1 = nanmax(m1, b);
        s0 += a;
        s1 += b;
    }
    out[0] = sqrt(m0);
    out[1] = sqrt(m1);
    out[2] = s0;
    out[3] = s1;
    return EXPD_OK;
}

// U output: u_1..u_{s-1} from the startup values, u_s..u_Nt from Uh.
// Uh holds double-float values when uh_dd (the mixed path's accurate phase).
expd_status write_solution(expd_plan p, double* U, cudaStream_t s, bool uh_dd = false) {
    const size_t M = (size_t)p->Mp;
    if (p->order > 1)
        EXPD_CUDA_TRY(cudaMemcpyAsync(U, p->startphys + M, (size_t)(p->order - 1) * M * sizeof(double),
                                      cudaMemcpyDeviceToDevice, s));
    if (uh_dd) return spatial_inverse_dd(p, p->Uh, U + (size_t)(p->order - 1) * M, p->Ns, s);
    const expd_status st = spatial_inverse64(p, p->Uh, U + (size_t)(p->order - 1) * M, p->Ns, s);
    return st == EXPD_OK ? dst_tc_check(p, s) : st;
}

struct float2_pair {
    float hi, lo;
};
float2_pair split_dd(double v) {
    const float hi = (float)v;
    return {hi, (float)(v - (double)hi)};
}

void info_reset(expd_info* info) {
    if (!info) return;
    memset(info, 0, sizeof(*info));
}

// ---- per-call bookkeeping: phase events, time limit, cancellation ----------
// A solver call records event 0 at its start, 1 when its iterations start, 2
// when its output starts and 3 at its end (only when the caller asked for an
// info report); call_end waits for event 3 and reports the three intervals.
expd_status call_begin(expd_plan p, expd_info* info, cudaStream_t s) {
    info_reset(info);
    nvtx_phase(p, "expd: set-up");
    p->call_t0 = std::chrono::steady_clock::now();
    p->call_cancelled = 0;
    if (!info) return EXPD_OK;
    for (cudaEvent_t& e : p->phase_ev)
        if (!e) EXPD_CUDA_TRY(cudaEventCreate(&e));
    EXPD_CUDA_TRY(cudaEventRecord(p->phase_ev[0], s));
    return EXPD_OK;
}

expd_status call_mark(expd_plan p, expd_info* info, int k, cudaStream_t s) {
    nvtx_phase(p, k == 1 ? "expd: iterations" : "expd: output");
    if (info) EXPD_CUDA_TRY(cudaEventRecord(p->phase_ev[k], s));
    return EXPD_OK;
}

// Ends a call that returns `result`: phase times into info; a failure to read
// them only replaces an OK result.
expd_status call_end(expd_plan p, expd_info* info, cudaStream_t s, expd_status result) {
    nvtx_phase(p, nullptr);
    if (p->canary && result == EXPD_OK) result = canary_check(p, s);
    if (!info) return result;
    cudaError_t e = cudaEventRecord(p->phase_ev[3], s);
    if (e == cudaSuccess) e = cudaEventSynchronize(p->phase_ev[3]);
    float t[3] = {0, 0, 0};
    for (int k = 0; k < 3 && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&t[k], p->phase_ev[k], p->phase_ev[k + 1]);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return result == EXPD_OK ? expd_cuda_fail(e, "phase events", __FILE__, __LINE__) : result;
    }
    info->ms_setup = t[0];
    info->ms_iterate = t[1];
    info->ms_output = t[2];
    return result;
}

// Between iterations: EXPD_ERR_CANCELLED when expd_plan_cancel asked for it
// (the request is consumed), EXPD_ERR_TIMEOUT when the scheme's time limit ran
// out, else EXPD_OK.
expd_status poll_stop(expd_plan p) {
    if (p->cancel_req.load(std::memory_order_acquire) && p->cancel_req.exchange(0)) {
        if (p->cancel_host) *p->cancel_host = 0;
        p->call_cancelled = 1;
        return expd_fail(EXPD_ERR_CANCELLED, "cancelled by expd_plan_cancel");
    }
    if (p->time_limit_ms > 0) {
        const double ms =
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - p->call_t0).count();
        if (ms > p->time_limit_ms)
            return expd_fail(EXPD_ERR_TIMEOUT, "time limit of " + std::to_string(p->time_limit_ms) + " ms reached");
    }
    return EXPD_OK;
}

}  // namespace

cudaError_t plan_malloc(expd_plan p, void** ptr, size_t bytes) {
    if (!p->pooled) return cudaMalloc(ptr, bytes);
    cudaError_t e = cudaMallocAsync(ptr, bytes, p->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    return e;
}

void plan_free(expd_plan p, void* ptr) {
    if (!ptr) return;
    if (p->pooled) cudaFreeAsync(ptr, p->stream);
    else cudaFree(ptr);
}

cudaError_t smem_allow(const void* kern, size_t smem) {
    static std::mutex mu;
    static std::vector<const void*> done;
    static int optin = -1;
    std::lock_guard<std::mutex> lk(mu);
    if (optin < 0) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) {
            optin = -1;
            return e;
        }
    }
    if (smem > (size_t)optin) return cudaErrorInvalidValue;
    if (std::find(done.begin(), done.end(), kern) != done.end()) return cudaSuccess;
    // the limit covers static plus dynamic shared memory
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    const int dyn_max = optin - (int)fa.sharedSizeBytes;
    if (smem > (size_t)std::max(dyn_max, 0)) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max);
    if (e == cudaSuccess) done.push_back(kern);
    return e;
}

cudaError_t plan_bind_stream(expd_plan p, cudaStream_t s) {
    if (p->stream == s) return cudaSuccess;
    cudaError_t e = cudaStreamSynchronize(p->stream);
    p->stream = s;
    return e;
}


expd_status expd_cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_err = buf;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? EXPD_ERR_OOM : EXPD_ERR_CUDA;
}

void expd_clear_error() { g_err.clear(); }

expd_status expd_fail(expd_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

KProf::KProf(expd_plan p_, cudaStream_t s_, int cls_, double bytes_, double flops_)
    : p(p_), s(s_), cls(cls_), bytes(bytes_), flops(flops_) {
    ++p->launches;
    nvtxRangePushA(kclass_name(cls));
    if (!p->timing) return;
    while (p->events.size() < p->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return;
        }
        p->events.push_back(e);
    }
    e0 = (int)p->ev_used;
    p->ev_used += 2;
    cudaEventRecord(p->events[e0], s);
}

KProf::~KProf() {
    nvtxRangePop();
    if (e0 < 0) return;
    cudaEventRecord(p->events[e0 + 1], s);
    p->recs.push_back({cls, e0, bytes, flops});
}

expd_status canary_check(expd_plan p, cudaStream_t s) {
    if (!p->canary) return EXPD_OK;
    std::vector<unsigned char> tail(CANARY_BYTES);
    for (const auto& c : p->canaries) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(tail.data(), static_cast<const char*>(c.first) + c.second, CANARY_BYTES,
                                      cudaMemcpyDeviceToHost, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        for (unsigned char b : tail)
            if (b != CANARY_BYTE)
                return expd_fail(EXPD_ERR_CUDA, "guard words after a workspace buffer of " +
                                                    std::to_string(c.second) + " bytes were overwritten");
    }
    return EXPD_OK;
}

expd_status plan_init_fields(expd_plan p, const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                             double alpha, const expd_scheme* scheme) {
    if (!grid || !op || !scheme) return expd_fail(EXPD_ERR_INVALID_ARG, "grid, operator and scheme are required");
    if (grid->ndim != 1 && grid->ndim != 2) return expd_fail(EXPD_ERR_INVALID_ARG, "ndim must be 1 or 2");
    if (grid->bc != EXPD_BC_PERIODIC && grid->bc != EXPD_BC_DIRICHLET && grid->bc != EXPD_BC_NEUMANN)
        return expd_fail(EXPD_ERR_INVALID_ARG, "bc must be EXPD_BC_PERIODIC, EXPD_BC_DIRICHLET or EXPD_BC_NEUMANN");
    for (int d = 0; d < grid->ndim; ++d) {
        const int n = grid->n[d];
        if (grid->bc == EXPD_BC_PERIODIC && (!is_pow2(n) || n < 8 || n > EXPD_MAX_PERIODIC_N))
            return expd_fail(EXPD_ERR_INVALID_ARG, "periodic grid sizes must be powers of two in [8, 4096]");
        if (grid->bc == EXPD_BC_DIRICHLET && (n < 2 || n > EXPD_MAX_DIRICHLET_N))
            return expd_fail(EXPD_ERR_INVALID_ARG, "Dirichlet grid sizes must be in [2, 4096]");
        if (grid->bc == EXPD_BC_NEUMANN && (n < 2 || n > EXPD_MAX_DIRICHLET_N))
            return expd_fail(EXPD_ERR_INVALID_ARG, "Neumann grid sizes must be in [2, 4096]");
        if (!(grid->length[d] > 0) || !isfinite(grid->length[d]))
            return expd_fail(EXPD_ERR_INVALID_ARG, "domain lengths must be positive");
    }
    if (!(dt > 0) || !isfinite(dt)) return expd_fail(EXPD_ERR_INVALID_ARG, "dt must be positive");
    if (!(alpha > 0 && alpha < 1)) return expd_fail(EXPD_ERR_INVALID_ARG, "alpha must lie in (0, 1)");
    if (scheme->order < 1 || scheme->order > 6) return expd_fail(EXPD_ERR_INVALID_ARG, "order must be 1..6");
    if (Nt < scheme->order + 1 || Nt > kMaxSlices)
        return expd_fail(EXPD_ERR_INVALID_ARG, "Nt must be at least order + 1");
    if (Nt - scheme->order + 1 > EXPD_MAX_NS)
        return expd_fail(EXPD_ERR_UNSUPPORTED, "Nt - order + 1 exceeds 512 unknown slices");
    if (op->nonlin != EXPD_NL_NONE && op->nonlin != EXPD_NL_ALLEN_CAHN)
        return expd_fail(EXPD_ERR_INVALID_ARG, "unknown nonlinearity");
    if (!isfinite(op->a) || !isfinite(op->c) || !isfinite(op->a_im) || !isfinite(op->c_im))
        return expd_fail(EXPD_ERR_INVALID_ARG, "a and c must be finite");
    if (op->complex_state != 0 && op->complex_state != 1)
        return expd_fail(EXPD_ERR_INVALID_ARG, "complex_state must be 0 or 1");
    if (!op->complex_state && (op->a_im != 0.0 || op->c_im != 0.0))
        return expd_fail(EXPD_ERR_INVALID_ARG, "a complex a or c needs complex_state = 1");
    if (op->complex_state && op->nonlin != EXPD_NL_NONE)
        return expd_fail(EXPD_ERR_UNSUPPORTED, "complex states are built for linear problems");
    if (op->complex_state && scheme->precision != EXPD_PREC_FP64)
        return expd_fail(EXPD_ERR_UNSUPPORTED, "complex states run in the float64 precision");
    if (scheme->precision != EXPD_PREC_FP64 && scheme->precision != EXPD_PREC_MIXED)
        return expd_fail(EXPD_ERR_INVALID_ARG, "unknown precision");
    if (scheme->max_iter < 1 || scheme->max_iter > 100000)
        return expd_fail(EXPD_ERR_INVALID_ARG, "max_iter must be in [1, 100000]");
    if (!(scheme->tol > 0)) return expd_fail(EXPD_ERR_INVALID_ARG, "tol must be positive");
    if (scheme->gmres_restart < 1 || scheme->gmres_restart > 64)
        return expd_fail(EXPD_ERR_INVALID_ARG, "gmres_restart must be in [1, 64]");
    if (scheme->jacobian != EXPD_JAC_LAGGED && scheme->jacobian != EXPD_JAC_MEAN_U0)
        return expd_fail(EXPD_ERR_INVALID_ARG, "jacobian must be EXPD_JAC_LAGGED or EXPD_JAC_MEAN_U0");
    if (scheme->guess != EXPD_GUESS_LINEAR && scheme->guess != EXPD_GUESS_ZERO && scheme->guess != EXPD_GUESS_GIVEN)
        return expd_fail(EXPD_ERR_INVALID_ARG, "guess must be EXPD_GUESS_LINEAR, EXPD_GUESS_ZERO or EXPD_GUESS_GIVEN");
    if (scheme->startup != EXPD_STARTUP_RAMP && scheme->startup != EXPD_STARTUP_GIVEN)
        return expd_fail(EXPD_ERR_INVALID_ARG, "unknown startup mode");
    if (scheme->kernel_flags & ~(EXPD_KF_TIME_SMEM | EXPD_KF_FFT_RADIX4 | EXPD_KF_DST_FP64 | EXPD_KF_DST_N64))
        return expd_fail(EXPD_ERR_INVALID_ARG, "unknown kernel_flags bits");
    if (scheme->nl_form != EXPD_NLF_IF && scheme->nl_form != EXPD_NLF_ETD1)
        return expd_fail(EXPD_ERR_INVALID_ARG, "nl_form must be EXPD_NLF_IF or EXPD_NLF_ETD1");
    if (scheme->nl_form == EXPD_NLF_ETD1 && op->nonlin != EXPD_NL_NONE && scheme->order != 1)
        return expd_fail(EXPD_ERR_INVALID_ARG, "the ETD1 form is a first-order scheme (order 1)");
    if (!(scheme->time_limit_ms >= 0) || !isfinite(scheme->time_limit_ms))
        return expd_fail(EXPD_ERR_INVALID_ARG, "time_limit_ms must be finite and >= 0");
    p->ndim = grid->ndim;
    if (p->ndim == 1) {
        p->NX = grid->n[0];
        p->NY = 1;
        p->LX = grid->length[0];
        p->LY = 1.0;
    } else {
        p->NY = grid->n[0];
        p->NX = grid->n[1];
        p->LY = grid->length[0];
        p->LX = grid->length[1];
    }
    p->bc = grid->bc;
    p->a = op->a;
    p->c = op->c;
    p->a_im = op->a_im;
    p->c_im = op->c_im;
    p->cplx = op->complex_state;
    p->nonlin = op->nonlin;
    if (!isfinite(op->b[0]) || !isfinite(op->b[1])) return expd_fail(EXPD_ERR_INVALID_ARG, "b must be finite");
    if (grid->ndim == 1) {
        p->bx = op->b[0];
    } else {
        p->by = op->b[0];  // axis 0 is the slow (NY) axis
        p->bx = op->b[1];
    }
    const bool velocity = p->bx != 0.0 || p->by != 0.0;
    if (velocity && grid->bc != EXPD_BC_PERIODIC)
        return expd_fail(EXPD_ERR_INVALID_ARG, "advection needs a periodic grid (the sine basis does not diagonalise it)");
    // complex E and coefficient tables whenever the symbol is complex
    p->adv = velocity || p->a_im != 0.0 || p->c_im != 0.0;
    if (op->nonlin != EXPD_NL_NONE && scheme->nl_form == EXPD_NLF_ETD1) {
        if (p->adv) return expd_fail(EXPD_ERR_UNSUPPORTED, "the ETD1 form takes real symbols (no advection)");
        if (scheme->jacobian == EXPD_JAC_MEAN_U0)
            return expd_fail(EXPD_ERR_INVALID_ARG, "the mean-Jacobian preconditioner is defined for the IF form only");
    }
    p->dt = dt;
    p->Nt = Nt;
    p->order = scheme->order;
    p->Ns = Nt - scheme->order + 1;
    p->alpha = alpha;
    p->precision = scheme->precision;
    p->max_iter = scheme->max_iter;
    p->tol = scheme->tol;
    p->restart = scheme->gmres_restart;
    p->startup = scheme->startup;
    p->jacobian = scheme->jacobian;
    p->guess = scheme->guess;
    p->nl_form = op->nonlin != EXPD_NL_NONE ? scheme->nl_form : EXPD_NLF_IF;
    p->time_limit_ms = scheme->time_limit_ms;
    // kernel variants: the scheme's flags, or the environment switches read here
    // (EXPD_TIME_KERNEL=smem, EXPD_FFT_KERNEL=radix4, EXPD_DST_TC=0)
    p->kernel_flags = scheme->kernel_flags;
    {
        const char* tk = getenv("EXPD_TIME_KERNEL");
        if (tk && strcmp(tk, "smem") == 0) p->kernel_flags |= EXPD_KF_TIME_SMEM;
        const char* cf = getenv("EXPD_FFT_KERNEL");
        if (cf && strcmp(cf, "radix4") == 0) p->kernel_flags |= EXPD_KF_FFT_RADIX4;
        const char* dt0 = getenv("EXPD_DST_TC");
        if (dt0 && strcmp(dt0, "0") == 0) p->kernel_flags |= EXPD_KF_DST_FP64;
        // mixed Krylov refinement threshold (a cycle ends once its residual fell by eta)
        const char* ke = getenv("EXPD_KRYLOV_ETA");
        if (ke) {
            const double v = atof(ke);
            if (v > 0 && v < 1) p->krylov_eta = v;
        }
    }
    for (int q = 1; q <= 6; ++q) bdf(q, p->acoef[q], &p->beta[q]);
    if (p->nonlin != EXPD_NL_NONE) {
        for (int q = 1; q <= p->order; ++q)
            if (!(p->beta[q] * dt < 1.0)) return expd_fail(EXPD_ERR_INVALID_ARG, "nonlinear problems need beta_s*dt < 1");
    }
    p->M = (long long)p->NX * p->NY;
    p->Mp = p->M * (p->cplx ? 2 : 1);
    // a real state on a Dirichlet grid has real sine coefficients; a complex
    // state keeps every mode (the full spectrum on a periodic grid: no
    // conjugate symmetry halves it)
    p->realcol = p->bc != EXPD_BC_PERIODIC && !p->cplx;
    p->KX = (p->bc != EXPD_BC_PERIODIC || p->cplx) ? p->NX : p->NX / 2 + 1;
    p->Mcol = (long long)p->NY * p->KX;
    p->esz = p->realcol ? sizeof(double) : sizeof(double2);
    if (p->bc == EXPD_BC_DIRICHLET) {
        auto fast = [](int n) { return n >= 3 && n + 1 <= 4096 && ((n + 1) & n) == 0; };
        p->fast_dst = fast(p->NX) && (p->ndim == 1 || fast(p->NY));
    }
    p->tc_dst = dst_tc_eligible(p) ? 1 : 0;
    if (p->tc_dst) dst_tc_layout(p);
    int dev = 0;
    cudaError_t ce = cudaGetDevice(&dev);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (ce != cudaSuccess) return expd_cuda_fail(ce, "cudaGetDevice/cudaDeviceGetAttribute", __FILE__, __LINE__);
    // EXPD_KF_TIME_SMEM selects the shared-memory time kernel for every window
    // (both kernels compute the same sweep; this lets them be compared)
    p->no_reg_time = (p->kernel_flags & EXPD_KF_TIME_SMEM) != 0;
    // EXPD_KF_FFT_RADIX4 selects the shared-memory radix-4 row and column
    // FFTs for every size (both compute the same transforms)
    p->no_fft4 = (p->kernel_flags & EXPD_KF_FFT_RADIX4) != 0;
    // EXPD_TIME_REAL=0: real (Dirichlet) columns take the generic shared-memory
    // kernel instead of the real-column one (both compute the same; tests)
    const char* tr = getenv("EXPD_TIME_REAL");
    p->no_real_time = tr && strcmp(tr, "0") == 0;
    // EXPD_TIME_TC=0: real columns keep the FFT time kernels instead of the
    // tensor-core one (both compute the same preconditioner; comparisons)
    const char* ttc = getenv("EXPD_TIME_TC");
    p->no_tc_time = ttc && strcmp(ttc, "0") == 0;
    const char* gr = getenv("EXPD_GRAPHS");
    p->no_graphs = gr && strcmp(gr, "0") == 0;
    const char* po = getenv("EXPD_POISON");
    p->poison = po && strcmp(po, "1") == 0;
    const char* ca = getenv("EXPD_CANARY");
    p->canary = ca && strcmp(ca, "1") == 0;
    // EXPD_TIME_CPLX=0: complex columns take the generic shared-memory kernel
    // instead of the fixed-length one (both compute the same; tests)
    const char* tc = getenv("EXPD_TIME_CPLX");
    p->no_cplx_time = tc && strcmp(tc, "0") == 0;
    // the device-controlled loop is opt-in (EXPD_DEVICE_LOOP=1): on GB300 its
    // while-node iterations measured slower than host round trips that read
    // the norms from mapped memory (0.624 against 0.594 ms per solve on
    // 256^2 x 64)
    const char* dl = getenv("EXPD_DEVICE_LOOP");
    p->no_device_loop = !(dl && strcmp(dl, "1") == 0);
    return EXPD_OK;
}

bool expd_is_device_ptr(const void* ptr) { return is_device_ptr(ptr); }

// Runs one fixed-point sweep: launched kernel by kernel when per-kernel timing
// is on (its events cannot sit in a graph), on the legacy default stream
// (which cannot be captured) or with EXPD_GRAPHS=0; otherwise captured once per
// phase (and per value of the pointer, shift and right-hand side slice count
// baked into its launches) and relaunched as one CUDA graph.
template <typename Issue>
static expd_status run_sweep(expd_plan p, int phase, const void* key_ptr, double key_shift, int key_fs,
                             cudaStream_t s, Issue&& issue) {
    if (p->timing || p->no_graphs || s == nullptr) return issue();
    auto& G = p->sweep_graph[phase];
    if (!G.eager) {  // the first sweep of a phase runs directly (one-time kernel set-up outside capture)
        G.eager = 1;
        return issue();
    }
    if (!G.exec || G.key_ptr != key_ptr || G.key_shift != key_shift || G.key_fs != key_fs) {
        if (G.exec) {
            cudaGraphExecDestroy(G.exec);
            G.exec = nullptr;
        }
        const long long before = p->launches;
        EXPD_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        const expd_status st = issue();
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != EXPD_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
        const cudaError_t ei = cudaGraphInstantiate(&G.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            G.exec = nullptr;
            return expd_cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
        }
        G.key_ptr = key_ptr;
        G.key_shift = key_shift;
        G.key_fs = key_fs;
        G.launches = p->launches - before;
        p->launches = before;
    }
    EXPD_CUDA_TRY(cudaGraphLaunch(G.exec, s));
    p->launches += G.launches;
    return EXPD_OK;
}

// ---- the fixed point under device control ----------------------------------
// After every sweep one warp reduces the per-slice totals (max over slices of
// the update and iterate norms, sums only for the finiteness test), runs the
// stopping test of expd_solve_fp's host loop on the same double values, and
// sets the while-node conditions: this loop continues, or it ends and (float32
// loop only) the accurate loop is entered.  A run is bounded by max_iter
// sweeps in all (the counter lives in LoopCtl), so the loop always ends.
struct CtlArgs {
    LoopCtl* c;
    const double2* tot;  // [Ns] per-slice totals from time_reduce
    int Ns, phase32, max_iter, sout_set;
    double tol;
    cudaGraphConditionalHandle self, next;
    int has_next;
};

__device__ __forceinline__ double ctl_nanmax(double a, double b) { return (a != a || b != b) ? CUDART_NAN : (a < b ? b : a); }

__global__ void loop_init_kernel(LoopCtl* c) {
    c->it = 0;
    c->it32 = 0;
    c->result = EXPD_ERR_NOT_CONVERGED;
    c->phys_valid = 0;
    c->prev = 0.0;
    c->rho = 0.5;
    c->rho_phase = -1.0;
    c->measure = 1.0;
    c->s_first = 0.0;
    c->last_rel = 1.0;
}

__global__ void set_slot_kernel(double** slot, double* v) { *slot = v; }

// the loop state into mapped host memory (no copy-engine round trip)
__global__ void loop_out_kernel(const LoopCtl* c, LoopCtl* h) {
    const double* src = reinterpret_cast<const double*>(c);
    double* dst = reinterpret_cast<double*>(h);
    for (int i = threadIdx.x; i < (int)EXPD_CTL_DOUBLES; i += blockDim.x) dst[i] = src[i];
}

__global__ void loop_ctl_kernel(CtlArgs a) {
    const int lane = threadIdx.x;
    double m0 = 0.0, m1 = 0.0, s0 = 0.0, s1 = 0.0;
    for (int n = lane; n < a.Ns; n += 32) {
        const double2 v = a.tot[n];
        m0 = ctl_nanmax(m0, v.x);
        m1 = ctl_nanmax(m1, v.y);
        s0 += v.x;
        s1 += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
        m0 = ctl_nanmax(m0, __shfl_xor_sync(0xffffffffu, m0, o));
        m1 = ctl_nanmax(m1, __shfl_xor_sync(0xffffffffu, m1, o));
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane != 0) return;
    LoopCtl& c = *a.c;
    const int it = ++c.it;
    if (a.phase32) ++c.it32;
    c.phys_valid = a.sout_set;
    const double smax = sqrt(m0), umax = sqrt(m1);
    c.last_rel = umax > 0 ? smax / umax : 1.0;
    if (it == 1) c.s_first = smax;
    bool stop = false, leave = false;
    if (!isfinite(smax) || !isfinite(umax) || !isfinite(s0) || !isfinite(s1) || (it > 1 && smax > 1e3 * c.s_first)) {
        c.result = EXPD_ERR_DIVERGED;
        stop = true;
    } else {
        const double rel = umax > 0 ? smax / umax : 0.0;
        if (it > 1 && c.prev > 0) {
            const double ratio = smax / c.prev;
            const double lo = 1e-12 < ratio ? ratio : 1e-12;
            c.rho = 0.95 < lo ? 0.95 : lo;
        }
        const double r_use = (c.rho_phase > 0 && !a.phase32) ? c.rho_phase : c.rho;
        c.measure = it == 1 ? rel : rel * r_use / (1.0 - r_use);
        if (it <= EXPD_MAX_HISTORY) c.history[it - 1] = c.measure;
        if (a.phase32) {
            const bool stalled = it > 2 && c.rho > 0.5;
            const double floor32 = 4.0 * 5.96e-8;
            const bool one_more = it > 2 && c.rho * (c.measure + floor32) <= a.tol;
            if (c.measure <= a.tol || stalled || one_more) {
                leave = true;
                if (!stalled) c.rho_phase = c.rho;
                else if (c.rho_phase < 0) c.rho_phase = 0.5;
            } else if (c.rho < 0.5) {
                c.rho_phase = c.rho;
            }
        } else if (c.measure <= a.tol) {
            c.result = EXPD_OK;
            stop = true;
        }
        c.prev = smax;
    }
    const bool budget = it < a.max_iter;
    cudaGraphSetConditional(a.self, (!stop && !leave && budget) ? 1u : 0u);
    if (a.has_next) cudaGraphSetConditional(a.next, (!stop && budget) ? 1u : 0u);
}

// Captures what f() launches on s into graph g after the nodes deps; leaves
// receives the capture's final dependency set (the nodes to continue from).
template <typename F>
static expd_status capture_into(cudaStream_t s, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                                std::vector<cudaGraphNode_t>* leaves, F&& f) {
    EXPD_CUDA_TRY(cudaStreamBeginCaptureToGraph(s, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeThreadLocal));
    const expd_status st = f();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t* d = nullptr;
    size_t nd = 0;
    const cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
    if (e == cudaSuccess && leaves) leaves->assign(d, d + nd);
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &out);
    if (st != EXPD_OK) return st;
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaStreamGetCaptureInfo", __FILE__, __LINE__);
    if (e2 != cudaSuccess) return expd_cuda_fail(e2, "cudaStreamEndCapture", __FILE__, __LINE__);
    return EXPD_OK;
}

static expd_status add_while(cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps, cudaGraphConditionalHandle h,
                             cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    EXPD_CUDA_TRY(cudaGraphAddNode(node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &np));
    *body = np.conditional.phGraph_out[0];
    return EXPD_OK;
}

struct LoopBody {
    int phase32;   // 1: the float32 loop (ends into the accurate loop)
    int sout_set;  // the sweep writes the float32 update copy
};

// Runs the fixed point as one graph: init, while(loop 1) { sweep1; control },
// then (two = true) between(), while(loop 2) { sweep2; control }.  The graph
// is built on the first call and relaunched while the pointer, shift and
// right-hand side slice count baked into its launches are unchanged.
template <typename Sweep1, typename Between, typename Sweep2>
static expd_status run_device_loop(expd_plan p, cudaStream_t s, bool two, LoopBody b1, LoopBody b2,
                                   const void* key_ptr, double key_shift, int key_fs, Sweep1&& sweep1,
                                   Between&& between, Sweep2&& sweep2, LoopCtl* out) {
    auto& LG = p->loop_graph;
    LoopCtl* dctl = reinterpret_cast<LoopCtl*>(p->redout + 8 + 2 * (size_t)p->Ns);
    const double2* tot = reinterpret_cast<const double2*>(p->redout + 8);
    if (!LG.exec || LG.key_ptr != key_ptr || LG.key_shift != key_shift || LG.key_fs != key_fs || LG.two != (int)two) {
        if (LG.exec) {
            cudaGraphExecDestroy(LG.exec);
            LG.exec = nullptr;
        }
        cudaGraph_t g = nullptr;
        EXPD_CUDA_TRY(cudaGraphCreate(&g, 0));
        const long long before = p->launches;
        auto build = [&]() -> expd_status {
            cudaGraphConditionalHandle h1 = 0, h2 = 0;
            EXPD_CUDA_TRY(cudaGraphConditionalHandleCreate(&h1, g, 1, cudaGraphCondAssignDefault));
            if (two) EXPD_CUDA_TRY(cudaGraphConditionalHandleCreate(&h2, g, 0, cudaGraphCondAssignDefault));
            std::vector<cudaGraphNode_t> deps;
            long long l0 = p->launches;
            expd_status st = capture_into(s, g, {}, &deps, [&]() -> expd_status {
                loop_init_kernel<<<1, 1, 0, s>>>(dctl);
                ++p->launches;
                EXPD_CUDA_TRY(cudaGetLastError());
                return EXPD_OK;
            });
            if (st != EXPD_OK) return st;
            LG.l_init = p->launches - l0;
            auto body = [&](cudaGraphConditionalHandle self, const LoopBody& lb, auto&& sweep, long long* count)
                -> expd_status {
                cudaGraphNode_t wn = nullptr;
                cudaGraph_t bg = nullptr;
                expd_status r = add_while(g, deps, self, &wn, &bg);
                if (r != EXPD_OK) return r;
                const long long c0 = p->launches;
                r = capture_into(s, bg, {}, nullptr, [&]() -> expd_status {
                    expd_status q = sweep();
                    if (q != EXPD_OK) return q;
                    CtlArgs a;
                    a.c = dctl;
                    a.tot = tot;
                    a.Ns = p->Ns;
                    a.phase32 = lb.phase32;
                    a.max_iter = p->max_iter;
                    a.sout_set = lb.sout_set;
                    a.tol = p->tol;
                    a.self = self;
                    a.next = h2;
                    a.has_next = lb.phase32 && two;
                    loop_ctl_kernel<<<1, 32, 0, s>>>(a);
                    ++p->launches;
                    EXPD_CUDA_TRY(cudaGetLastError());
                    return EXPD_OK;
                });
                if (r != EXPD_OK) return r;
                *count = p->launches - c0;
                deps.assign(1, wn);
                return EXPD_OK;
            };
            st = body(h1, b1, sweep1, &LG.l_body1);
            if (st != EXPD_OK) return st;
            if (two) {
                l0 = p->launches;
                st = capture_into(s, g, deps, &deps, between);
                if (st != EXPD_OK) return st;
                LG.l_between = p->launches - l0;
                st = body(h2, b2, sweep2, &LG.l_body2);
                if (st != EXPD_OK) return st;
            }
            // tail: the loop state into mapped host memory
            return capture_into(s, g, deps, nullptr, [&]() -> expd_status {
                loop_out_kernel<<<1, 64, 0, s>>>(dctl, reinterpret_cast<LoopCtl*>(p->redhost_dev + 2 * (size_t)p->Ns));
                ++p->launches;
                EXPD_CUDA_TRY(cudaGetLastError());
                return EXPD_OK;
            });
        };
        const expd_status st = build();
        p->launches = before;
        if (st != EXPD_OK) {
            cudaGraphDestroy(g);
            return st;
        }
        const cudaError_t ei = cudaGraphInstantiate(&LG.exec, g, 0);
        cudaGraphDestroy(g);
        if (ei != cudaSuccess) {
            LG.exec = nullptr;
            return expd_cuda_fail(ei, "cudaGraphInstantiate(fixed point)", __FILE__, __LINE__);
        }
        LG.key_ptr = key_ptr;
        LG.key_shift = key_shift;
        LG.key_fs = key_fs;
        LG.two = two;
    }
    EXPD_CUDA_TRY(cudaGraphLaunch(LG.exec, s));
    EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    *out = *reinterpret_cast<const LoopCtl*>(p->redhost + 2 * (size_t)p->Ns);
    const long long n1 = two ? out->it32 : out->it;
    p->launches += LG.l_init + n1 * LG.l_body1 + (two ? LG.l_between + (out->it - n1) * LG.l_body2 : 0) + 1;
    return EXPD_OK;
}

extern "C" {

const char* expd_status_string(expd_status s) {
    switch (s) {
        case EXPD_OK: return "ok";
        case EXPD_ERR_INVALID_ARG: return "invalid argument";
        case EXPD_ERR_OOM: return "out of device memory";
        case EXPD_ERR_NOT_CONVERGED: return "not converged";
        case EXPD_ERR_DIVERGED: return "diverged";
        case EXPD_ERR_CUDA: return "CUDA error";
        case EXPD_ERR_UNSUPPORTED: return "unsupported";
        case EXPD_ERR_TIMEOUT: return "timed out";
        case EXPD_ERR_CANCELLED: return "cancelled";
    }
    return "unknown status";
}

const char* expd_last_error(void) { return g_err.c_str(); }

int expd_version(void) { return 10000; }

expd_status expd_plan_create(const expd_grid* grid, const expd_operator* op, double dt, int Nt, double alpha,
                             const expd_scheme* scheme, void* stream, expd_plan* out) {
    if (!out) return expd_fail(EXPD_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    g_err.clear();
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    expd_plan p = new expd_plan_s();
    expd_status st0 = plan_init_fields(p, grid, op, dt, Nt, alpha, scheme);
    if (st0 != EXPD_OK) {
        delete p;
        return st0;
    }
    p->stream = s;
    {
        int dev = 0, pools = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess)
            p->pooled = pools;
        cudaGetLastError();
    }
    expd_status st = EXPD_OK;
    // ---- eigenvalues of L_h: E_m = exp(dt mu_m) ----
    {
        const int cw = p->adv ? 2 : 1;  // complex tables (re, im) with advection
        std::vector<double> E((size_t)cw * p->Mcol), C64((size_t)cw * p->order * p->Mcol);
        std::vector<float> C32((size_t)cw * p->order * p->Mcol);
        for (long long m = 0; m < p->Mcol; ++m) {
            const int kx = (int)(m % p->KX);
            const int ky = (int)(m / p->KX);
            // symbol mu + i nu = (a + i a_im) lap_m - i b.k - (c + i c_im), lap_m
            // the Laplacian's eigenvalue on mode m
            double lap = 0.0, nu = -p->c_im;
            if (p->bc == EXPD_BC_PERIODIC) {
                // signed wavenumber (a complex state stores the full spectrum)
                const int kxf = kx <= p->NX / 2 ? kx : kx - p->NX;
                const double wx = 2.0 * M_PI * kxf / p->LX;
                lap -= wx * wx;
                if (2 * kx != p->NX) nu -= p->bx * wx;  // first derivative: 0 at the Nyquist wavenumber
                if (p->ndim == 2) {
                    const int kyf = ky <= p->NY / 2 ? ky : ky - p->NY;
                    const double wy = 2.0 * M_PI * kyf / p->LY;
                    lap -= wy * wy;
                    if (2 * ky != p->NY) nu -= p->by * wy;
                }
            } else {
                lap = fd_laplacian_symbol(p, kx, ky);
            }
            const double mu = p->a * lap - p->c;
            nu += p->a_im * lap;
            if (!p->adv) {
                E[m] = exp(dt * mu);
                for (int j = 1; j <= p->order; ++j) {
                    const double cjm = p->acoef[p->order][j] * exp(j * dt * mu);
                    C64[(size_t)(j - 1) * p->Mcol + m] = cjm;
                    C32[(size_t)(j - 1) * p->Mcol + m] = (float)cjm;
                }
            } else {
                // E = e^{dt mu} (cos dt nu + i sin dt nu), a_j E^j likewise
                E[2 * m] = exp(dt * mu) * cos(dt * nu);
                E[2 * m + 1] = exp(dt * mu) * sin(dt * nu);
                for (int j = 1; j <= p->order; ++j) {
                    const double r = p->acoef[p->order][j] * exp(j * dt * mu);
                    const size_t i = (size_t)(j - 1) * p->Mcol + m;
                    C64[2 * i] = r * cos(j * dt * nu);
                    C64[2 * i + 1] = r * sin(j * dt * nu);
                    C32[2 * i] = (float)C64[2 * i];
                    C32[2 * i + 1] = (float)C64[2 * i + 1];
                }
            }
        }
        st = upload_vec(p, &p->E, E, "E", s);
        if (st == EXPD_OK) st = upload_vec(p, &p->C64, C64, "coefficients", s);
        if (st == EXPD_OK) st = upload_vec(p, &p->C32, C32, "coefficients (float32)", s);
        if (st == EXPD_OK && p->precision == EXPD_PREC_MIXED && p->bc == EXPD_BC_PERIODIC) {
            std::vector<float2> Cdd(C64.size());
            for (size_t i = 0; i < C64.size(); ++i) {
                const float2_pair d = split_dd(C64[i]);
                Cdd[i] = make_float2(d.hi, d.lo);
            }
            float2* dptr = nullptr;
            st = upload_vec(p, &dptr, Cdd, "coefficients (double-float)", s);
            p->Cdd = dptr;
        }
    }
    // ---- ETD1: dt phi_1(dt mu_m), phi_1(z) = expm1(z)/z, phi_1(0) = 1 ----
    if (st == EXPD_OK && p->nl_form == EXPD_NLF_ETD1) {
        std::vector<double> ph((size_t)p->Mcol);
        std::vector<float> ph32((size_t)p->Mcol);
        std::vector<float2> phdd((size_t)p->Mcol);
        for (long long m = 0; m < p->Mcol; ++m) {
            const int kx = (int)(m % p->KX), ky = (int)(m / p->KX);
            double mu = -p->c;
            if (p->bc == EXPD_BC_PERIODIC) {
                const double wx = 2.0 * M_PI * kx / p->LX;
                mu -= p->a * wx * wx;
                if (p->ndim == 2) {
                    const int kyf = ky <= p->NY / 2 ? ky : ky - p->NY;
                    const double wy = 2.0 * M_PI * kyf / p->LY;
                    mu -= p->a * wy * wy;
                }
            } else {
                mu += p->a * fd_laplacian_symbol(p, kx, ky);
            }
            const double z = dt * mu;
            ph[m] = dt * (z == 0.0 ? 1.0 : std::expm1(z) / z);
            ph32[m] = (float)ph[m];
            const float2_pair d = split_dd(ph[m]);
            phdd[m] = make_float2(d.hi, d.lo);
        }
        st = upload_vec(p, &p->PHI64, ph, "phi_1 table", s);
        if (st == EXPD_OK) st = upload_vec(p, &p->PHI32, ph32, "phi_1 table (float32)", s);
        if (st == EXPD_OK && p->precision == EXPD_PREC_MIXED && p->bc == EXPD_BC_PERIODIC) {
            float2* dptr = nullptr;
            st = upload_vec(p, &dptr, phdd, "phi_1 table (double-float)", s);
            p->PHIdd = dptr;
        }
    }
    // ---- spatial transform tables ----
    if (st == EXPD_OK && p->bc == EXPD_BC_PERIODIC) {
        std::vector<double2> w64(p->NX / 2 + 1);
        std::vector<float2> w32(p->NX / 2 + 1);
        for (int k = 0; k <= p->NX / 2; ++k) {
            const double ang = -2.0 * M_PI * k / p->NX;
            w64[k] = make_double2(cos(ang), sin(ang));
            w32[k] = make_float2((float)cos(ang), (float)sin(ang));
        }
        st = upload_vec(p, &p->Wx64, w64, "Wx", s);
        if (st == EXPD_OK) st = upload_vec(p, &p->Wx32, w32, "Wx32", s);
        if (st == EXPD_OK && p->ndim == 2) {
            std::vector<double2> y64(std::max(1, p->NY / 2));
            std::vector<float2> y32(std::max(1, p->NY / 2));
            for (int k = 0; k < p->NY / 2; ++k) {
                const double ang = -2.0 * M_PI * k / p->NY;
                y64[k] = make_double2(cos(ang), sin(ang));
                y32[k] = make_float2((float)cos(ang), (float)sin(ang));
            }
            st = upload_vec(p, &p->Wy64, y64, "Wy", s);
            if (st == EXPD_OK) st = upload_vec(p, &p->Wy32, y32, "Wy32", s);
        }
    }
    // double-float copies of the twiddles and of Gamma_alpha / the output scale
    if (st == EXPD_OK && p->precision == EXPD_PREC_MIXED && p->bc == EXPD_BC_PERIODIC) {
        for (int d = 0; d < p->ndim && st == EXPD_OK; ++d) {
            const int n = d == 0 ? p->NX : p->NY;
            const int cnt = d == 0 ? n / 2 + 1 : std::max(1, n / 2);
            std::vector<float4> w(cnt);
            for (int k = 0; k < cnt; ++k) {
                const double ang = -2.0 * M_PI * k / n;
                const float2_pair c = split_dd(cos(ang)), sn = split_dd(sin(ang));
                w[k] = make_float4(c.hi, c.lo, sn.hi, sn.lo);
            }
            float4* dptr = nullptr;
            st = upload_vec(p, &dptr, w, "twiddles (double-float)", s);
            (d == 0 ? p->Wxdd : p->Wydd) = dptr;
        }
        if (st == EXPD_OK) {
            const TimeTablesHost th = time_tables_host(Nt - scheme->order + 1, alpha);
            const double extra = th.bluestein ? 1.0 / ((double)th.L * (double)th.L) : 1.0;
            std::vector<float2> g(th.gamma.size()), o(th.gamma.size());
            for (size_t n = 0; n < g.size(); ++n) {
                const float2_pair a = split_dd(th.gamma[n]);
                const float2_pair b = split_dd(extra / ((double)p->Ns * th.gamma[n]));
                g[n] = make_float2(a.hi, a.lo);
                o[n] = make_float2(b.hi, b.lo);
            }
            float2* gp = nullptr;
            float2* op = nullptr;
            st = upload_vec(p, &gp, g, "Gamma (double-float)", s);
            if (st == EXPD_OK) st = upload_vec(p, &op, o, "output scale (double-float)", s);
            p->gamdd = gp;
            p->oscdd = op;
        }
    }
    if (st == EXPD_OK && p->fast_dst) {
        for (int d = 0; d < p->ndim && st == EXPD_OK; ++d) {
            const int n = d == 0 ? p->NX : p->NY;
            const int N = 2 * (n + 1);
            std::vector<double2> t((size_t)N / 2);
            for (int k = 0; k < N / 2; ++k) t[k] = make_double2(cos(2.0 * M_PI * k / N), -sin(2.0 * M_PI * k / N));
            st = upload_vec(p, d == 0 ? &p->Dtx : &p->Dty, t, "fast DST twiddles", s);
        }
    } else if (st == EXPD_OK && p->bc == EXPD_BC_DIRICHLET) {
        for (int d = 0; d < p->ndim && st == EXPD_OK; ++d) {
            const int n = d == 0 ? p->NX : p->NY;
            std::vector<double> S((size_t)n * n);
            const double sc = sqrt(2.0 / (n + 1));
            for (int j = 0; j < n; ++j)
                for (int k = 0; k < n; ++k) {
                    const long long r = ((long long)(j + 1) * (k + 1)) % (2LL * (n + 1));
                    S[(size_t)j * n + k] = sc * sin(M_PI * (double)r / (n + 1));
                }
            st = upload_vec(p, d == 0 ? &p->Sx : &p->Sy, S, "DST matrix", s);
        }
        if (st == EXPD_OK && p->tc_dst) st = dst_tc_setup(p, s);
    } else if (st == EXPD_OK && p->bc == EXPD_BC_NEUMANN) {
        // orthonormal DCT-II C[k][j] = w_k cos(pi k (2j + 1)/(2n)), w_0 = sqrt(1/n),
        // w_k = sqrt(2/n): forward Y = C_y X C_x^T, inverse X = C_y^T Y C_x.
        // Sx = C_x^T and SxT = C_x are the right operands of the two
        // directions, Sy = C_y and SyT = C_y^T the left ones
        for (int d = 0; d < p->ndim && st == EXPD_OK; ++d) {
            const int n = d == 0 ? p->NX : p->NY;
            std::vector<double> Cm((size_t)n * n), Ct((size_t)n * n);
            for (int k = 0; k < n; ++k)
                for (int j = 0; j < n; ++j) {
                    const long long r = ((long long)k * (2 * j + 1)) % (4LL * n);  // angle pi r/(2n)
                    const double v = sqrt((k == 0 ? 1.0 : 2.0) / n) * cos(M_PI * (double)r / (2.0 * n));
                    Cm[(size_t)k * n + j] = v;
                    Ct[(size_t)j * n + k] = v;
                }
            if (d == 0) {
                st = upload_vec(p, &p->Sx, Ct, "DCT matrix", s);
                if (st == EXPD_OK) st = upload_vec(p, &p->SxT, Cm, "DCT matrix (inverse)", s);
            } else {
                st = upload_vec(p, &p->Sy, Cm, "DCT matrix", s);
                if (st == EXPD_OK) st = upload_vec(p, &p->SyT, Ct, "DCT matrix (inverse)", s);
            }
        }
    }
    // ---- state and workspace ----
    const size_t vec = (size_t)p->Ns * p->Mcol * p->esz;
    if (st == EXPD_OK) st = dalloc(p, &p->Uh, vec, "iterate");
    if (st == EXPD_OK) st = dalloc(p, &p->Fh, vec, "right-hand side");
    if (st == EXPD_OK) st = dalloc(p, &p->Sh, (size_t)p->order * p->Mcol * p->esz, "startup (eigen)");
    if (st == EXPD_OK)
        st = dalloc(p, reinterpret_cast<void**>(&p->startphys), (size_t)p->order * p->Mp * sizeof(double),
                    "startup (physical)");
    const size_t work = work64_bytes(p);
    if (st == EXPD_OK) st = dalloc(p, &p->work64, work, "work64");
    if (st == EXPD_OK && p->nonlin != EXPD_NL_NONE) {
        st = dalloc(p, &p->NL64, vec, "N (float64)");
        if (st == EXPD_OK && p->precision == EXPD_PREC_MIXED && p->bc == EXPD_BC_PERIODIC) {
            st = dalloc(p, &p->NL32, (size_t)p->Ns * p->Mcol * sizeof(float2), "N (float32)");
            if (st == EXPD_OK) st = dalloc(p, &p->work32, (size_t)p->Ns * p->NY * p->KX * sizeof(float2), "work32");
        }
    }
    // float32 sweeps of the mixed path: iterate and right-hand side in float32
    if (st == EXPD_OK && p->precision == EXPD_PREC_MIXED && (p->nonlin == EXPD_NL_NONE || p->bc == EXPD_BC_PERIODIC)) {
        st = dalloc(p, &p->U32, vec / 2, "iterate (float32)");
        if (st == EXPD_OK) st = dalloc(p, &p->F32, vec / 2, "right-hand side (float32)");
    }
    // norms: [8..] per-slice totals of the update and iterate norms (the host
    // or the device loop reduces them), then the device loop's state
    const size_t nred = 8 + 2 * (size_t)p->Ns + EXPD_CTL_DOUBLES + 1;
    if (st == EXPD_OK) st = dalloc(p, reinterpret_cast<void**>(&p->redout), nred * sizeof(double), "norms");
    if (st == EXPD_OK) {
        cudaError_t e = cudaMemsetAsync(p->redout, 0, nred * sizeof(double), s);
        if (e != cudaSuccess) st = expd_cuda_fail(e, "cudaMemsetAsync(norms)", __FILE__, __LINE__);
    }
    if (st == EXPD_OK) {
        p->redhost = pinned_acquire(pinned_words(p));
        p->phys_slot = reinterpret_cast<double**>(p->redout + nred - 1);
        if (p->redhost) {
            void* d = nullptr;
            const cudaError_t e = cudaHostGetDevicePointer(&d, p->redhost, 0);
            if (e != cudaSuccess) st = expd_cuda_fail(e, "cudaHostGetDevicePointer(norms)", __FILE__, __LINE__);
            p->redhost_dev = static_cast<double*>(d);
            // the last word: the cancel flag the tensor-core kernel polls
            const size_t cw = pinned_words(p) - 1;
            p->cancel_host = reinterpret_cast<volatile int*>(p->redhost + cw);
            *p->cancel_host = 0;
            if (p->redhost_dev) p->cancel_dev = reinterpret_cast<const int*>(p->redhost_dev + cw);
        }
        if (!p->redhost) st = expd_fail(EXPD_ERR_OOM, "pinned host memory for the norms");
    }
    if (st == EXPD_OK) st = time_tables_build(p, s);
    if (st == EXPD_OK) st = time_tc_setup(p, s);
    if (st != EXPD_OK) {
        free_plan(p);
        return st;
    }
    *out = p;
    return EXPD_OK;
}

expd_status expd_plan_footprint_bytes(const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                                      double alpha, const expd_scheme* scheme, int flags, size_t* bytes) {
    if (!bytes) return expd_fail(EXPD_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = 0;
    expd_plan_s pl;
    expd_plan p = &pl;
    expd_status st = plan_init_fields(p, grid, op, dt, Nt, alpha, scheme);
    if (st != EXPD_OK) return st;
    const size_t Mcol = (size_t)p->Mcol, Ns = (size_t)p->Ns, ord = (size_t)p->order;
    const bool per = p->bc == EXPD_BC_PERIODIC, mixed = p->precision == EXPD_PREC_MIXED;
    const bool nl = p->nonlin != EXPD_NL_NONE;
    const size_t vec = Ns * Mcol * p->esz;
    size_t b = 0;
    const size_t cw = p->adv ? 2 : 1;                                      // complex tables with advection
    b += cw * (Mcol * 8 + ord * Mcol * 8 + ord * Mcol * 4);                 // E, C64, C32
    if (mixed && per) b += cw * ord * Mcol * 8;                             // Cdd
    if (p->nl_form == EXPD_NLF_ETD1) b += Mcol * (8 + 4) + (mixed && per ? Mcol * 8 : 0);  // PHI64, PHI32, PHIdd
    if (per) {
        b += (size_t)(p->NX / 2 + 1) * (16 + 8);                            // Wx64, Wx32
        if (p->ndim == 2) b += (size_t)std::max(1, p->NY / 2) * (16 + 8);  // Wy64, Wy32
        if (mixed) {
            b += (size_t)(p->NX / 2 + 1) * 16;                              // Wxdd
            if (p->ndim == 2) b += (size_t)std::max(1, p->NY / 2) * 16;    // Wydd
            b += 2 * Ns * 8;                                                // gamdd, oscdd
        }
    } else if (p->fast_dst) {
        b += (size_t)(p->NX + 1) * 16;
        if (p->ndim == 2) b += (size_t)(p->NY + 1) * 16;
    } else {
        const size_t mats = p->bc == EXPD_BC_NEUMANN ? 2 : 1;                // DCT: forward and inverse
        b += mats * (size_t)p->NX * p->NX * 8;
        if (p->ndim == 2) b += mats * (size_t)p->NY * p->NY * 8;
        if (p->tc_dst) b += dst_tc_bytes(p);                                // tensor-core DST digits
    }
    b += 2 * vec + ord * Mcol * p->esz + ord * (size_t)p->Mp * 8;            // Uh, Fh, Sh, startphys
    b += work64_bytes(p);                                                   // work64
    if (nl) {
        b += vec;
        if (mixed && per) b += Ns * Mcol * 8 + Ns * p->NY * p->KX * 8;      // NL32, work32
    }
    if (mixed && (!nl || per)) b += vec;                                    // U32, F32
    b += (8 + 2 * Ns + EXPD_CTL_DOUBLES + 1) * 8;                           // norms, loop state, slot
    const TimeTablesHost th = time_tables_host(p->Ns, alpha);
    for (int q = 0; q < 2; ++q) {
        const size_t e = q == 0 ? 16 : 8, g = q == 0 ? 8 : 4;
        b += e * (th.tw.size()) + 16 + e * Ns + 16 + 2 * g * Ns;
        if (th.bluestein) b += e * Ns + 16 + 2 * (e * th.L + 16);
    }
    b += time_tc_bytes(p);                                                  // tensor-core time tables
    int grid_t = 0;
    st = time_grid_for(p, &grid_t);
    if (st != EXPD_OK) return st;
    b += (size_t)std::max(grid_t, p->sm_count * 8) * Ns * 16;              // norm partials
    if (flags & EXPD_FOOTPRINT_SOURCE) b += (size_t)p->Nt * Mcol * p->esz;
    if (flags & EXPD_FOOTPRINT_HOST) b += (size_t)(2 * p->Nt + 1) * p->Mp * 8;
    if (flags & EXPD_FOOTPRINT_GMRES) {
        const size_t n = (size_t)eigen_elems(p);
        const size_t grid = (size_t)p->sm_count * 4;
        b += (size_t)std::max(p->restart + 3, 7) * n * 8 + (p->cplx ? 256 + 131 * grid : 128 + 65 * grid) * 8;
    }
    *bytes = b;
    return EXPD_OK;
}

expd_status expd_plan_workspace_bytes(expd_plan p, size_t* bytes) {
    if (!p || !bytes) return expd_fail(EXPD_ERR_INVALID_ARG, "plan and bytes are required");
    *bytes = p->bytes;
    return EXPD_OK;
}

expd_status expd_timing_enable(expd_plan p, int enable) {
    if (!p) return expd_fail(EXPD_ERR_INVALID_ARG, "plan is NULL");
    p->timing = enable ? 1 : 0;
    return EXPD_OK;
}

expd_status expd_timing_read(expd_plan p, expd_timing* out, int reset) {
    if (!p || !out) return expd_fail(EXPD_ERR_INVALID_ARG, "plan and out are required");
    memset(out, 0, sizeof(*out));
    out->launches = p->launches;
    for (const auto& r : p->recs) {
        EXPD_CUDA_TRY(cudaEventSynchronize(p->events[r.e0 + 1]));
        float ms = 0.f;
        EXPD_CUDA_TRY(cudaEventElapsedTime(&ms, p->events[r.e0], p->events[r.e0 + 1]));
        if (r.cls < 0 || r.cls >= EXPD_NUM_KCLASS) continue;
        out->count[r.cls] += 1;
        out->ms[r.cls] += ms;
        out->bytes[r.cls] += r.bytes;
        out->flops[r.cls] += r.flops;
    }
    if (reset) {
        p->recs.clear();
        p->ev_used = 0;
        p->launches = 0;
    }
    return EXPD_OK;
}

expd_status expd_destroy(expd_plan p) {
    if (!p) return EXPD_OK;
    cudaStreamSynchronize(p->stream);  // the plan's last call has finished with its buffers
    free_plan(p);
    return EXPD_OK;
}

expd_status expd_residual(expd_plan p, const double* u0, const double* f, const double* U, double* R,
                          void* stream) {
    if (!p || !u0 || !U || !R) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, u0, U and R are required");
    if (f && p->nl_form == EXPD_NLF_ETD1) return expd_fail(EXPD_ERR_INVALID_ARG, "the ETD1 form takes no source term");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    const size_t M = (size_t)p->Mp;
    Staging sg;
    expd_status st = stage_in(p, u0, f, const_cast<double*>(U), p->Nt, true, sg, s);
    if (st != EXPD_OK) return st;
    // R may be host (or unaligned device) memory: compute into the staging
    // area or the caller's buffer
    const bool hR = needs_stage(R);
    double* Rd = R;
    if (hR) {
        st = ensure_stage(p);
        if (st != EXPD_OK) return st;
        Rd = p->stage + M;  // the source slot; f has been transformed before it is overwritten
    }
    const int saved = p->startup;
    p->startup = EXPD_STARTUP_GIVEN;
    st = setup_start(p, sg.u0, sg.f, sg.U, s);
    p->startup = saved;
    if (st != EXPD_OK) return st;
    st = spatial_forward64(p, sg.U + (size_t)(p->order - 1) * M, p->Uh, p->Ns, s);
    if (st != EXPD_OK) return st;
    TimeOp op;
    op.X = p->Uh;
    op.F = p->Fh;
    op.f_slices = p->f_slices;
    op.sigR = -1.0;
    op.precond = 0;
    op.out = p->Fh;  // in-place per tile: each tile is loaded before it is written
    if (p->nonlin != EXPD_NL_NONE) {
        st = nonlinear_eval(p, p->Uh, p->NL64, 0, s);
        // ETD1: dt phi_1(dt L) N of the previous slice
        if (st == EXPD_OK && p->nl_form == EXPD_NLF_ETD1) st = etd_shift(p, p->NL64, 0, s);
        if (st != EXPD_OK) return st;
        op.NL = p->NL64;
        op.bdt = p->nl_form == EXPD_NLF_ETD1 ? 1.0 : p->beta[p->order] * p->dt;
    }
    st = time_apply(p, op, s);
    if (st != EXPD_OK) return st;
    st = spatial_inverse64(p, p->Fh, Rd, p->Ns, s);
    if (st == EXPD_OK) st = dst_tc_check(p, s);
    if (st != EXPD_OK) return st;
    if (hR) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(R, Rd, (size_t)p->Ns * M * sizeof(double), cudaMemcpyDefault, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return EXPD_OK;
}

expd_status expd_precond_apply(expd_plan p, const double* R, double* S, void* stream) {
    if (!p || !R || !S) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, R and S are required");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    const size_t M = (size_t)p->Mp;
    const size_t bytes = (size_t)p->Ns * M * sizeof(double);
    const double* Rd = R;
    double* Sd = S;
    const bool hR = needs_stage(R), hS = needs_stage(S);
    if (hR || hS) {
        expd_status st = ensure_stage(p);
        if (st != EXPD_OK) return st;
    }
    if (hR) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(p->stage, R, bytes, cudaMemcpyDefault, s));
        Rd = p->stage;
    }
    if (hS) Sd = p->stage + (size_t)p->Nt * M;
    expd_status st = spatial_forward64(p, Rd, p->Fh, p->Ns, s);
    if (st != EXPD_OK) return st;
    TimeOp op;
    op.F = p->Fh;  // the transformed R: every slice
    op.precond = 1;
    op.out = p->Fh;
    op.f32 = p->precision == EXPD_PREC_MIXED;
    st = time_apply(p, op, s);
    if (st != EXPD_OK) return st;
    st = spatial_inverse64(p, p->Fh, Sd, p->Ns, s);
    if (st == EXPD_OK) st = dst_tc_check(p, s);
    if (st != EXPD_OK) return st;
    if (hS) {
        EXPD_CUDA_TRY(cudaMemcpyAsync(S, Sd, bytes, cudaMemcpyDefault, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return EXPD_OK;
}

expd_status expd_solve_fp(expd_plan p, const double* u0, const double* f, double* U, expd_info* info,
                          void* stream) {
    if (!p || !u0 || !U) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, u0 and U are required");
    if (f && p->nl_form == EXPD_NLF_ETD1) return expd_fail(EXPD_ERR_INVALID_ARG, "the ETD1 form takes no source term");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    expd_status st = call_begin(p, info, s);
    if (st != EXPD_OK) return st;
    Staging sg;
    st = stage_in(p, u0, f, U, p->Nt, u_is_input(p), sg, s);
    if (st != EXPD_OK) return st;
    const bool nl = p->nonlin != EXPD_NL_NONE;
    const bool etd = nl && p->nl_form == EXPD_NLF_ETD1;
    const bool mixed = p->precision == EXPD_PREC_MIXED;
    // the mixed path's right-hand side comes out of its assembly in float32
    // and, for the double-float phase, as double-float pairs
    const bool start32 = mixed && p->U32 != nullptr;
    const bool dd_rhs = start32 && p->bc == EXPD_BC_PERIODIC && p->Cdd != nullptr;
    st = setup_start(p, sg.u0, sg.f, sg.U, s, start32 ? static_cast<float*>(p->F32) : nullptr, dd_rhs ? 1 : 0);
    if (st != EXPD_OK) return st;
    const long long nelem = p->Mcol * (p->realcol ? 1 : 2);
    const long long nvec = (long long)p->Ns * nelem;
    // Mixed path: float32 sweeps (iterate, right-hand side, residual, N and the
    // preconditioner all in float32) until the estimated error reaches tol or
    // the float32 floor stops the contraction; then sweeps with an accurate
    // iterate, residual and N -- double-float (float hi + float lo, on the
    // float32 pipes) on periodic grids, float64 otherwise -- converge to the
    // float64 fixed point with the float32 preconditioner.
    enum { PH32, PHDD, PH64 };
    const bool use_dd = mixed && p->bc == EXPD_BC_PERIODIC && p->Cdd != nullptr;
    int phase = (mixed && p->U32 != nullptr) ? PH32 : PH64;
    // the initial iterate: the last start-up slice propagated by A, the
    // caller's (a checkpoint), or zero
    if (p->guess == EXPD_GUESS_LINEAR) {
        st = linear_guess(p, phase == PH32 ? p->U32 : p->Uh, phase == PH32, s);
        if (st != EXPD_OK) return st;
    } else if (p->guess == EXPD_GUESS_GIVEN) {
        st = load_guess(p, sg.U, p->Uh, s);
        if (st == EXPD_OK && phase == PH32)
            st = convert_f64_to_f32(p, static_cast<const double*>(p->Uh), static_cast<float*>(p->U32), nvec, s);
        if (st != EXPD_OK) return st;
    } else if (phase == PH32) {
        EXPD_CUDA_TRY(cudaMemsetAsync(p->U32, 0, (size_t)nvec * sizeof(float), s));
    } else {
        EXPD_CUDA_TRY(cudaMemsetAsync(p->Uh, 0, (size_t)nvec * sizeof(double), s));
    }
    // With EXPD_DEVICE_LOOP=1 the stopping test runs on the GPU (one graph per
    // solve, no host round trip per sweep) on a capturable stream once the
    // plan has run a solve (its first solve sets up every kernel outside
    // capture); otherwise the host reads the norms after every sweep.
    const bool device_loop = !p->timing && !p->no_graphs && !p->no_device_loop && s != nullptr &&
                             p->fp_solves > 0 && p->max_iter >= 1;
    // The host loop's first double-float sweep reads the float32 iterate itself
    // (exact in double-float) and writes X + s in double-float: no conversion
    // pass.  The same values as converting first, so results do not change.
    const bool x32_first = use_dd && !device_loop && time_reg_usable(p);
    bool dd_first = false;  // the next double-float sweep is the first
    // leave the float32 sweeps: the iterate (exact in float32) becomes the
    // accurate phase's starting point
    auto leave32 = [&]() -> expd_status {
        expd_status r = EXPD_OK;
        if (use_dd) {
            if (x32_first) dd_first = true;
            else r = convert_f32_to_dd(p, static_cast<const float*>(p->U32), p->Uh, nvec, s);  // Fh is double-float already
            phase = PHDD;
        } else {
            r = convert_f32_to_f64(p, static_cast<const float*>(p->U32), static_cast<double*>(p->Uh), nvec, s);
            phase = PH64;
        }
        return r;
    };
    // Output of a nonlinear double-float solve: the last sweep's N evaluation
    // leaves the physical iterate before that sweep's update in U (float64), and
    // its time kernel a float32 copy of the update s; U + inverse transform of
    // s in float32 is the solution (the update is orders of magnitude below U,
    // so float32 rounding of its transform is far below the tolerance), which
    // replaces the double-float output transform.
    // inexact Newton with the mean Jacobian at u_0: Step (b) solves with
    // (1 - beta dt nbar) I - ..., nbar = mean of N'(u_0) = 1 - 3 mean(u_0^2)
    double dshift = 0.0;
    if (nl && p->jacobian == EXPD_JAC_MEAN_U0) {
        double* scratch = reinterpret_cast<double*>(p->partial);  // free until the first time kernel
        st = sum_squares(p, p->startphys, p->M, p->redout, scratch, s);
        if (st != EXPD_OK) return st;
        EXPD_CUDA_TRY(cudaMemcpyAsync(p->redhost, p->redout, sizeof(double), cudaMemcpyDeviceToHost, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        const double nbar = 1.0 - 3.0 * p->redhost[0] / (double)p->M;
        dshift = p->beta[p->order] * p->dt * nbar;
    }
    double* phys_out = sg.U + (size_t)(p->order - 1) * p->Mp;
    const bool fast_out = use_dd && nl && inverse32_accum_supported(p);
    // the time operator of a sweep of phase ph (first: the first double-float
    // sweep reading the float32 iterate)
    auto make_op = [&](int ph, bool first = false) -> TimeOp {
        TimeOp op;
        op.X = ph == PH32 ? p->U32 : p->Uh;
        if (first) op.X32 = p->U32;  // read; X + s goes to Uh
        op.F = ph == PH32 ? p->F32 : p->Fh;
        op.f_slices = p->f_slices;
        op.sigR = -1.0;
        op.precond = 1;
        op.accum = 1;
        op.f32 = mixed;
        op.st32 = ph == PH32;
        op.stdd = ph == PHDD;
        op.dshift = dshift;
        if (nl && ph == PHDD && fast_out) op.sout = p->U32;  // free in this phase
        return op;
    };
    // one sweep: N(iterate) through the spatial transforms, the time kernel,
    // the per-slice reduction
    auto sweep = [&](int ph, bool first = false) -> expd_status {
        expd_status r = EXPD_OK;
        TimeOp o = make_op(ph, first);
        if (nl) {
            void* NL;
            if (ph == PH32) {
                NL = p->NL32;
                r = nonlinear_eval(p, o.X, NL, 1, s, 1);
                o.nl_f32 = 1;
            } else if (ph == PHDD) {
                NL = p->NL64;  // holds double-float values in this phase
                r = nonlinear_eval_dd(p, first ? o.X32 : o.X, NL, s, fast_out ? p->phys_slot : nullptr, first ? 1 : 0);
            } else {
                NL = p->NL64;
                r = nonlinear_eval(p, o.X, NL, 0, s, 0);
            }
            // ETD1: dt phi_1(dt L) N of the previous slice, in the phase's storage
            if (r == EXPD_OK && etd) r = etd_shift(p, NL, ph == PH32 ? 1 : ph == PHDD ? 2 : 0, s);
            if (r != EXPD_OK) return r;
            o.NL = NL;
            o.bdt = etd ? 1.0 : p->beta[p->order] * p->dt;
        }
        r = time_apply(p, o, s);
        if (r == EXPD_OK) r = time_reduce(p, s);
        return r;
    };
    const int acc_phase = use_dd ? PHDD : PH64;
    if (fast_out && p->phys_slot_value != phys_out) {  // the destination of the physical iterate
        set_slot_kernel<<<1, 1, 0, s>>>(p->phys_slot, phys_out);
        ++p->launches;
        EXPD_CUDA_TRY(cudaGetLastError());
        p->phys_slot_value = phys_out;
    }
    bool phys_valid = false;
    double last_rel = 1.0;
    double prev = 0.0, rho = 0.5, rho_phase = -1.0, measure = 1.0, s_first = 0.0;
    int it = 0, it32 = 0;
    expd_status result = EXPD_ERR_NOT_CONVERGED;
    ++p->fp_solves;
    st = call_mark(p, info, 1, s);
    if (st != EXPD_OK) return st;
    if (device_loop) {
        const bool two = phase == PH32;
        LoopBody b1{two ? 1 : 0, make_op(two ? PH32 : acc_phase).sout != nullptr ? 1 : 0};
        LoopBody b2{0, make_op(acc_phase).sout != nullptr ? 1 : 0};
        const int ph1 = two ? PH32 : acc_phase;
        auto convert = [&]() -> expd_status {
            return use_dd ? convert_f32_to_dd(p, static_cast<const float*>(p->U32), p->Uh, nvec, s)
                          : convert_f32_to_f64(p, static_cast<const float*>(p->U32), static_cast<double*>(p->Uh), nvec, s);
        };
        LoopCtl c;
        st = run_device_loop(p, s, two, b1, b2, nullptr, dshift, p->f_slices,
                             [&]() { return sweep(ph1); }, convert, [&]() { return sweep(acc_phase); }, &c);
        if (st != EXPD_OK) return st;
        phase = acc_phase;  // the conversion always follows the float32 loop
        it = c.it;
        it32 = c.it32;
        measure = c.measure;
        rho = c.rho;
        last_rel = c.last_rel;
        phys_valid = c.phys_valid != 0;
        if (info) {
            for (int i = 0; i < it && i < EXPD_MAX_HISTORY; ++i) info->history[i] = c.history[i];
            info->contraction = rho;
        }
        result = c.result == EXPD_ERR_DIVERGED ? expd_fail(EXPD_ERR_DIVERGED, "fixed-point update is non-finite or growing")
                                               : static_cast<expd_status>(c.result);
    } else {
    for (it = 1; it <= p->max_iter; ++it) {
        const bool used32 = phase == PH32;
        const int ph = phase;
        const bool first = ph == PHDD && dd_first;
        // graphs: one per phase, the double-float sweeps after the first apart
        st = run_sweep(p, ph == PHDD && !first ? 4 : ph, nullptr, dshift, p->f_slices, s,
                       [&]() { return sweep(ph, first); });
        if (st != EXPD_OK) return st;
        if (first) dd_first = false;
        phys_valid = make_op(ph).sout != nullptr;
        double nr[4];
        st = read_reduced_norms(p, s, nr);
        if (st != EXPD_OK) return st;
        if (used32) ++it32;
        const double smax = nr[0], umax = nr[1];
        last_rel = umax > 0 ? smax / umax : 1.0;
        if (it == 1) s_first = smax;
        if (!isfinite(smax) || !isfinite(umax) || !isfinite(nr[2]) || !isfinite(nr[3]) ||
            (it > 1 && smax > 1e3 * s_first)) {
            result = expd_fail(EXPD_ERR_DIVERGED, "fixed-point update is non-finite or growing");
            break;
        }
        const double rel = umax > 0 ? smax / umax : 0.0;
        if (it > 1 && prev > 0) {
            const double ratio = smax / prev;
            rho = std::min(0.95, std::max(1e-12, ratio));
        }
        // in the accurate phase after a float32 phase, the contraction is the
        // one observed before the float32 floor was reached
        const double r_use = (rho_phase > 0 && phase != PH32) ? rho_phase : rho;
        measure = it == 1 ? rel : rel * r_use / (1.0 - r_use);
        if (info && it <= EXPD_MAX_HISTORY) info->history[it - 1] = measure;
        if (info) info->contraction = rho;
        if (phase == PH32) {
            const bool stalled = it > 2 && rho > 0.5;
            // the next (accurate) sweep contracts the iterate's error and the
            // float32 rounding floor by rho: leave now if that is predicted to
            // reach the tolerance (the floor is taken as 4 float32 ulps, above
            // the 2-3 ulps the accurate sweep's first update measures)
            const double floor32 = 4.0 * 5.96e-8;
            const bool one_more = it > 2 && rho * (measure + floor32) <= p->tol;
            if (measure <= p->tol || stalled || one_more) {
                st = leave32();
                if (st != EXPD_OK) return st;
                if (!stalled) rho_phase = rho;
                else if (rho_phase < 0) rho_phase = 0.5;
            } else if (rho < 0.5) {
                rho_phase = rho;
            }
        } else if (measure <= p->tol) {
            result = EXPD_OK;
            prev = smax;
            break;
        }
        prev = smax;
        const expd_status stop = poll_stop(p);
        if (stop != EXPD_OK) {
            result = stop;
            break;
        }
    }
    if (it > p->max_iter) it = p->max_iter;
    if (phase == PH32) {
        st = leave32();
        if (st != EXPD_OK) return st;
    }
    if (dd_first) {  // no double-float sweep ran: the output reads the converted iterate
        st = convert_f32_to_dd(p, static_cast<const float*>(p->U32), p->Uh, nvec, s);
        if (st != EXPD_OK) return st;
        dd_first = false;
    }
    }
    if (info) {
        info->iterations = it;
        info->fp32_iterations = it32;
        info->final_measure = measure;
    }
    st = call_mark(p, info, 2, s);
    if (st != EXPD_OK) return st;
    if (phase == PHDD && phys_valid && last_rel <= 1e-4) {
        if (p->order > 1)
            EXPD_CUDA_TRY(cudaMemcpyAsync(sg.U, p->startphys + p->Mp, (size_t)(p->order - 1) * p->Mp * sizeof(double),
                                          cudaMemcpyDeviceToDevice, s));
        st = spatial_inverse32_accum(p, p->U32, phys_out, s);
    } else {
        st = write_solution(p, sg.U, s, phase == PHDD);
    }
    if (st != EXPD_OK) return st;
    st = stage_out(p, sg, s);
    if (st != EXPD_OK) return st;
    if (result == EXPD_ERR_NOT_CONVERGED) g_err = "max_iter reached before tol";
    return call_end(p, info, s, result);
}

// The Krylov block: nvec vectors of eigen_elems doubles, then the dot results
// and partials (128 + 65 x dots grid doubles).
// results and per-block partials of the Krylov dot products: up to 65 results
// (128 slots; 256 and twice the partials for a complex state's re/im pairs)
static size_t krylov_hblock(expd_plan p) {
    return p->cplx ? 256 + 131 * (size_t)(p->sm_count * 4) : 128 + 65 * (size_t)(p->sm_count * 4);
}

static expd_status ensure_krylov(expd_plan p, int nvec) {
    const size_t n = (size_t)eigen_elems(p);
    if (p->gm && p->gm_vecs >= nvec) return EXPD_OK;
    if (p->gm) {
        for (size_t i = 0; i < p->canaries.size(); ++i)
            if (p->canaries[i].first == p->gm) {
                p->canaries.erase(p->canaries.begin() + i);
                break;
            }
        plan_free(p, p->gm);
        p->bytes -= ((size_t)p->gm_vecs * n + krylov_hblock(p)) * sizeof(double);
        p->gm = nullptr;
        p->gm_vecs = 0;
    }
    expd_status st = dalloc(p, &p->gm, ((size_t)nvec * n + krylov_hblock(p)) * sizeof(double), "Krylov vectors");
    if (st == EXPD_OK) p->gm_vecs = nvec;
    return st;
}

expd_status expd_solve_sequential(expd_plan p, const double* u0, const double* f, double* U, void* stream) {
    if (!p || !u0 || !U) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, u0 and U are required");
    if (f && p->nl_form == EXPD_NLF_ETD1) return expd_fail(EXPD_ERR_INVALID_ARG, "the ETD1 form takes no source term");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    Staging sg;
    expd_status st = stage_in(p, u0, f, U, p->Nt, u_is_input(p), sg, s);
    if (st != EXPD_OK) return st;
    // u_0 .. u_{s-1} (the ramp or the given values) exactly as the all-at-once solve takes them
    st = setup_start(p, sg.u0, sg.f, sg.U, s);
    if (st != EXPD_OK) return st;
    const int so = p->order;
    const long long M = p->M;
    // eigen slice n: Sh for n < s, Uh for s <= n <= Nt
    auto slice = [&](int n) -> void* { return n < so ? eig_slice(p, p->Sh, n) : eig_slice(p, p->Uh, n - so); };
    const bool nl = p->nonlin != EXPD_NL_NONE;
    void* tmp = p->Fh;                             // eigen scratch (the right-hand side is not used here)
    double* phys = static_cast<double*>(p->NL64);  // physical scratch of M values (nonlinear plans)
    const double bdt = p->beta[so] * p->dt;
    auto steps = [&]() -> expd_status {
        expd_status r = EXPD_OK;
        if (nl && p->nl_form == EXPD_NLF_ETD1) {
            // ETD1: u_n = A u_{n-1} + dt phi_1(dt L) N(u_{n-1})
            for (int n = 1; n <= p->Nt && r == EXPD_OK; ++n) {
                r = spatial_inverse64(p, slice(n - 1), phys, 1, s);
                if (r == EXPD_OK) r = nonlinearity_eval_phys(p, phys, phys, M, s);
                if (r == EXPD_OK) r = spatial_forward64(p, phys, tmp, 1, s);
                if (r == EXPD_OK) r = etd_step(p, slice(n), slice(n - 1), tmp, s);
            }
            return r;
        }
        for (int n = so; n <= p->Nt && r == EXPD_OK; ++n) {
            // IF-BDF-s step: w = sum_j a_j A^j u_{n-j} + beta_s dt f(t_n), then
            // u_n = w (linear) or u_n - beta_s dt N(u_n) = w pointwise (Eq. (7.3))
            const void* in[6];
            double coef[6];
            for (int j = 1; j <= so; ++j) {
                in[j - 1] = slice(n - j);
                coef[j - 1] = p->acoef[so][j];
            }
            const void* src = f ? eig_slice(p, p->fh, n - 1) : nullptr;
            if (!nl) {
                r = eigen_combine(p, slice(n), in, coef, so, src, bdt, s);
            } else {
                r = eigen_combine(p, tmp, in, coef, so, src, bdt, s);
                if (r == EXPD_OK) r = spatial_inverse64(p, tmp, phys, 1, s);
                if (r == EXPD_OK) r = pointwise_solve(p, phys, phys, M, bdt, s);
                if (r == EXPD_OK) r = spatial_forward64(p, phys, slice(n), 1, s);
            }
        }
        return r;
    };
    // the Nt - s + 1 steps are launch-bound on small grids: one CUDA graph
    // (keyed by whether a source is present), like the fixed point's sweeps
    st = run_sweep(p, 3, f ? p->fh : nullptr, 0.0, 0, s, steps);
    if (st != EXPD_OK) return st;
    st = write_solution(p, sg.U, s);
    if (st != EXPD_OK) return st;
    return stage_out(p, sg, s);
}

expd_status expd_solve_gmres(expd_plan p, const double* u0, const double* f, double* U, expd_info* info,
                             void* stream) {
    if (!p || !u0 || !U) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, u0 and U are required");
    if (p->nonlin != EXPD_NL_NONE) return expd_fail(EXPD_ERR_INVALID_ARG, "GMRES needs a linear problem");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    expd_status st = call_begin(p, info, s);
    if (st != EXPD_OK) return st;
    const int m = p->restart;
    const long long n = eigen_elems(p);
    // mixed precision: the float32 preconditioner inside iterative refinement
    const bool mixed = p->precision == EXPD_PREC_MIXED;
    // block: V[0..m], c, w, then h/partials
    st = ensure_krylov(p, m + 3);
    if (st != EXPD_OK) return st;
    double* V = static_cast<double*>(p->gm);
    double* c = V + (size_t)(m + 1) * n;
    double* w = c + n;
    double* h = w + n;  // [128] results + partials
    Staging sg;
    st = stage_in(p, u0, f, U, p->Nt, u_is_input(p), sg, s);
    if (st != EXPD_OK) return st;
    st = setup_start(p, sg.u0, sg.f, sg.U, s);
    if (st != EXPD_OK) return st;
    st = call_mark(p, info, 1, s);
    if (st != EXPD_OK) return st;
    double* x = static_cast<double*>(p->Uh);
    if (p->guess == EXPD_GUESS_GIVEN) {
        st = load_guess(p, sg.U, x, s);  // resume from the caller's iterate
        if (st != EXPD_OK) return st;
    } else {
        EXPD_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    }

    // out = P^{-1} R v  (the preconditioned operator of Theorem 3.3)
    auto apply_op = [&](const double* v, double* out) -> expd_status {
        TimeOp op;
        op.X = v;
        op.sigR = 1.0;
        op.precond = 1;
        op.f32 = mixed;
        op.out = out;
        return time_apply(p, op, s);
    };
    // out = P^{-1} (f_s - R x): the residual in float64, then preconditioned,
    // in one pass of the time kernel
    auto residual_op = [&](double* out) -> expd_status {
        TimeOp op;
        op.F = p->Fh;
        op.f_slices = p->f_slices;
        op.X = x;
        op.sigR = -1.0;
        op.precond = 1;
        op.f32 = mixed;
        op.out = out;
        return time_apply(p, op, s);
    };
    auto dots = [&](const double* Vb, int k, const double* vec, double* hh) -> expd_status {
        expd_status r = gm_dots(p, Vb, n, k, vec, h, s);
        if (r != EXPD_OK) return r;
        EXPD_CUDA_TRY(cudaMemcpyAsync(hh, h, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        return EXPD_OK;
    };
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hh(m + 1), hh2(m + 1), y(m);
    // The relative preconditioned residual bounds the global relative error
    // (the eigenvalues of P^{-1}R lie within alpha/(1-alpha) of 1, Lemma 3.4);
    // the per-slice maximum of Sec. 7's error norm can exceed the global ratio
    // by at most sqrt(Ns), so GMRES stops at sqrt(Ns) * relres <= tol.
    const double tol_res = p->tol / sqrt((double)p->Ns);
    int total = 0, refinements = 0;
    double relres = 1.0, cn = 0.0;
    expd_status result = EXPD_ERR_NOT_CONVERGED;
    if (info) info->history[0] = 1.0;
    if (mixed) {
        // ---- float32 preconditioner, float64 residual refinement ----
        // The basis vectors are kept unnormalised: V_j = sc[j] v_j with the
        // orthonormal v_j, so the operator applies to V_j directly (it is
        // linear) and no pass rescales a vector.  On Dirichlet grids the time
        // kernel returns ||w||^2 and <V_j, w> of its output w = P^{-1} R V_j
        // (and ||out||^2 of a residual) from its epilogue; the norm of the
        // orthogonal part then follows from those exact dots of the same w,
        // ||w/sc_j - sum_i h_ij v_i||^2 = ||w||^2/sc_j^2 - sum_i h_ij^2, and the
        // next basis vector is formed only when the cycle continues.
        auto launch = [&](const double* X, const void* F, double sigR, double* out) -> expd_status {
            TimeOp op;
            op.X = X;
            op.F = F;
            op.f_slices = p->f_slices;
            op.sigR = sigR;
            op.precond = 1;
            op.f32 = 1;
            op.out = out;
            op.dots = 1;
            return time_apply(p, op, s);
        };
        // (||out||^2, <X, out>) of the last launch: fused partials, or dot passes
        auto out_dots = [&](const double* X, const double* out, double* oo, double* xo) -> expd_status {
            if (p->dots_fused) {
                expd_status r = time_reduce(p, s);
                if (r != EXPD_OK) return r;
                double nr[4];
                r = read_reduced_norms(p, s, nr);
                *oo = nr[2];
                *xo = nr[3];
                return r;
            }
            expd_status r = dots(out, 1, out, oo);
            if (r == EXPD_OK && X) r = dots(X, 1, out, xo);
            return r;
        };
        std::vector<double> sc(m + 1), hcol(m + 1), coef(m + 1);
        // c = P^{-1} f_s, the first cycle's residual (x = 0), into V_0
        st = launch(nullptr, p->Fh, 0.0, V);
        if (st != EXPD_OK) return st;
        double cn2 = 0, unused = 0;
        st = out_dots(nullptr, V, &cn2, &unused);
        if (st != EXPD_OK) return st;
        cn = sqrt(cn2);
        double beta = cn;
        bool first = p->guess != EXPD_GUESS_GIVEN;  // x = 0: the first residual is c
        while (cn > 0) {
            if (!first) {
                // r = P^{-1}(f_s - R x): the residual in float64, then preconditioned
                st = launch(x, p->Fh, -1.0, V);
                double b2 = 0;
                if (st == EXPD_OK) st = out_dots(x, V, &b2, &unused);
                if (st != EXPD_OK) return st;
                beta = sqrt(b2);
                ++refinements;
            }
            first = false;
            relres = beta / cn;
            if (!(relres == relres)) {
                result = expd_fail(EXPD_ERR_DIVERGED, "GMRES residual is non-finite");
                break;
            }
            if (relres <= tol_res) {
                result = EXPD_OK;
                break;
            }
            if (total >= p->max_iter) break;
            std::fill(g.begin(), g.end(), 0.0);
            g[0] = beta;
            sc[0] = beta;
            int jdone = 0;
            expd_status stop = EXPD_OK;
            for (int j = 0; j < m; ++j) {
                double* w = V + (size_t)(j + 1) * n;
                st = launch(V + (size_t)j * n, nullptr, 1.0, w);
                if (st != EXPD_OK) return st;
                double ww = 0, dj = 0;
                if (p->dots_fused) {
                    st = out_dots(V + (size_t)j * n, w, &ww, &dj);
                    if (st == EXPD_OK && j > 0) st = dots(V, j, w, hh.data());  // <V_i, w>, i < j
                } else {
                    st = dots(V, j + 1, w, hh.data());
                    if (st == EXPD_OK) st = dots(w, 1, w, &ww);
                    dj = hh[j];
                }
                if (st != EXPD_OK) return st;
                hh[j] = dj;
                const double wn = ww / (sc[j] * sc[j]);
                double orth = wn;
                for (int i = 0; i <= j; ++i) {
                    hcol[i] = hh[i] / (sc[i] * sc[j]);
                    H[(size_t)i * m + j] = hcol[i];
                    orth -= hcol[i] * hcol[i];
                }
                // the fused partials come from float32 products: below 2^-20 of
                // ||w||^2 the difference is rounding, so the orthogonal part is
                // taken at that resolution (the cycle then ends and the
                // recomputed float64 residual tells the truth)
                const double floor2 = p->dots_fused ? wn * 0x1p-20 : 0.0;
                const double hn = sqrt(orth > floor2 ? orth : floor2);
                H[(size_t)(j + 1) * m + j] = hn;
                for (int i = 0; i < j; ++i) {
                    const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
                    H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
                    H[(size_t)i * m + j] = t;
                }
                const double den = hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
                cs[j] = H[(size_t)j * m + j] / den;
                sn[j] = H[(size_t)(j + 1) * m + j] / den;
                H[(size_t)j * m + j] = den;
                H[(size_t)(j + 1) * m + j] = 0.0;
                g[j + 1] = -sn[j] * g[j];
                g[j] = cs[j] * g[j];
                ++total;
                jdone = j + 1;
                relres = fabs(g[j + 1]) / cn;
                if (info && total < EXPD_MAX_HISTORY) info->history[total] = relres;
                // the cycle ends once its residual fell by eta or claims
                // convergence; the restart recomputes it in float64
                if (relres <= tol_res || hn == 0 || fabs(g[j + 1]) <= p->krylov_eta * beta || j + 1 == m ||
                    total >= p->max_iter)
                    break;
                stop = poll_stop(p);
                if (stop != EXPD_OK) break;
                // V_{j+1} = (w - sum_i hcol_i (sc_j / sc_i) V_i) / (sc_j hn), of norm ~1
                for (int i = 0; i <= j; ++i) coef[i] = hcol[i] * sc[j] / sc[i];
                EXPD_CUDA_TRY(cudaMemcpyAsync(h + 64, coef.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
                st = gm_update_norm(p, V, n, j + 1, h + 64, 1.0 / (sc[j] * hn), w, h, s);
                double nn = 0;
                if (st == EXPD_OK) {
                    EXPD_CUDA_TRY(cudaMemcpyAsync(&nn, h, sizeof(double), cudaMemcpyDeviceToHost, s));
                    EXPD_CUDA_TRY(cudaStreamSynchronize(s));
                }
                if (st != EXPD_OK) return st;
                sc[j + 1] = sqrt(nn);
            }
            // x += sum_i y_i v_i = sum_i (y_i / sc_i) V_i,  H y = g
            for (int i = jdone - 1; i >= 0; --i) {
                double acc = g[i];
                for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * m + k] * y[k];
                y[i] = acc / H[(size_t)i * m + i];
            }
            for (int i = 0; i < jdone; ++i) hh[i] = -y[i] / sc[i];
            if (jdone > 0) {
                EXPD_CUDA_TRY(cudaMemcpyAsync(h, hh.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, s));
                st = gm_update(p, V, n, jdone, h, x, s);
                if (st != EXPD_OK) return st;
            }
            if (stop != EXPD_OK) {
                EXPD_CUDA_TRY(cudaStreamSynchronize(s));
                result = stop;
                break;
            }
        }
    } else if (p->cplx) {
        // ---- complex state: complex GMRES (float64) ----
        // The Hermitian inner product <v, w> = sum conj(v) w (its real part is
        // the plain dot product of the interleaved arrays), complex Hessenberg
        // entries, classical Gram-Schmidt with one re-orthogonalisation and
        // complex Givens rotations G = [[conj(c), s], [-s, c]], |c|^2 + s^2 = 1
        // with s real (the subdiagonal entry is a norm).
        typedef std::complex<double> cd;
        std::vector<double> tbuf(2 * (size_t)(m + 1));
        auto cdots = [&](const double* Vb, int k, const double* vec, cd* out) -> expd_status {
            expd_status r = gm_cdots(p, Vb, n, k, vec, h, s);
            if (r != EXPD_OK) return r;
            EXPD_CUDA_TRY(cudaMemcpyAsync(tbuf.data(), h, 2 * (size_t)k * sizeof(double), cudaMemcpyDeviceToHost, s));
            EXPD_CUDA_TRY(cudaStreamSynchronize(s));
            for (int i = 0; i < k; ++i) out[i] = cd(tbuf[2 * i], tbuf[2 * i + 1]);
            return EXPD_OK;
        };
        // x -= sum_i coef_i V_i
        auto cupdate = [&](const double* Vb, int k, const cd* coef, double* xv) -> expd_status {
            for (int i = 0; i < k; ++i) {
                tbuf[2 * i] = coef[i].real();
                tbuf[2 * i + 1] = coef[i].imag();
            }
            EXPD_CUDA_TRY(cudaMemcpyAsync(h, tbuf.data(), 2 * (size_t)k * sizeof(double), cudaMemcpyHostToDevice, s));
            return gm_cupdate(p, Vb, n, k, h, xv, s);
        };
        {
            TimeOp op;
            op.F = p->Fh;
            op.f_slices = p->f_slices;
            op.precond = 1;
            op.out = c;
            st = time_apply(p, op, s);
            if (st != EXPD_OK) return st;
        }
        double cn2 = 0;
        st = dots(c, 1, c, &cn2);
        if (st != EXPD_OK) return st;
        cn = sqrt(cn2);
        std::vector<cd> Hc((size_t)(m + 1) * m), csc(m), gc(m + 1), h1(m + 1), h2(m + 1), yc(m);
        std::vector<double> snc(m);
        bool first = p->guess != EXPD_GUESS_GIVEN;  // x = 0: the first residual is c
        while (cn > 0) {
            if (first) {
                EXPD_CUDA_TRY(cudaMemcpyAsync(V, c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
            } else {
                st = residual_op(V);
                if (st != EXPD_OK) return st;
            }
            first = false;
            double b2 = 0;
            st = dots(V, 1, V, &b2);
            if (st != EXPD_OK) return st;
            const double beta = sqrt(b2);
            relres = beta / cn;
            if (!(relres == relres)) {
                result = expd_fail(EXPD_ERR_DIVERGED, "GMRES residual is non-finite");
                break;
            }
            if (relres <= tol_res) {
                result = EXPD_OK;
                break;
            }
            if (total >= p->max_iter) break;
            st = gm_axpby(p, n, 1.0 / beta, V, 0.0, V, s);
            if (st != EXPD_OK) return st;
            std::fill(gc.begin(), gc.end(), cd(0.0));
            gc[0] = beta;
            int jdone = 0;
            bool conv = false;
            expd_status stop = EXPD_OK;
            for (int j = 0; j < m && total < p->max_iter; ++j) {
                double* vj1 = V + (size_t)(j + 1) * n;
                st = apply_op(V + (size_t)j * n, w);
                if (st != EXPD_OK) return st;
                st = cdots(V, j + 1, w, h1.data());
                if (st == EXPD_OK) st = cupdate(V, j + 1, h1.data(), w);
                if (st == EXPD_OK) st = cdots(V, j + 1, w, h2.data());
                if (st == EXPD_OK) st = cupdate(V, j + 1, h2.data(), w);
                if (st != EXPD_OK) return st;
                for (int i = 0; i <= j; ++i) Hc[(size_t)i * m + j] = h1[i] + h2[i];
                double wn2 = 0;
                st = dots(w, 1, w, &wn2);
                if (st != EXPD_OK) return st;
                const double hn = sqrt(wn2);
                Hc[(size_t)(j + 1) * m + j] = hn;
                if (hn > 0) {
                    st = gm_axpby(p, n, 1.0 / hn, w, 0.0, vj1, s);
                    if (st != EXPD_OK) return st;
                }
                for (int i = 0; i < j; ++i) {
                    const cd a0 = Hc[(size_t)i * m + j], a1 = Hc[(size_t)(i + 1) * m + j];
                    Hc[(size_t)i * m + j] = std::conj(csc[i]) * a0 + snc[i] * a1;
                    Hc[(size_t)(i + 1) * m + j] = -snc[i] * a0 + csc[i] * a1;
                }
                const cd hjj = Hc[(size_t)j * m + j];
                const double den = hypot(std::abs(hjj), hn);
                csc[j] = hjj / den;
                snc[j] = hn / den;
                Hc[(size_t)j * m + j] = den;
                Hc[(size_t)(j + 1) * m + j] = 0.0;
                gc[j + 1] = -snc[j] * gc[j];
                gc[j] = std::conj(csc[j]) * gc[j];
                ++total;
                jdone = j + 1;
                relres = std::abs(gc[j + 1]) / cn;
                if (info && total < EXPD_MAX_HISTORY) info->history[total] = relres;
                if (relres <= tol_res || hn == 0) {
                    conv = true;
                    break;
                }
                stop = poll_stop(p);
                if (stop != EXPD_OK) break;
            }
            // x += V y,  H y = g (back substitution); the update subtracts -y
            for (int i = jdone - 1; i >= 0; --i) {
                cd acc = gc[i];
                for (int k = i + 1; k < jdone; ++k) acc -= Hc[(size_t)i * m + k] * yc[k];
                yc[i] = acc / Hc[(size_t)i * m + i];
            }
            for (int i = 0; i < jdone; ++i) h1[i] = -yc[i];
            if (jdone > 0) {
                st = cupdate(V, jdone, h1.data(), x);
                if (st != EXPD_OK) return st;
            }
            EXPD_CUDA_TRY(cudaStreamSynchronize(s));
            if (stop != EXPD_OK) {
                result = stop;
                break;
            }
            if (conv) {
                result = EXPD_OK;
                break;
            }
        }
    } else {
    // c = P^{-1} f_s
    {
        TimeOp op;
        op.F = p->Fh;
        op.f_slices = p->f_slices;
        op.precond = 1;
        op.out = c;
        st = time_apply(p, op, s);
        if (st != EXPD_OK) return st;
    }
    double cn2 = 0;
    st = dots(c, 1, c, &cn2);
    if (st != EXPD_OK) return st;
    cn = sqrt(cn2);
    bool first = p->guess != EXPD_GUESS_GIVEN;  // x = 0: the first residual is c
    while (cn > 0) {
        // r = P^{-1}(f_s - R x)   (= c on the first cycle, x = 0)
        if (first) {
            EXPD_CUDA_TRY(cudaMemcpyAsync(V, c, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        } else {
            st = residual_op(V);
            if (st != EXPD_OK) return st;
        }
        first = false;
        double b2 = 0;
        st = dots(V, 1, V, &b2);
        if (st != EXPD_OK) return st;
        const double beta = sqrt(b2);
        relres = beta / cn;
        if (!(relres == relres)) {
            result = expd_fail(EXPD_ERR_DIVERGED, "GMRES residual is non-finite");
            break;
        }
        if (relres <= tol_res) {
            result = EXPD_OK;
            break;
        }
        if (total >= p->max_iter) break;
        st = gm_axpby(p, n, 1.0 / beta, V, 0.0, V, s);
        if (st != EXPD_OK) return st;
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int jdone = 0;
        bool conv = false;
        expd_status stop = EXPD_OK;
        for (int j = 0; j < m && total < p->max_iter; ++j) {
            double* vj1 = V + (size_t)(j + 1) * n;
            st = apply_op(V + (size_t)j * n, w);
            if (st != EXPD_OK) return st;
            // classical Gram-Schmidt with one re-orthogonalisation
            st = dots(V, j + 1, w, hh.data());
            if (st == EXPD_OK) st = gm_update(p, V, n, j + 1, h, w, s);
            if (st == EXPD_OK) st = dots(V, j + 1, w, hh2.data());
            if (st == EXPD_OK) st = gm_update(p, V, n, j + 1, h, w, s);
            if (st != EXPD_OK) return st;
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hh[i] + hh2[i];
            double wn2 = 0;
            st = dots(w, 1, w, &wn2);
            if (st != EXPD_OK) return st;
            const double hn = sqrt(wn2);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0) {
                st = gm_axpby(p, n, 1.0 / hn, w, 0.0, vj1, s);
                if (st != EXPD_OK) return st;
            }
            for (int i = 0; i < j; ++i) {
                const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = t;
            }
            const double den = hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
            cs[j] = H[(size_t)j * m + j] / den;
            sn[j] = H[(size_t)(j + 1) * m + j] / den;
            H[(size_t)j * m + j] = den;
            H[(size_t)(j + 1) * m + j] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            ++total;
            jdone = j + 1;
            relres = fabs(g[j + 1]) / cn;
            if (info && total < EXPD_MAX_HISTORY) info->history[total] = relres;
            if (relres <= tol_res || hn == 0) {
                conv = true;
                break;
            }
            stop = poll_stop(p);
            if (stop != EXPD_OK) break;
        }
        // x += V y,  H y = g
        for (int i = jdone - 1; i >= 0; --i) {
            double acc = g[i];
            for (int k = i + 1; k < jdone; ++k) acc -= H[(size_t)i * m + k] * y[k];
            y[i] = acc / H[(size_t)i * m + i];
        }
        for (int i = 0; i < jdone; ++i) hh[i] = -y[i];
        if (jdone > 0) {
            EXPD_CUDA_TRY(cudaMemcpyAsync(h, hh.data(), jdone * sizeof(double), cudaMemcpyHostToDevice, s));
            st = gm_update(p, V, n, jdone, h, x, s);
            if (st != EXPD_OK) return st;
        }
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        if (stop != EXPD_OK) {
            result = stop;
            break;
        }
        // float64 preconditioner: the recurrence's residual is the true one
        if (conv) {
            result = EXPD_OK;
            break;
        }
    }
    }
    if (cn == 0) result = EXPD_OK;
    if (info) {
        info->iterations = total;
        info->final_measure = relres;
        info->refinements = refinements;
    }
    st = call_mark(p, info, 2, s);
    if (st != EXPD_OK) return st;
    st = write_solution(p, sg.U, s);
    if (st != EXPD_OK) return st;
    st = stage_out(p, sg, s);
    if (st != EXPD_OK) return st;
    if (result == EXPD_ERR_NOT_CONVERGED) g_err = "max_iter reached before tol";
    return call_end(p, info, s, result);
}

expd_status expd_solve_bicgstab(expd_plan p, const double* u0, const double* f, double* U, expd_info* info,
                                void* stream) {
    if (!p || !u0 || !U) return expd_fail(EXPD_ERR_INVALID_ARG, "plan, u0 and U are required");
    if (p->nonlin != EXPD_NL_NONE) return expd_fail(EXPD_ERR_INVALID_ARG, "BiCGStab needs a linear problem");
    if (p->cplx) return expd_fail(EXPD_ERR_UNSUPPORTED, "BiCGStab takes real states (complex states: GMRES)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    EXPD_CUDA_TRY(plan_bind_stream(p, s));
    expd_status st = call_begin(p, info, s);
    if (st != EXPD_OK) return st;
    const long long n = eigen_elems(p);
    const bool mixed = p->precision == EXPD_PREC_MIXED;
    st = ensure_krylov(p, 7);
    if (st != EXPD_OK) return st;
    // [rhat][r] and [s][t] adjacent, so one dot kernel gives two products
    double* rhat = static_cast<double*>(p->gm);
    double* r = rhat + n;
    double* sv = r + n;
    double* t = sv + n;
    double* pv = t + n;
    double* v = pv + n;
    double* c = v + n;
    double* h = c + n;
    Staging sg;
    st = stage_in(p, u0, f, U, p->Nt, u_is_input(p), sg, s);
    if (st != EXPD_OK) return st;
    st = setup_start(p, sg.u0, sg.f, sg.U, s);
    if (st != EXPD_OK) return st;
    st = call_mark(p, info, 1, s);
    if (st != EXPD_OK) return st;
    double* x = static_cast<double*>(p->Uh);
    if (p->guess == EXPD_GUESS_GIVEN) {
        st = load_guess(p, sg.U, x, s);  // resume from the caller's iterate
        if (st != EXPD_OK) return st;
    } else {
        EXPD_CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), s));
    }
    auto apply_op = [&](const double* in, double* out) -> expd_status {  // out = P^{-1} R in
        TimeOp op;
        op.X = in;
        op.sigR = 1.0;
        op.precond = 1;
        op.f32 = mixed;
        op.out = out;
        return time_apply(p, op, s);
    };
    auto residual_op = [&](double* out) -> expd_status {  // out = P^{-1}(f_s - R x), residual in float64
        TimeOp op;
        op.F = p->Fh;
        op.f_slices = p->f_slices;
        op.X = x;
        op.sigR = -1.0;
        op.precond = 1;
        op.f32 = mixed;
        op.out = out;
        return time_apply(p, op, s);
    };
    auto dots = [&](const double* Vb, int k, const double* w, double* hh) -> expd_status {
        expd_status e = gm_dots(p, Vb, n, k, w, h, s);
        if (e != EXPD_OK) return e;
        EXPD_CUDA_TRY(cudaMemcpyAsync(hh, h, k * sizeof(double), cudaMemcpyDeviceToHost, s));
        EXPD_CUDA_TRY(cudaStreamSynchronize(s));
        return EXPD_OK;
    };
    auto copy = [&](const double* from, double* to) -> expd_status {
        EXPD_CUDA_TRY(cudaMemcpyAsync(to, from, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        return EXPD_OK;
    };
    // c = P^{-1} f_s;  r = rhat = c
    {
        TimeOp op;
        op.F = p->Fh;
        op.f_slices = p->f_slices;
        op.precond = 1;
        op.f32 = mixed;
        op.out = c;
        st = time_apply(p, op, s);
    }
    // r = P^{-1}(f_s - R x): c from x = 0, recomputed from a given iterate
    if (st == EXPD_OK) st = p->guess == EXPD_GUESS_GIVEN ? residual_op(r) : copy(c, r);
    if (st == EXPD_OK) st = copy(r, rhat);
    if (st == EXPD_OK) EXPD_CUDA_TRY(cudaMemsetAsync(pv, 0, 2 * n * sizeof(double), s));  // p, v
    if (st != EXPD_OK) return st;
    double cc = 0;
    st = dots(c, 1, c, &cc);
    if (st != EXPD_OK) return st;
    const double cn = sqrt(cc);
    // stop as GMRES does: sqrt(Ns) * ||P^{-1}(f - R v)|| / ||P^{-1} f|| <= tol
    const double tol_res = p->tol / sqrt((double)p->Ns);
    double rho = 1.0, alpha = 1.0, omega = 1.0, relres = 1.0;
    // mixed: norm of the residual at the last replacement; r is the recomputed
    // (true) residual right after a replacement
    double r_ref = cn;
    bool r_true = true;
    int it = 0, refinements = 0;
    expd_status result = EXPD_ERR_NOT_CONVERGED;
    if (info) info->history[0] = 1.0;
    while (cn > 0) {
        double d2[2];
        st = dots(rhat, 2, r, d2);  // (rhat, r), (r, r)
        if (st != EXPD_OK) return st;
        relres = sqrt(d2[1]) / cn;
        if (it > 0 && info && it < EXPD_MAX_HISTORY && !r_true) info->history[it] = relres;
        if (!(relres == relres) || relres > 1e12) {
            result = expd_fail(EXPD_ERR_DIVERGED, "BiCGStab residual non-finite or growing without bound");
            break;
        }
        // mixed: when the recurrence's residual has fallen by eta since the last
        // replacement, or claims convergence, replace it by the residual
        // recomputed in float64 and restart the recurrences from it
        if (mixed && !r_true && (relres <= tol_res || sqrt(d2[1]) <= p->krylov_eta * r_ref)) {
            st = residual_op(r);
            if (st == EXPD_OK) st = copy(r, rhat);
            if (st == EXPD_OK) EXPD_CUDA_TRY(cudaMemsetAsync(pv, 0, 2 * n * sizeof(double), s));
            if (st != EXPD_OK) return st;
            rho = alpha = omega = 1.0;
            r_true = true;
            ++refinements;
            continue;
        }
        if (mixed && r_true) r_ref = sqrt(d2[1]);
        r_true = false;
        if (relres <= tol_res) {
            result = EXPD_OK;
            break;
        }
        if (it >= p->max_iter) break;
        const expd_status stop = it > 0 ? poll_stop(p) : EXPD_OK;
        if (stop != EXPD_OK) {
            result = stop;
            break;
        }
        double rho_new = d2[0];
        if (rho_new == 0.0) {  // breakdown: restart the shadow residual from r
            st = copy(r, rhat);
            if (st == EXPD_OK) EXPD_CUDA_TRY(cudaMemsetAsync(pv, 0, 2 * n * sizeof(double), s));
            if (st != EXPD_OK) return st;
            rho = alpha = omega = 1.0;
            rho_new = d2[1];
        }
        const double beta = (rho_new / rho) * (alpha / omega);
        st = gm_axpby(p, n, -omega, v, 1.0, pv, s);             // p = r + beta (p - omega v)
        if (st == EXPD_OK) st = gm_axpby(p, n, 1.0, r, beta, pv, s);
        if (st == EXPD_OK) st = apply_op(pv, v);                // v = P^{-1} R p
        double rv = 0;
        if (st == EXPD_OK) st = dots(rhat, 1, v, &rv);
        if (st != EXPD_OK) return st;
        alpha = rho_new / rv;
        st = copy(r, sv);                                       // s = r - alpha v
        if (st == EXPD_OK) st = gm_axpby(p, n, -alpha, v, 1.0, sv, s);
        if (st == EXPD_OK) st = apply_op(sv, t);                // t = P^{-1} R s
        double d3[2];
        if (st == EXPD_OK) st = dots(sv, 2, t, d3);            // (s, t), (t, t)
        if (st != EXPD_OK) return st;
        omega = d3[1] > 0 ? d3[0] / d3[1] : 0.0;
        st = gm_axpby(p, n, alpha, pv, 1.0, x, s);              // x += alpha p + omega s
        if (st == EXPD_OK) st = gm_axpby(p, n, omega, sv, 1.0, x, s);
        if (st == EXPD_OK) st = copy(sv, r);                    // r = s - omega t
        if (st == EXPD_OK) st = gm_axpby(p, n, -omega, t, 1.0, r, s);
        if (st != EXPD_OK) return st;
        rho = rho_new;
        ++it;
    }
    if (cn == 0) result = EXPD_OK;
    if (info) {
        info->iterations = it;
        info->final_measure = relres;
        info->refinements = refinements;
    }
    st = call_mark(p, info, 2, s);
    if (st != EXPD_OK) return st;
    st = write_solution(p, sg.U, s);
    if (st != EXPD_OK) return st;
    st = stage_out(p, sg, s);
    if (st != EXPD_OK) return st;
    if (result == EXPD_ERR_NOT_CONVERGED) g_err = "max_iter reached before tol";
    return call_end(p, info, s, result);
}

expd_status expd_plan_cancel(expd_plan p) {
    if (!p) return expd_fail(EXPD_ERR_INVALID_ARG, "plan is NULL");
    p->cancel_req.store(1, std::memory_order_release);
    if (p->cancel_host) *p->cancel_host = 1;
    return EXPD_OK;
}

}  // extern "C"
