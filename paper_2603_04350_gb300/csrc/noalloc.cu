// expd_precond_apply_noalloc: the preconditioner solve of expd_precond_apply
// for callers that must not allocate device memory.
//
// Why it exists: some callers own all of the device's memory through an
// allocator of their own (a serving engine that reserves the free HBM up front,
// a framework memory pool) or run where an allocation could fail or stall in the
// middle of their work; they cannot create a plan, because a plan calls
// cudaMalloc.  This entry point builds everything a plan would hold -- the
// spectral tables, the eigen-space buffer, the spatial scratch and the per-slice
// norm partials of the time kernel -- inside one fixed file-scope device array.
//
// The array (EXPD_NOALLOC_SCRATCH_BYTES) lives in every GPU that loads the
// library until the process exits.  Host code cannot use the symbol itself (in
// host code it names a host-side stand-in), so a call looks up the array's
// device address with cudaGetSymbolAddress, with the call's device current:
// every call on a stream that is not being captured looks it up afresh (so a
// context torn down and re-created, e.g. after cudaDeviceReset, never leaves a
// stale address behind), and a call during stream capture, where the lookup
// may not run, uses the address the last uncaptured call on that device found.
// So the first call on a device must come before any stream capture.  Every
// call shares the array and leaves its contents behind; each call rewrites all
// of it that it reads, and calls that overlap on the GPU (on different streams
// or threads) race on it.
#include <math.h>

#include <mutex>

#include "common.cuh"
#include "plan.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[EXPD_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
char* g_scratch_addr[kMaxDevices] = {};

expd_status scratch_base(cudaStream_t s, char** base) {
    int dev = 0;
    EXPD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return expd_fail(EXPD_ERR_UNSUPPORTED, "device index out of range");
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusActive;  // undecidable: do not call into the runtime's symbol lookup
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return expd_cuda_fail(e, "cudaGetSymbolAddress(scratch)", __FILE__, __LINE__);
        g_scratch_addr[dev] = static_cast<char*>(ptr);
    } else if (!g_scratch_addr[dev]) {
        return expd_fail(EXPD_ERR_INVALID_ARG,
                         "the first allocation-free call on a device must come before any stream capture");
    }
    *base = g_scratch_addr[dev];
    return EXPD_OK;
}

// Bump allocator over the scratch array (256-byte aligned regions).
struct Carve {
    char* base;
    size_t used = 0;
    template <typename T>
    T* take(size_t count) {
        T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += ((count * sizeof(T) + 255) / 256) * 256;
        return p;
    }
};

// Spatial tables: E_m = exp(dt mu_m), FFT twiddles, DST-I matrices (float64,
// the same formulas expd_plan_create evaluates on the host).
struct BdfRow {
    double a[7];
    int order;
};

__global__ void spatial_tables_kernel(int bc, int ndim, int NX, int NY, double LX, double LY, double a, double c,
                                      double dt, int KX, long long Mcol, double* E, double* C64, float* C32,
                                      BdfRow bdf, double2* Wx64, float2* Wx32, double2* Wy64, float2* Wy32,
                                      double* Sx, double* Sy) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long m = t0; m < Mcol; m += stride) {
        const int kx = (int)(m % KX), ky = (int)(m / KX);
        double mu = -c;
        if (bc == EXPD_BC_PERIODIC) {
            const double wx = 2.0 * M_PI * kx / LX;
            mu -= a * wx * wx;
            if (ndim == 2) {
                const int kyf = ky <= NY / 2 ? ky : ky - NY;
                const double wy = 2.0 * M_PI * kyf / LY;
                mu -= a * wy * wy;
            }
        } else {
            const double hx = LX / (NX + 1);
            const double sx = sin(M_PI * (kx + 1) * hx / (2.0 * LX));
            mu -= a * (4.0 / (hx * hx)) * sx * sx;
            if (ndim == 2) {
                const double hy = LY / (NY + 1);
                const double sy = sin(M_PI * (ky + 1) * hy / (2.0 * LY));
                mu -= a * (4.0 / (hy * hy)) * sy * sy;
            }
        }
        E[m] = exp(dt * mu);
        for (int j = 1; j <= bdf.order; ++j) {
            const double cjm = bdf.a[j] * exp(j * dt * mu);
            C64[(long long)(j - 1) * Mcol + m] = cjm;
            C32[(long long)(j - 1) * Mcol + m] = (float)cjm;
        }
    }
    if (bc == EXPD_BC_PERIODIC) {
        for (long long k = t0; k <= NX / 2; k += stride) {
            double sn, cs;
            sincospi(-2.0 * (double)k / NX, &sn, &cs);
            Wx64[k] = make_double2(cs, sn);
            Wx32[k] = make_float2((float)cs, (float)sn);
        }
        if (ndim == 2)
            for (long long k = t0; k < NY / 2; k += stride) {
                double sn, cs;
                sincospi(-2.0 * (double)k / NY, &sn, &cs);
                Wy64[k] = make_double2(cs, sn);
                Wy32[k] = make_float2((float)cs, (float)sn);
            }
    } else {
        for (int d = 0; d < ndim; ++d) {
            const int n = d == 0 ? NX : NY;
            double* S = d == 0 ? Sx : Sy;
            const double sc = sqrt(2.0 / (n + 1));
            for (long long idx = t0; idx < (long long)n * n; idx += stride) {
                const long long j = idx / n, k = idx % n;
                const long long r = ((j + 1) * (k + 1)) % (2LL * (n + 1));
                S[idx] = sc * sinpi((double)r / (n + 1));
            }
        }
    }
}

// Time tables (both precisions): twiddles, lambda_n, Gamma_alpha, and for
// Bluestein the chirp and the FFT_L of the two convolution kernels, computed by
// one warp with the same shared-memory FFT the time kernel uses (its
// bit-reversed output order is the order the time kernel expects).
__global__ void time_tables_kernel(int Ns, double alpha, int L, int log2L, int bluestein, double* gam64,
                                   double* osc64, float* gam32, float* osc32, double2* tw64, float2* tw32,
                                   double2* lam64, float2* lam32, double2* ch64, float2* ch32, double2* bp64,
                                   float2* bp32, double2* bm64, float2* bm32) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* stw = reinterpret_cast<double2*>(smem_raw);  // [L/2]
    double2* sb = stw + (L / 2 > 0 ? L / 2 : 1);           // [L]
    const double ar = pow(alpha, 1.0 / Ns);
    for (int k = threadIdx.x; k < L / 2; k += blockDim.x) {
        double sn, cs;
        sincospi(-2.0 * (double)k / L, &sn, &cs);
        stw[k] = make_double2(cs, sn);
        tw64[k] = stw[k];
        tw32[k] = make_float2((float)cs, (float)sn);
    }
    for (int k = threadIdx.x; k < Ns; k += blockDim.x) {
        double sn, cs;
        sincospi(2.0 * (double)k / Ns, &sn, &cs);
        lam64[k] = make_double2(ar * cs, ar * sn);
        lam32[k] = make_float2((float)(ar * cs), (float)(ar * sn));
        const double g = pow(alpha, (double)k / Ns);
        const double o = (bluestein ? 1.0 / ((double)L * (double)L) : 1.0) / ((double)Ns * g);
        gam64[k] = g;
        osc64[k] = o;
        gam32[k] = (float)g;
        osc32[k] = (float)o;
        if (bluestein) {
            const long long r = ((long long)k * k) % (2LL * Ns);
            sincospi((double)r / Ns, &sn, &cs);
            ch64[k] = make_double2(cs, sn);
            ch32[k] = make_float2((float)cs, (float)sn);
        }
    }
    if (!bluestein) return;
    __syncthreads();
    if (threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: kernel conj(c_j) (forward, + sign); pass 1: c_j (inverse, - sign)
        for (int j = lane; j < L; j += 32) sb[j] = make_double2(0.0, 0.0);
        __syncwarp();
        for (int j = lane; j < Ns; j += 32) {
            double2 cj = ch64[j];
            if (pass == 0) cj.y = -cj.y;
            sb[j] = cj;
            if (j > 0) sb[L - j] = cj;
        }
        __syncwarp();
        fft_dif(sb, log2L, stw, 1, -1, lane, 32);
        double2* o64 = pass == 0 ? bp64 : bm64;
        float2* o32 = pass == 0 ? bp32 : bm32;
        for (int j = lane; j < L; j += 32) {
            o64[j] = sb[j];
            o32[j] = make_float2((float)sb[j].x, (float)sb[j].y);
        }
        __syncwarp();
    }
}

}  // namespace

extern "C" expd_status expd_precond_apply_noalloc(const expd_grid* grid, const expd_operator* op, double dt, int Nt,
                                                  double alpha, const expd_scheme* scheme, const double* R, double* S,
                                                  void* stream) {
    expd_clear_error();
    if (!R || !S) return expd_fail(EXPD_ERR_INVALID_ARG, "R and S are required");
    if (!expd_is_device_ptr(R) || !expd_is_device_ptr(S))
        return expd_fail(EXPD_ERR_INVALID_ARG, "R and S must be device pointers (host buffers would need staging)");
    if (((reinterpret_cast<uintptr_t>(R) | reinterpret_cast<uintptr_t>(S)) & 15u) != 0)
        return expd_fail(EXPD_ERR_INVALID_ARG, "R and S must be 16-byte aligned (unaligned buffers would need staging)");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    expd_plan_s pl;  // plan fields on the stack; every buffer below points into the scratch array
    expd_plan p = &pl;
    expd_status st = plan_init_fields(p, grid, op, dt, Nt, alpha, scheme);
    if (st != EXPD_OK) return st;
    if (p->cplx) return expd_fail(EXPD_ERR_UNSUPPORTED, "the no-allocation entry point takes real states");
    if (p->bc == EXPD_BC_NEUMANN)
        return expd_fail(EXPD_ERR_UNSUPPORTED, "the no-allocation entry point takes periodic and Dirichlet grids");
    if (p->adv) return expd_fail(EXPD_ERR_UNSUPPORTED, "the no-allocation entry point has no advection tables");
    p->fast_dst = 0;  // Dirichlet transforms use the dense sine matrices built below
    p->tc_dst = 0;    // (in float64: the tensor-core digits would need device memory of their own)
    int L = 1;
    while (L < p->Ns) L <<= 1;
    const int blue = (L != p->Ns);
    if (blue) {
        L = 1;
        while (L < 2 * p->Ns - 1) L <<= 1;
    }
    if (L > 1024) return expd_fail(EXPD_ERR_UNSUPPORTED, "the allocation-free entry point takes at most 512 slices");
    int tgrid = 0;
    st = time_grid_for(p, &tgrid);
    if (st != EXPD_OK) return st;

    // ---- layout of the scratch array (first pass sizes it, second carves it) ----
    char* base = nullptr;
    for (int pass = 0; pass < 2; ++pass) {
        Carve cv{pass == 0 ? nullptr : base};
        p->E = cv.take<double>(p->Mcol);
        p->C64 = cv.take<double>((size_t)p->order * p->Mcol);
        p->C32 = cv.take<float>((size_t)p->order * p->Mcol);
        if (p->bc == EXPD_BC_PERIODIC) {
            p->Wx64 = cv.take<double2>(p->NX / 2 + 1);
            p->Wx32 = cv.take<float2>(p->NX / 2 + 1);
            if (p->ndim == 2) {
                p->Wy64 = cv.take<double2>(p->NY / 2);
                p->Wy32 = cv.take<float2>(p->NY / 2);
            }
        } else {
            p->Sx = cv.take<double>((size_t)p->NX * p->NX);
            if (p->ndim == 2) p->Sy = cv.take<double>((size_t)p->NY * p->NY);
        }
        TimeTables* tt[2] = {&p->t64, &p->t32};
        for (int q = 0; q < 2; ++q) {
            const size_t e = q == 0 ? sizeof(double2) : sizeof(float2);
            TimeTables& t = *tt[q];
            t.L = L;
            t.log2L = ilog2(L);
            t.bluestein = blue;
            t.gam = cv.take<char>(e / 2 * p->Ns);
            t.osc = cv.take<char>(e / 2 * p->Ns);
            t.tw = cv.take<char>(e * (L / 2 > 0 ? L / 2 : 1));
            t.lam = cv.take<char>(e * p->Ns);
            t.chirp = blue ? cv.take<char>(e * p->Ns) : nullptr;
            t.bplus = blue ? cv.take<char>(e * L) : nullptr;
            t.bminus = blue ? cv.take<char>(e * L) : nullptr;
        }
        p->partial = cv.take<double2>((size_t)tgrid * p->Ns);
        p->Fh = cv.take<char>((size_t)p->Ns * p->Mcol * p->esz);
        p->work64 = cv.take<double2>((size_t)p->Ns * p->NY * p->KX);
        if (pass == 0) {
            if (cv.used > (size_t)EXPD_NOALLOC_SCRATCH_BYTES)
                return expd_fail(EXPD_ERR_INVALID_ARG,
                                 "problem needs " + std::to_string(cv.used) + " bytes of scratch; the allocation-free "
                                 "entry point holds " + std::to_string((size_t)EXPD_NOALLOC_SCRATCH_BYTES));
            st = scratch_base(s, &base);
            if (st != EXPD_OK) return st;
        }
    }
    p->time_grid = tgrid;
    p->partial_cap = tgrid;

    // ---- tables, then the three steps around the spatial transforms ----
    {
        KProf kp(p, s, EXPD_K_POINTWISE, 8.0 * (double)p->Mcol, 0.0);
        BdfRow bdf;
        for (int j = 0; j < 7; ++j) bdf.a[j] = p->acoef[p->order][j];
        bdf.order = p->order;
        spatial_tables_kernel<<<p->sm_count * 4, 256, 0, s>>>(p->bc, p->ndim, p->NX, p->NY, p->LX, p->LY, p->a, p->c,
                                                              p->dt, p->KX, p->Mcol, p->E, p->C64, p->C32, bdf,
                                                              p->Wx64, p->Wx32, p->Wy64, p->Wy32, p->Sx, p->Sy);
        EXPD_CUDA_TRY(cudaGetLastError());
    }
    {
        KProf kp(p, s, EXPD_K_POINTWISE, 64.0 * L, 0.0);
        const size_t smem = (size_t)((L / 2 > 0 ? L / 2 : 1) + L) * sizeof(double2);
        time_tables_kernel<<<1, 256, smem, s>>>(
            p->Ns, p->alpha, L, ilog2(L), blue, static_cast<double*>(p->t64.gam), static_cast<double*>(p->t64.osc),
            static_cast<float*>(p->t32.gam), static_cast<float*>(p->t32.osc), static_cast<double2*>(p->t64.tw),
            static_cast<float2*>(p->t32.tw), static_cast<double2*>(p->t64.lam), static_cast<float2*>(p->t32.lam),
            static_cast<double2*>(p->t64.chirp), static_cast<float2*>(p->t32.chirp), static_cast<double2*>(p->t64.bplus),
            static_cast<float2*>(p->t32.bplus), static_cast<double2*>(p->t64.bminus), static_cast<float2*>(p->t32.bminus));
        EXPD_CUDA_TRY(cudaGetLastError());
    }
    st = spatial_forward64(p, R, p->Fh, p->Ns, s);
    if (st != EXPD_OK) return st;
    TimeOp opr;
    opr.F = p->Fh;
    opr.precond = 1;
    opr.out = p->Fh;
    opr.f32 = p->precision == EXPD_PREC_MIXED;
    st = time_apply(p, opr, s);
    if (st != EXPD_OK) return st;
    return spatial_inverse64(p, p->Fh, S, p->Ns, s);
}
