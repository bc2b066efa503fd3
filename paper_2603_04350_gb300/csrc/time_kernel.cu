// Time direction of the hot path, in L_h's eigenbasis where every spatial mode m
// decouples into one column of Ns time values.  One fused kernel computes, per
// column,
//
//   q_n  = F_n + bdt*NL_n + sigR*(X_n - sum_{j=1..s, n-j>=0} a_j E_m^j X_{n-j})
//          (the all-at-once residual f_s + beta dt N(v) - R_s v of Eq. (3.2),
//           or R_s X for the GMRES operator; float64)
//   s    = (R_s^alpha)^{-1} q by Eq. (3.3) / Eq. (4.5):
//          Step (a)  Y_k = sum_n alpha^(n/Ns) q_n e^{+2 pi i kn/Ns}
//          Step (b)  Z_k = Y_k / (1 - sum_j a_j (lambda_k E_m)^j),
//                    lambda_k = alpha^(1/Ns) e^{2 pi i k/Ns}  (Sec. 2, Sec. 4)
//          Step (c)  s_n = alpha^(-n/Ns) (1/Ns) sum_k Z_k e^{-2 pi i kn/Ns}
//   X   += s (Richardson update, Eq. (3.2) / Eq. (4.4)) or out = s
//
// and accumulates per-slice norms of s and of the updated X.
//
// Layout: the eigen arrays are [Ns][Mcol] (slice-major).  A CTA owns a tile of
// EXPD_TIME_COLS consecutive modes and all Ns slices: the tile is loaded with
// coalesced reads along the mode index into shared memory, each warp then
// transforms one column in shared memory (radix-2 FFT for power-of-two Ns,
// Bluestein's chirp-z with a power-of-two length otherwise), and the tile is
// written back coalesced.  The grid is a multiple of the SM count and loops
// over tiles in a fixed order, so the per-slice norm partials are deterministic.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include <type_traits>

#include "common.cuh"
#include "plan.h"
#include "time_column.cuh"

namespace {

struct TimeArgs {
    const void* X;
    const void* F;
    const void* NL;
    void* out;
    int nl_f32;
    double bdt, sigR;
    int precond, accum;
    long long Mcol;
    int Ns, order;
    double a[7];
    const double* E;
    int KX, NX, realcol;
    const double* gamma;
    const void* lam;
    const void* tw;
    const void* chirp;
    const void* bplus;
    const void* bminus;
    int L, log2L, bluestein;
    long long ntiles;
    double2* partial;
};

template <bool REAL>
__device__ __forceinline__ double2 ldcol(const void* p, long long i) {
    if (REAL) return make_double2(static_cast<const double*>(p)[i], 0.0);
    return static_cast<const double2*>(p)[i];
}
template <bool REAL>
__device__ __forceinline__ void stcol(void* p, long long i, double2 v) {
    if (REAL) static_cast<double*>(p)[i] = v.x;
    else static_cast<double2*>(p)[i] = v;
}
template <bool REAL>
__device__ __forceinline__ double2 ldnl(const void* p, long long i, int f32) {
    if (REAL) {
        return make_double2(f32 ? (double)static_cast<const float*>(p)[i] : static_cast<const double*>(p)[i], 0.0);
    }
    return f32 ? to_c64(static_cast<const float2*>(p)[i]) : static_cast<const double2*>(p)[i];
}

__device__ __forceinline__ double mode_weight(long long m, int KX, int NX, int realcol) {
    if (realcol) return 1.0;
    const int kx = (int)(m % KX);
    return (kx == 0 || 2 * kx == NX) ? 1.0 : 2.0;
}

template <typename PT, bool REAL>
__global__ void __launch_bounds__(32 * EXPD_TIME_COLS) time_kernel(TimeArgs A) {
    typedef typename cplx<PT>::t PT2;
    constexpr int C = EXPD_TIME_COLS;
    const int Ns = A.Ns, L = A.L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // ---- shared-memory carve-up (all offsets 16-byte aligned) ----
    double2* sX = reinterpret_cast<double2*>(smem_raw);        // [Ns][C]
    double2* sR = sX + (size_t)Ns * C;                          // [Ns][C]
    double2* sAcc = sR + (size_t)Ns * C;                        // [Ns]
    PT2* sW = reinterpret_cast<PT2*>(sAcc + Ns);                // [C][L]
    PT2* tw = sW + (size_t)C * L;                               // [L/2]
    PT2* lam = tw + (L >> 1);                                   // [Ns]
    PT2* chirp = lam + ((Ns + 1) & ~1);                         // [Ns]   (Bluestein)
    PT2* bp = chirp + (A.bluestein ? ((Ns + 1) & ~1) : 0);      // [L]
    PT2* bm = bp + (A.bluestein ? L : 0);                       // [L]
    double* gam = reinterpret_cast<double*>(bm + (A.bluestein ? L : 0));  // [Ns]

    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = tid; i < (L >> 1); i += nth) tw[i] = static_cast<const PT2*>(A.tw)[i];
    for (int i = tid; i < Ns; i += nth) {
        lam[i] = static_cast<const PT2*>(A.lam)[i];
        gam[i] = A.gamma[i];
        sAcc[i] = make_double2(0.0, 0.0);
        if (A.bluestein) chirp[i] = static_cast<const PT2*>(A.chirp)[i];
    }
    if (A.bluestein)
        for (int i = tid; i < L; i += nth) {
            bp[i] = static_cast<const PT2*>(A.bplus)[i];
            bm[i] = static_cast<const PT2*>(A.bminus)[i];
        }
    __syncthreads();

    const int lane = tid & 31, warp = tid >> 5;
    const long long Mcol = A.Mcol;
    for (long long tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const long long m0 = tile * C;
        // ---- coalesced load of the tile: X and the additive right-hand side ----
        for (int idx = tid; idx < Ns * C; idx += nth) {
            const int n = idx / C, c = idx - n * C;
            const long long m = m0 + c;
            double2 x = make_double2(0.0, 0.0), r = make_double2(0.0, 0.0);
            if (m < Mcol) {
                const long long g = (long long)n * Mcol + m;
                if (A.X) x = ldcol<REAL>(A.X, g);
                if (A.F) r = ldcol<REAL>(A.F, g);
                if (A.NL) {
                    const double2 v = ldnl<REAL>(A.NL, g, A.nl_f32);
                    r.x = fma(A.bdt, v.x, r.x);
                    r.y = fma(A.bdt, v.y, r.y);
                }
            }
            sX[idx] = x;
            sR[idx] = r;
        }
        __syncthreads();

        // ---- one warp per column ----
        const long long m = m0 + warp;
        if (warp < C && m < Mcol) {
            const double Em = A.E[m];
            double cj[7];
            {
                double Ej = 1.0;
                for (int j = 1; j <= A.order; ++j) {
                    Ej *= Em;
                    cj[j] = A.a[j] * Ej;
                }
            }
            PT2* w = sW + (size_t)warp * L;
            // residual-type combination q_n (float64), then Gamma_alpha
            for (int n = lane; n < Ns; n += 32) {
                double2 q = sR[n * C + warp];
                if (A.X) {
                    double2 rx = sX[n * C + warp];
                    for (int j = 1; j <= A.order && j <= n; ++j) {
                        const double2 xv = sX[(n - j) * C + warp];
                        rx.x = fma(-cj[j], xv.x, rx.x);
                        rx.y = fma(-cj[j], xv.y, rx.y);
                    }
                    q.x = fma(A.sigR, rx.x, q.x);
                    q.y = fma(A.sigR, rx.y, q.y);
                }
                if (!A.precond) {
                    sR[n * C + warp] = q;
                } else {
                    const PT2 y = from_c64<PT2>(cscale(q, gam[n]));
                    w[A.bluestein ? n : (int)bitrev(n, A.log2L)] = y;
                }
            }
            if (A.precond) {
                EXPD_SYNCWARP();
                const double scale_all = precond_column<PT, PT2>(w, Ns, L, A.log2L, A.bluestein, tw, lam, chirp,
                                                                 bp, bm, cj, A.order, lane, 32);
                for (int n = lane; n < Ns; n += 32) {
                    const double2 v = to_c64(w[A.bluestein ? n : (int)bitrev(n, A.log2L)]);
                    sR[n * C + warp] = cscale(v, scale_all / gam[n]);
                }
            }
        }
        __syncthreads();

        // ---- coalesced write-back and per-slice norms ----
        for (int idx = tid; idx < Ns * C; idx += nth) {
            const int n = idx / C, c = idx - n * C;
            const long long mm = m0 + c;
            double2 nrm = make_double2(0.0, 0.0);
            if (mm < Mcol) {
                const long long g = (long long)n * Mcol + mm;
                const double2 res = sR[idx];
                const double wgt = mode_weight(mm, A.KX, A.NX, A.realcol);
                nrm.x = wgt * (res.x * res.x + res.y * res.y);
                if (A.accum) {
                    const double2 xn = cadd(sX[idx], res);
                    stcol<REAL>(const_cast<void*>(A.X), g, xn);
                    nrm.y = wgt * (xn.x * xn.x + xn.y * xn.y);
                } else {
                    stcol<REAL>(A.out, g, res);
                }
            }
            sX[idx] = nrm;
        }
        __syncthreads();
        for (int n = tid; n < Ns; n += nth) {
            double2 acc = sAcc[n];
            for (int c = 0; c < C; ++c) {
                acc.x += sX[n * C + c].x;
                acc.y += sX[n * C + c].y;
            }
            sAcc[n] = acc;
        }
        __syncthreads();
    }
    for (int n = tid; n < Ns; n += nth) A.partial[(size_t)blockIdx.x * Ns + n] = sAcc[n];
}

// max that propagates NaN (fmax would drop it and hide a diverged iterate)
__device__ __forceinline__ double nanmax(double a, double b) { return (a != a || b != b) ? NAN : fmax(a, b); }

// Per-slice totals over the CTAs (fixed order), then max/sum over slices.
__global__ void reduce_kernel(const double2* __restrict__ partial, int grid, int Ns, double* __restrict__ out) {
    __shared__ double smax[2][32], ssum[2][32];
    double mx0 = 0, mx1 = 0, sm0 = 0, sm1 = 0;
    for (int n = threadIdx.x; n < Ns; n += blockDim.x) {
        double a = 0, b = 0;
        for (int g = 0; g < grid; ++g) {
            const double2 v = partial[(size_t)g * Ns + n];
            a += v.x;
            b += v.y;
        }
        mx0 = nanmax(mx0, a);
        mx1 = nanmax(mx1, b);
        sm0 += a;
        sm1 += b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx0 = nanmax(mx0, __shfl_xor_sync(0xffffffffu, mx0, o));
        mx1 = nanmax(mx1, __shfl_xor_sync(0xffffffffu, mx1, o));
        sm0 += __shfl_xor_sync(0xffffffffu, sm0, o);
        sm1 += __shfl_xor_sync(0xffffffffu, sm1, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        smax[0][warp] = mx0;
        smax[1][warp] = mx1;
        ssum[0][warp] = sm0;
        ssum[1][warp] = sm1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0, d = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            a = nanmax(a, smax[0][w]);
            b = nanmax(b, smax[1][w]);
            c += ssum[0][w];
            d += ssum[1][w];
        }
        out[0] = sqrt(a);
        out[1] = sqrt(b);
        out[2] = c;
        out[3] = d;
    }
}

size_t time_smem_bytes(int Ns, int L, int bluestein, size_t pt2) {
    const int C = EXPD_TIME_COLS;
    size_t b = (size_t)(2 * Ns * C + Ns) * sizeof(double2);
    b += (size_t)C * L * pt2 + (size_t)(L / 2) * pt2 + (size_t)((Ns + 1) & ~1) * pt2;
    if (bluestein) b += (size_t)((Ns + 1) & ~1) * pt2 + 2 * (size_t)L * pt2;
    b += (size_t)Ns * sizeof(double);
    return b;
}

template <typename PT, bool REAL>
expd_status launch_time(expd_plan p, TimeArgs& a, cudaStream_t s) {
    const TimeTables& t = std::is_same<PT, float>::value ? p->t32 : p->t64;
    a.gamma = t.gamma;
    a.lam = t.lam;
    a.tw = t.tw;
    a.chirp = t.chirp;
    a.bplus = t.bplus;
    a.bminus = t.bminus;
    a.L = t.L;
    a.log2L = t.log2L;
    a.bluestein = t.bluestein;
    const size_t smem = time_smem_bytes(p->Ns, t.L, t.bluestein, sizeof(typename cplx<PT>::t));
    auto kern = time_kernel<PT, REAL>;
    EXPD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const double esz = REAL ? 8.0 : 16.0;
    const double per = (a.X ? esz : 0.0) + (a.F ? esz : 0.0) + (a.NL ? (a.nl_f32 ? esz / 2 : esz) : 0.0) + esz;
    const double lg = (double)t.log2L;
    const double fl_col = (a.precond ? (t.bluestein ? 4.0 : 2.0) * 5.0 * t.L * lg + 8.0 * p->order * p->Ns : 0.0) +
                          4.0 * p->order * p->Ns;
    KProf kp(p, s, EXPD_K_TIME, per * p->Ns * (double)p->Mcol, fl_col * (double)p->Mcol);
    kern<<<p->time_grid, 32 * EXPD_TIME_COLS, smem, s>>>(a);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

template <typename T2, typename T>
void* upload(const std::vector<std::complex<double>>& v, cudaStream_t s, size_t& bytes, expd_status& st) {
    std::vector<T2> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        h[i].x = (T)v[i].real();
        h[i].y = (T)v[i].imag();
    }
    void* d = nullptr;
    cudaError_t e = cudaMalloc(&d, h.size() * sizeof(T2) + 16);
    if (e != cudaSuccess) {
        st = expd_cuda_fail(e, "cudaMalloc(time table)", __FILE__, __LINE__);
        return nullptr;
    }
    bytes += h.size() * sizeof(T2) + 16;
    e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = expd_cuda_fail(e, "cudaMemcpyAsync(time table)", __FILE__, __LINE__);
    return d;
}

template <typename T2, typename T>
expd_status build_tables(expd_plan p, TimeTables& t, cudaStream_t s) {
    const TimeTablesHost h = time_tables_host(p->Ns, p->alpha);
    t.L = h.L;
    t.log2L = h.log2L;
    t.bluestein = h.bluestein;
    expd_status st = EXPD_OK;
    t.tw = upload<T2, T>(h.tw, s, p->bytes, st);
    if (st == EXPD_OK) t.lam = upload<T2, T>(h.lam, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.chirp = upload<T2, T>(h.chirp, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.bplus = upload<T2, T>(h.bplus, s, p->bytes, st);
    if (st == EXPD_OK && t.bluestein) t.bminus = upload<T2, T>(h.bminus, s, p->bytes, st);
    if (st != EXPD_OK) return st;
    cudaError_t e = cudaMalloc(&t.gamma, h.gamma.size() * sizeof(double));
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMalloc(gamma)", __FILE__, __LINE__);
    p->bytes += h.gamma.size() * sizeof(double);
    e = cudaMemcpyAsync(t.gamma, h.gamma.data(), h.gamma.size() * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMemcpyAsync(gamma)", __FILE__, __LINE__);
    return EXPD_OK;
}

}  // namespace

expd_status time_tables_build(expd_plan p, cudaStream_t s) {
    expd_status st = build_tables<double2, double>(p, p->t64, s);
    if (st != EXPD_OK) return st;
    st = build_tables<float2, float>(p, p->t32, s);
    if (st != EXPD_OK) return st;
    int grid = 0;
    st = time_grid_for(p, &grid);
    if (st != EXPD_OK) return st;
    p->time_grid = grid;
    cudaError_t e = cudaMalloc(&p->partial, (size_t)grid * p->Ns * sizeof(double2));
    if (e != cudaSuccess) return expd_cuda_fail(e, "cudaMalloc(partial)", __FILE__, __LINE__);
    p->bytes += (size_t)grid * p->Ns * sizeof(double2);
    return EXPD_OK;
}

expd_status time_grid_for(expd_plan p, int* grid_out) {
    // a multiple of the SM count, as many CTAs as fit, never more than tiles
    const long long ntiles = (p->Mcol + EXPD_TIME_COLS - 1) / EXPD_TIME_COLS;
    int L = 1;
    while (L < p->Ns) L <<= 1;
    const int blue = (L != p->Ns);
    if (blue) {
        L = 1;
        while (L < 2 * p->Ns - 1) L <<= 1;
    }
    int per_sm = 1;
    const size_t smem = time_smem_bytes(p->Ns, L, blue, sizeof(double2));
    auto kern = p->realcol ? time_kernel<double, true> : time_kernel<double, false>;
    if (smem > 227 * 1024) return expd_fail(EXPD_ERR_UNSUPPORTED, "time window too long for shared memory");
    EXPD_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    EXPD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * EXPD_TIME_COLS, smem));
    if (per_sm < 1) per_sm = 1;
    long long grid = (long long)p->sm_count * per_sm;
    if (grid > ntiles) grid = ntiles;
    *grid_out = (int)grid;
    return EXPD_OK;
}

void time_tables_free(expd_plan p) {
    TimeTables* ts[2] = {&p->t64, &p->t32};
    for (TimeTables* t : ts) {
        cudaFree(t->gamma);
        cudaFree(t->lam);
        cudaFree(t->tw);
        cudaFree(t->chirp);
        cudaFree(t->bplus);
        cudaFree(t->bminus);
        *t = TimeTables();
    }
}

expd_status time_apply(expd_plan p, const TimeOp& op, cudaStream_t s) {
    TimeArgs a;
    a.X = op.X;
    a.F = op.F;
    a.NL = op.NL;
    a.out = op.out;
    a.nl_f32 = op.nl_f32;
    a.bdt = op.bdt;
    a.sigR = op.sigR;
    a.precond = op.precond;
    a.accum = op.accum;
    a.Mcol = p->Mcol;
    a.Ns = p->Ns;
    a.order = p->order;
    for (int j = 0; j < 7; ++j) a.a[j] = p->acoef[p->order][j];
    a.E = p->E;
    a.KX = p->KX;
    a.NX = p->NX;
    a.realcol = p->realcol;
    a.ntiles = (p->Mcol + EXPD_TIME_COLS - 1) / EXPD_TIME_COLS;
    a.partial = p->partial;
    if (op.f32) return p->realcol ? launch_time<float, true>(p, a, s) : launch_time<float, false>(p, a, s);
    return p->realcol ? launch_time<double, true>(p, a, s) : launch_time<double, false>(p, a, s);
}

expd_status time_reduce(expd_plan p, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_REDUCE, 16.0 * p->time_grid * p->Ns, 2.0 * p->time_grid * p->Ns);
    reduce_kernel<<<1, 256, 0, s>>>(p->partial, p->time_grid, p->Ns, p->redout);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}
