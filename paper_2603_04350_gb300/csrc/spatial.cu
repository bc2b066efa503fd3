// Spatial side of the hot path: the change of basis to L_h's eigenvectors and
// back (the spatial half of the preconditioner's Step (b), Eq. (3.3), which is
// diagonal in that basis), the pointwise nonlinearity and the pointwise implicit
// solve of the IF scheme (Eq. (6.1)), and the eigen-space combinations that build
// the startup ramp and the known right-hand side f_s (Eq. (4.2), Sec. 5).
//
// Periodic grids: real <-> half-spectrum FFTs.  The contiguous axis is one warp
// per row (a real row of NX samples packed as NX/2 complex values, a radix-2
// FFT in shared memory, then the even/odd split); the strided axis is one warp
// per column of a [NY x C] tile staged through shared memory so that global
// loads stay coalesced along the contiguous axis.  The nonlinear evaluation
// fuses inverse row FFT, N(u) and forward row FFT in one pass.
//
// Dirichlet grids: the orthonormal DST-I as a dense matrix product (float64).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "common.cuh"
#include "dd.cuh"
#include "plan.h"

namespace {

template <typename R>
__device__ __forceinline__ R nl_ac(R u) { return u - u * u * u; }

// ------------------------------------------------------------ row pass ----
// KIND 0: complex half-spectrum row (KX = NX/2+1) -> real row      (c2r)
// KIND 1: real row -> complex half-spectrum row                     (r2c)
// KIND 2: c2r, u -> N(u), r2c (fused nonlinear evaluation)
template <typename PT, typename TIN, typename TOUT, int KIND>
__global__ void row_kernel(const TIN* in, TOUT* out, long long rows, int NX,
                           int log2NH, const typename cplx<PT>::t* __restrict__ Wg, PT scale, int nonlin,
                           double* const* phys_slot) {
    typedef typename cplx<PT>::t PT2;
    constexpr int PAD = sizeof(PT2) >= 16;  // padded rows for 16-byte elements
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // KIND 2: where to write the physical rows (read from device memory, so a
    // captured launch serves any output buffer), or nowhere
    double* const phys = (KIND == 2 && phys_slot) ? *phys_slot : nullptr;
    const int NH = NX >> 1;
    const int KX = NH + 1;
    PT2* W = reinterpret_cast<PT2*>(smem_raw);
    // per-pass twiddle pairs of the length-NH FFTs (consecutive lanes read
    // consecutive entries), then the rows
    TwPair<PT2>* twp = reinterpret_cast<TwPair<PT2>*>(W + ((KX + 1) & ~1));
    PT2* buf = reinterpret_cast<PT2*>(twp + twp_entries(NH));
    for (int i = threadIdx.x; i < KX; i += blockDim.x) W[i] = Wg[i];
    __syncthreads();
    twp_build(twp, W, 2, NH, (int)threadIdx.x, (int)blockDim.x);
    pdl_wait();  // the rows come from the previous kernel
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, R = blockDim.x >> 5;
    PT2* s = buf + (size_t)warp * padded_len<PAD>(NH);
    for (long long row = (long long)blockIdx.x * R + warp; row < rows; row += (long long)gridDim.x * R) {
        if constexpr (KIND == 1) {
            const TIN* x = in + row * NX;
            for (int n = lane; n < NH; n += 32)
                s[padi<PAD>(bitrev(n, log2NH))] = c2((PT)x[2 * n], (PT)x[2 * n + 1]);
        } else {
            // Hermitian half spectrum -> packed even/odd spectrum Z = E + i O
            const TIN* X = in + row * KX;
            for (int k = lane; k < NH; k += 32) {
                const PT2 xk = cvt2<PT2>(X[k]);
                const PT2 xm = cconj(cvt2<PT2>(X[NH - k]));
                const PT2 e = cscale(cadd(xk, xm), (PT)0.5);
                const PT2 o = cmulc(cscale(csub(xk, xm), (PT)0.5), W[k]);
                s[padi<PAD>(bitrev(k, log2NH))] = cadd(e, cmuli(o));
            }
        }
        EXPD_SYNCWARP();
        fft_dit_tp<PT2, PAD>(s, log2NH, twp, KIND == 1 ? -1 : +1, lane, 32);  // natural order
        if constexpr (KIND == 0) {
            // z_n = x_{2n} + i x_{2n+1}
            TOUT* x = out + row * NX;
            for (int n = lane; n < NH; n += 32) {
                const PT2 z = s[padi<PAD>(n)];
                x[2 * n] = (TOUT)(z.x * scale);
                x[2 * n + 1] = (TOUT)(z.y * scale);
            }
            EXPD_SYNCWARP();
        } else {
        if constexpr (KIND == 2) {
            for (int n = lane; n < NH; n += 32) {
                PT2 z = cscale(s[padi<PAD>(n)], scale);
                if (phys) {  // the physical row before N, in float64 (phys[row][NX])
                    phys[row * NX + 2 * n] = (double)z.x;
                    phys[row * NX + 2 * n + 1] = (double)z.y;
                }
                if (nonlin == EXPD_NL_ALLEN_CAHN) z = c2(nl_ac(z.x), nl_ac(z.y));
                else z = c2((PT)0, (PT)0);
                s[padi<PAD>(n)] = z;
            }
            EXPD_SYNCWARP();
            fft_dif_tp<PT2, PAD>(s, log2NH, twp, -1, lane, 32);  // bit-reversed order
        }
        // even/odd split: X_k = E_k + W^k O_k, k = 0..NH
        TOUT* X = out + row * KX;
        for (int k = lane; k <= NH; k += 32) {
            const int k1 = (k == NH) ? 0 : k;
            const int k2 = (k == 0) ? 0 : NH - k;
            const int p1 = (KIND == 2) ? (int)bitrev(k1, log2NH) : k1;
            const int p2 = (KIND == 2) ? (int)bitrev(k2, log2NH) : k2;
            const PT2 zk = s[padi<PAD>(p1)];
            const PT2 zm = cconj(s[padi<PAD>(p2)]);
            const PT2 e = cscale(cadd(zk, zm), (PT)0.5);
            const PT2 o = cscale(cmuli(csub(zm, zk)), (PT)0.5);
            X[k] = cvt2<TOUT>(cadd(e, cmul(W[k], o)));
        }
        EXPD_SYNCWARP();
        }
    }
}

// --------------------------------------------------------- column pass ----
// In-place-capable c2c FFT along the strided axis of [nslices][NY][KX] arrays.
template <typename PT, typename TIN, typename TOUT>
__global__ void col_kernel(const TIN* __restrict__ in, TOUT* __restrict__ out, int NY, int KX, int log2NY,
                           int C, const typename cplx<PT>::t* __restrict__ Wg, int sign, PT scale) {
    typedef typename cplx<PT>::t PT2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PT2* W = reinterpret_cast<PT2*>(smem_raw);
    const int nw = NY >> 1;
    TwPair<PT2>* twp = reinterpret_cast<TwPair<PT2>*>(W + ((nw + 1) & ~1));  // per-pass twiddle pairs
    PT2* buf = reinterpret_cast<PT2*>(twp + twp_entries(NY));
    for (int i = threadIdx.x; i < nw; i += blockDim.x) W[i] = Wg[i];
    __syncthreads();
    twp_build(twp, W, 1, NY, (int)threadIdx.x, (int)blockDim.x);
    pdl_wait();
    const long long base = (long long)blockIdx.y * NY * KX;
    const int kx0 = blockIdx.x * C;
    // columns are contiguous in shared memory with a padded stride, so the
    // transposing load and store spread consecutive columns over the banks
    const int NYP = NY + 1;
    for (int idx = threadIdx.x; idx < NY * C; idx += blockDim.x) {
        const int y = idx / C, c = idx - y * C, kx = kx0 + c;
        PT2 v = c2((PT)0, (PT)0);
        if (kx < KX) v = cvt2<PT2>(in[base + (long long)y * KX + kx]);
        buf[c * NYP + bitrev(y, log2NY)] = v;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp < C && kx0 + warp < KX) fft_dit_tp(buf + warp * NYP, log2NY, twp, sign, lane, 32);
    __syncthreads();
    for (int idx = threadIdx.x; idx < NY * C; idx += blockDim.x) {
        const int y = idx / C, c = idx - y * C, kx = kx0 + c;
        if (kx < KX) out[base + (long long)y * KX + kx] = cvt2<TOUT>(cscale(buf[c * NYP + y], scale));
    }
}

// ---------------------------------------------------------- dense DST ----
// C[b] = A[b] (MxK) * B[b] (KxN), row-major, float64, 64x64 tiles.
__global__ void __launch_bounds__(256) dgemm_kernel(int M, int N, int K, const double* __restrict__ A,
                                                    long long lda, long long sA, const double* __restrict__ B,
                                                    long long ldb, long long sB, double* __restrict__ C,
                                                    long long ldc, long long sC) {
    const long long b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    __shared__ double As[16][65];
    __shared__ double Bs[16][65];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int k0 = 0; k0 < K; k0 += 16) {
        for (int i = tid; i < 64 * 16; i += 256) {
            const int r = i >> 4, kk = i & 15, gm = m0 + r, gk = k0 + kk;
            As[kk][r] = (gm < M && gk < K) ? A[(long long)gm * lda + gk] : 0.0;
        }
        for (int i = tid; i < 16 * 64; i += 256) {
            const int kk = i >> 6, cc = i & 63, gk = k0 + kk, gn = n0 + cc;
            Bs[kk][cc] = (gk < K && gn < N) ? B[(long long)gk * ldb + gn] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gm = m0 + ty * 4 + i, gn = n0 + tx * 4 + j;
            if (gm < M && gn < N) C[(long long)gm * ldc + gn] = acc[i][j];
        }
}

// ----------------------------------------------------------- pointwise ----
__global__ void newton_kernel(const double* w, double* u, long long n, double bdt,
                              int nonlin) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double wi = w[i];
        double x = wi;
        if (nonlin == EXPD_NL_ALLEN_CAHN) {
            for (int it = 0; it < 60; ++it) {
                const double g = x - bdt * (x - x * x * x) - wi;
                const double dg = 1.0 - bdt + 3.0 * bdt * x * x;
                const double dx = g / dg;
                x -= dx;
                if (fabs(dx) <= 1e-16 * fmax(1.0, fabs(x))) break;
            }
        }
        u[i] = x;
    }
}

__global__ void nl_pointwise_kernel(double* __restrict__ u, long long n, int nonlin) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = u[i];
        u[i] = (nonlin == EXPD_NL_ALLEN_CAHN) ? x - x * x * x : 0.0;
    }
}

// ---- ETD1 (first-order exponential time differencing, phi_1) ----
// N of the unknown slices moved one slice later and scaled per mode:
// NL_n <- phi_m NL_{n-1} for n = Ns-1 .. 1, NL_0 <- 0 (row 0's N(u_0) term is
// in the right-hand side).  In place: one thread per scalar element walks its
// slices downward (every old value is read before it is overwritten),
// coalesced across the elements.  T: float64, float32 or double-float storage.
template <typename T, typename P>
__global__ void etd_shift_kernel(T* __restrict__ NL, const P* __restrict__ phi, long long nelem, int eshift, int Ns) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nelem;
         e += (long long)gridDim.x * blockDim.x) {
        const P ph = phi[e >> eshift];
        for (int n = Ns - 1; n >= 1; --n) NL[(long long)n * nelem + e] = ph * NL[(long long)(n - 1) * nelem + e];
        NL[e] = T(0.0f);
    }
}

// ETD1 step in the eigenbasis: out = E_m prev + phi_m nl (float64)
__global__ void etd_step_kernel(double* __restrict__ out, const double* __restrict__ prev,
                                const double* __restrict__ nl, const double* __restrict__ E,
                                const double* __restrict__ phi, long long nelem, int eshift) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nelem;
         e += (long long)gridDim.x * blockDim.x) {
        const long long m = e >> eshift;
        out[e] = fma(E[m], prev[e], phi[m] * nl[e]);
    }
}

// out = N(u) pointwise (float64 physical values)
__global__ void nl_eval_kernel(const double* __restrict__ u, double* __restrict__ out, long long n, int nonlin) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = u[i];
        out[i] = (nonlin == EXPD_NL_ALLEN_CAHN) ? x - x * x * x : 0.0;
    }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// double -> double-float in place (same 8 bytes per value)
__global__ void f64_to_dd_kernel(double* __restrict__ a, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const dd v(a[i]);
        reinterpret_cast<dd*>(a)[i] = v;
    }
}

// float32 -> double-float (exact: lo = 0), four values per thread and step
__global__ void f32_to_dd_kernel(const float* __restrict__ in, dd* __restrict__ out, long long n) {
    pdl_wait();
    const long long n4 = n >> 2;
    const float4* in4 = reinterpret_cast<const float4*>(in);
    float4* out4 = reinterpret_cast<float4*>(out);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4; i += (long long)gridDim.x * blockDim.x) {
        const float4 v = in4[i];
        out4[2 * i] = make_float4(v.x, 0.0f, v.y, 0.0f);
        out4[2 * i + 1] = make_float4(v.z, 0.0f, v.w, 0.0f);
    }
    for (long long i = 4 * n4 + blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = dd(in[i]);
}

struct CombineArgs {
    const double* in[6];
    double coef[6];
    int q;
    const double* src;
    double g;
    double* out;
    const double* E;  // E_m (real), or (Re, Im) pairs with advection
    long long nelem;
    int eshift;
    int adv;
};

// a_j E^j z for one stored double of a complex mode z: with a complex E the
// element e (real part for even e, imaginary for odd) also needs its partner
__device__ __forceinline__ double cmul_elem(double cr, double ci, const double* z, long long e) {
    const double self = z[e], other = z[e ^ 1];
    return (e & 1) ? fma(cr, self, ci * other) : fma(cr, self, -ci * other);
}

__global__ void combine_kernel(CombineArgs a) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < a.nelem;
         e += (long long)gridDim.x * blockDim.x) {
        double acc = a.src ? a.g * a.src[e] : 0.0;
        if (!a.adv) {
            const double Em = a.E[e >> a.eshift];
            double Ej = 1.0;
            for (int j = 0; j < a.q; ++j) {
                Ej *= Em;
                acc = fma(a.coef[j] * Ej, a.in[j][e], acc);
            }
        } else {
            const long long m = e >> 1;
            const double er = a.E[2 * m], ei = a.E[2 * m + 1];
            double pr = 1.0, pi = 0.0;  // E^j
            for (int j = 0; j < a.q; ++j) {
                const double t = pr * er - pi * ei;
                pi = pr * ei + pi * er;
                pr = t;
                acc += cmul_elem(a.coef[j] * pr, a.coef[j] * pi, a.in[j], e);
            }
        }
        a.out[e] = acc;
    }
}

struct RhsArgs {
    const double* fh;  // [Nt][nelem] or null
    const double* Sh;  // [s][nelem]
    double* Fh;        // [Ns][nelem]
    float* F32;        // optional float32 copy [Ns][nelem]
    int fh_dd;         // write Fh as double-float (hi, lo) instead of float64
    int adv;           // E holds complex (Re, Im) pairs
    const double* E;
    double a[7];
    double bdt;
    long long nelem;
    int eshift, s, Ns;
    const double* nl0;  // ETD1: N(u_0) transformed ([nelem]); row 0 gains phi_m N(u_0)
    const double* phi;  // ETD1: dt phi_1(dt mu_m) per mode
};

// Initial iterate X_k[m] = E_m^(k+1) S[m], k < Ns: one thread per mode walks
// the slices (multiplying by E_m, complex with advection), coalesced across
// the modes; in float32 for the float32 iterate (a guess needs no more).
template <typename ST, bool REAL, bool ADV>
__global__ void linear_guess_kernel(const double* __restrict__ E, const double* __restrict__ S, ST* __restrict__ X,
                                    long long Mcol, int Ns) {
    typedef typename cplx<ST>::t ST2;
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < Mcol;
         m += (long long)gridDim.x * blockDim.x) {
        if constexpr (REAL) {
            ST e, x;
            if constexpr (std::is_same<ST, float>::value) {
                e = f32_rn_from_f64(E[m]);
                x = f32_rn_from_f64(S[m]);
            } else {
                e = E[m];
                x = S[m];
            }
            for (int k = 0; k < Ns; ++k) {
                x *= e;
                X[(long long)k * Mcol + m] = x;
            }
        } else {
            const ST2 x0 = cvt2<ST2>(reinterpret_cast<const double2*>(S)[m]);
            ST2 e = c2((ST)0, (ST)0), x = x0;
            if constexpr (ADV) e = cvt2<ST2>(reinterpret_cast<const double2*>(E)[m]);
            else e.x = std::is_same<ST, float>::value ? (ST)f32_rn_from_f64(E[m]) : (ST)E[m];
            ST2* X2 = reinterpret_cast<ST2*>(X);
            for (int k = 0; k < Ns; ++k) {
                x = ADV ? cmul(x, e) : cscale(x, e.x);
                X2[(long long)k * Mcol + m] = x;
            }
        }
    }
}

// grid: x over a slice's elements, y over the Ns slices; a thread takes four
// elements a grid stride apart per iteration, their source loads issued
// together (four loads in flight per thread)
__global__ void rhs_kernel(RhsArgs r) {
    const int i = blockIdx.y;
    const int n = r.s + i;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x; e0 < r.nelem; e0 += 4 * stride) {
        double fv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long e = e0 + u * stride;
            fv[u] = r.fh && e < r.nelem ? r.fh[(long long)(n - 1) * r.nelem + e] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long e = e0 + u * stride;
            if (e >= r.nelem) break;
            const long long idx = (long long)i * r.nelem + e;
            double acc = r.fh ? r.bdt * fv[u] : 0.0;
            if (i < r.s && !r.adv) {
                const double Em = r.E[e >> r.eshift];
                double Ej = 1.0;
                for (int j = 1; j <= r.s; ++j) {
                    Ej *= Em;
                    if (n - j < r.s) acc = fma(r.a[j] * Ej, r.Sh[(long long)(n - j) * r.nelem + e], acc);
                }
            } else if (i < r.s) {
                const long long m = e >> 1;
                const double er = r.E[2 * m], ei = r.E[2 * m + 1];
                double pr = 1.0, pi = 0.0;
                for (int j = 1; j <= r.s; ++j) {
                    const double t = pr * er - pi * ei;
                    pi = pr * ei + pi * er;
                    pr = t;
                    if (n - j < r.s) acc += cmul_elem(r.a[j] * pr, r.a[j] * pi, r.Sh + (long long)(n - j) * r.nelem, e);
                }
            }
            if (i == 0 && r.nl0) acc = fma(r.phi[e >> r.eshift], r.nl0[e], acc);
            if (r.F32) r.F32[idx] = f32_rn_from_f64(acc);
            if (r.fh_dd) reinterpret_cast<dd*>(r.Fh)[idx] = dd_from_f64(acc);
            else r.Fh[idx] = acc;
        }
    }
}

// Sum of squares of n doubles: fixed-order per-block partials, then one block
// sums them in order (deterministic).
__global__ void __launch_bounds__(256) sumsq_partial_kernel(const double* __restrict__ x, long long n,
                                                            double* __restrict__ partial) {
    __shared__ double red[8];
    double acc = 0.0;
    for (long long i = blockIdx.x * 256LL + threadIdx.x; i < n; i += (long long)gridDim.x * 256)
        acc = fma(x[i], x[i], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        partial[blockIdx.x] = t;
    }
}

__global__ void sumsq_final_kernel(const double* __restrict__ partial, int nb, double* __restrict__ out) {
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int b = 0; b < nb; ++b) t += partial[b];
        *out = t;
    }
}

int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152LL * 32) b = 152LL * 32;
    return (int)b;
}

// Strided-axis FFT of length N = N1 x N2 along the columns of every slice,
// four-step.  A CTA owns C columns (flattened over slices) with T = N2
// threads per column, the column index fastest across the threads so that
// every global access of a warp covers whole row segments.  Step 1: each
// thread loads its N1 elements n1 N2 + r straight from global memory, runs
// the N1-point FFT in registers and multiplies by w_N^(r k1); one
// shared-memory transpose; step 2: the thread runs P = N1 / N2 of the
// N2-point FFTs (k1 = r + p T) and stores X[k1 + N1 k2] straight to global
// memory.  One shared-memory round trip per element, conflict-free (the
// column stride is odd).  sign > 0 runs the inverse by conjugating input and
// output.
constexpr int COL4_THREADS = 256;

// columns per CTA (one per T = N2 threads) and the column stride in shared memory
constexpr int col4_columns(int N1, int N2) { return (void)N1, COL4_THREADS / N2; }
constexpr int col4_stride(int N1, int N2) { return (N1 * (N2 + 1)) | 1; }

// resident CTAs per SM the register budget is sized for: float32 data takes
// 2 registers per complex value, double-float 4
template <typename PT>
constexpr int fft4_min_blocks(int N1) {
    return sizeof(PT) == 4 ? (N1 >= 32 ? 2 : 4) : (N1 >= 32 ? 1 : 2);
}

template <typename PT, typename TIN, typename TOUT, int N1, int N2>
__global__ void __launch_bounds__(COL4_THREADS, fft4_min_blocks<PT>(N1)) col4_kernel(const TIN* __restrict__ in, TOUT* __restrict__ out,
                                                                long long ncols, int KX,
                                                                const typename cplx<PT>::t* __restrict__ Wg,
                                                                int sign, PT scale) {
    typedef typename cplx<PT>::t PT2;
    constexpr int N = N1 * N2;
    constexpr int T = N2, P = N1 / N2;
    constexpr int C = col4_columns(N1, N2);
    constexpr int CS = col4_stride(N1, N2);
    static_assert(N1 % N2 == 0, "four-step split needs N2 | N1");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PT2* TW = reinterpret_cast<PT2*>(smem_raw);  // exp(-2 pi i k/N), k < N
    PT2* tile = TW + N;
    const int tid = threadIdx.x;
    const int c = tid % C, r = tid / C;
    const long long g = (long long)blockIdx.x * C + c;
    const bool valid = g < ncols;
    const long long sl = valid ? g / KX : 0;
    const long long base = valid ? sl * (long long)N * KX + (g - sl * KX) : 0;
    const TIN* src = in + base;  // this column; element y at src[y KX] (N KX < 2^31)
    TOUT* dst = out + base;
    const bool inv = sign > 0;
    // ---- the twiddle table, then (once the previous kernel is done) the
    // step-1 loads, all in flight ----
    for (int k = tid; k < N / 2; k += COL4_THREADS) {
        const PT2 w = Wg[k];
        TW[k] = w;
        TW[k + N / 2] = c2(-w.x, -w.y);
    }
    pdl_wait();
    PT2 v[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        PT2 x = c2((PT)0, (PT)0);
        if (valid) x = cvt2<PT2>(src[((int)bitrev((unsigned)j, ilog2_ct(N1)) * N2 + r) * KX]);
        if (inv) x.y = -x.y;
        v[j] = x;
    }
    __syncthreads();
    // ---- step 1: N1-point FFT over n1 (bit-reversed slots), twiddle ----
    reg_fft_dit<N1, N2, -1>(v, TW);
#pragma unroll
    for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], TW[r * k1]);
    PT2* col = tile + c * CS;
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) col[k1 * (N2 + 1) + r] = v[k1];
    __syncthreads();
    // ---- step 2: N2-point FFTs over n2 for k1 = r + pp T, stored to global ----
#pragma unroll
    for (int pp = 0; pp < P; ++pp) {
        const int k1 = r + pp * T;
        PT2 w[N2];
#pragma unroll
        for (int j = 0; j < N2; ++j) w[j] = col[k1 * (N2 + 1) + (int)bitrev((unsigned)j, ilog2_ct(N2))];
        reg_fft_dit<N2, N1, -1>(w, TW);
        if (valid) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                PT2 y = w[k2];
                if (inv) y.y = -y.y;
                dst[(k1 + N1 * k2) * KX] = cvt2<TOUT>(cscale(y, scale));
            }
        }
    }
}

// Tile-staged variant (double-float): the CTA loads C columns into shared
// memory with coalesced row loads, runs both register FFT steps through the
// tile (N2 threads per column in step 1, N1 in step 2) and stores the tile
// with coalesced rows.  For double-float it measured faster than the direct
// variant above (38 against 44 us on 64 x 129 columns of 256).
constexpr int col4s_columns(int N1, int N2, int esz) {
    const int CS = N1 * N2 + N1 + 1, CR = COL4_THREADS / N1;
    int C = esz == 8 ? 16 : 8;
    while (C > 1 && (long long)C * CS * esz > 96 * 1024) C >>= 1;
    return C < CR ? CR : C;
}

template <typename PT, typename TIN, typename TOUT, int N1, int N2>
__global__ void __launch_bounds__(COL4_THREADS, fft4_min_blocks<PT>(N1)) col4s_kernel(const TIN* __restrict__ in, TOUT* __restrict__ out,
                                                                long long ncols, int KX,
                                                                const typename cplx<PT>::t* __restrict__ Wg,
                                                                int sign, PT scale) {
    typedef typename cplx<PT>::t PT2;
    constexpr int N = N1 * N2;
    constexpr int C = col4s_columns(N1, N2, (int)sizeof(PT2));
    constexpr int LOADS = (N * C + COL4_THREADS - 1) / COL4_THREADS;
    constexpr int CS = N + N1 + 1;  // column stride in shared memory (odd)
    constexpr int CR = COL4_THREADS / N1;  // columns per round
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PT2* TW = reinterpret_cast<PT2*>(smem_raw);  // exp(-2 pi i k/N), k < N
    long long* cbase = reinterpret_cast<long long*>(TW + N);
    PT2* tile = reinterpret_cast<PT2*>(cbase + C);
    const int tid = threadIdx.x;
    for (int k = tid; k < N / 2; k += COL4_THREADS) {
        const PT2 w = Wg[k];
        TW[k] = w;
        TW[k + N / 2] = c2(-w.x, -w.y);
    }
    const long long g0 = (long long)blockIdx.x * C;
    for (int c = tid; c < C; c += COL4_THREADS) {
        const long long g = g0 + c;
        const long long sl = g / KX;
        cbase[c] = g < ncols ? sl * (long long)N * KX + (g - sl * KX) : -1;
    }
    pdl_wait();
    __syncthreads();
    const bool inv = sign > 0;
    // ---- coalesced load: row y of C consecutive columns, all loads in flight ----
    {
        TIN ld[LOADS];
#pragma unroll
        for (int it = 0; it < LOADS; ++it) {
            const int i = tid + it * COL4_THREADS;
            const int y = i / C, c = i % C;
            const long long b = i < N * C ? cbase[c] : -1;
            if (b >= 0) ld[it] = in[b + (long long)y * KX];
            else ld[it] = TIN{};
        }
#pragma unroll
        for (int it = 0; it < LOADS; ++it) {
            const int i = tid + it * COL4_THREADS;
            if (i < N * C) {
                PT2 v = cvt2<PT2>(ld[it]);
                if (inv) v.y = -v.y;
                tile[(i % C) * CS + i / C] = v;
            }
        }
    }
    __syncthreads();
    const int q = tid / N1, r = tid - q * N1;
    for (int c0 = 0; c0 < C; c0 += CR) {
        PT2* col = tile + (c0 + q) * CS;
        const bool act = c0 + q < C;
        PT2 v[N1];
        // step 1: N1-point FFT over n1 (bit-reversed slots), twiddle
        if (act && r < N2) {
#pragma unroll
            for (int j = 0; j < N1; ++j) v[j] = col[(int)bitrev((unsigned)j, ilog2_ct(N1)) * N2 + r];
            reg_fft_dit<N1, N2, -1>(v, TW);
#pragma unroll
            for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], TW[r * k1]);
        }
        __syncthreads();
        if (act && r < N2) {
#pragma unroll
            for (int k1 = 0; k1 < N1; ++k1) col[k1 * (N2 + 1) + r] = v[k1];
        }
        __syncthreads();
        // step 2: N2-point FFT over n2 for k1 = r
        PT2 w[N2];
        if (act) {
#pragma unroll
            for (int j = 0; j < N2; ++j) w[j] = col[r * (N2 + 1) + (int)bitrev((unsigned)j, ilog2_ct(N2))];
            reg_fft_dit<N2, N1, -1>(w, TW);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) col[r + N1 * k2] = w[k2];
        }
    }
    __syncthreads();
    // ---- coalesced store ----
#pragma unroll 4
    for (int it = 0; it < LOADS; ++it) {
        const int i = tid + it * COL4_THREADS;
        const int y = i / C, c = i % C;
        const long long b = i < N * C ? cbase[c] : -1;
        if (b < 0) continue;
        PT2 v = tile[c * CS + y];
        if (inv) v.y = -v.y;
        out[b + (long long)y * KX] = cvt2<TOUT>(cscale(v, scale));
    }
}

template <typename PT>
const typename cplx<PT>::t* Wx(expd_plan p);
template <>
const double2* Wx<double>(expd_plan p) { return p->Wx64; }
template <>
const float2* Wx<float>(expd_plan p) { return p->Wx32; }
template <>
const dd2* Wx<dd>(expd_plan p) { return static_cast<const dd2*>(p->Wxdd); }
template <typename PT>
const typename cplx<PT>::t* Wy(expd_plan p);
template <>
const double2* Wy<double>(expd_plan p) { return p->Wy64; }
template <>
const float2* Wy<float>(expd_plan p) { return p->Wy32; }
template <>
const dd2* Wy<dd>(expd_plan p) { return static_cast<const dd2*>(p->Wydd); }

// Contiguous-axis real FFTs of length NX = 2 NH on C rows per CTA, with the
// length-NH complex FFT done four-step (NH = N1 x N2: register FFTs of N1 and
// N2 points around one shared-memory transpose, as in col4_kernel).  Rows are
// staged in shared memory with one contiguous coalesced load (in place is
// allowed: a CTA reads all its rows before writing any).
//   KIND 1: real row -> half spectrum X_k, k = 0..NH (forward)
//   KIND 0: half spectrum -> real row (inverse, times scale)
//   KIND 2: half spectrum -> real row -> N(u) pointwise -> half spectrum
//   KIND 3: as KIND 0, added to the output row (out += result)
// Real data of length 2 NH is packed as z_n = x_{2n} + i x_{2n+1}; the
// half spectrum and Z = FFT_NH(z) are related by the even/odd split with
// w^k = exp(-2 pi i k / NX).
constexpr int row4_stride(int N1, int N2) {
    const int need = (N1 * N2 + 1) > N1 * (N2 + 1) ? N1 * N2 + 1 : N1 * (N2 + 1);
    return need | 1;
}
// T = N2 threads per row (each runs one N1-point FFT in step 1 and N1 / N2 of
// the N2-point FFTs in step 2, so no thread idles), 16 rows per CTA (8 for
// N2 = 32), one round
constexpr int row4_rows(int N1, int N2, int esz) { return (void)N1, (void)esz, N2 >= 32 ? 8 : 16; }
constexpr int row4_threads(int N1, int N2) { return row4_rows(N1, N2, 0) * N2; }
// resident CTAs the register budget is sized for (64 registers per thread for
// the float32 shapes up to N1 = 16, 128 beyond)
constexpr int row4_min_blocks(int N1, int N2) { return (N1 >= 32 ? 2 : 4) * 256 / row4_threads(N1, N2); }

template <typename PT, typename TIN, typename TOUT, int KIND, int N1, int N2>
__global__ void __launch_bounds__(row4_threads(N1, N2), row4_min_blocks(N1, N2))
    row4_kernel(const TIN* in, TOUT* out, long long rows, const typename cplx<PT>::t* __restrict__ Wg, PT scale,
                int nonlin) {
    typedef typename cplx<PT>::t PT2;
    constexpr int NH = N1 * N2, NX = 2 * NH, KXc = NH + 1;
    constexpr int CS = row4_stride(N1, N2);
    constexpr int C = row4_rows(N1, N2, (int)sizeof(PT2));
    constexpr int ROW4_THREADS = row4_threads(N1, N2);
    constexpr int T = N2, P = N1 / N2;
    constexpr int RR = ROW4_THREADS / T;
    static_assert(N1 % N2 == 0, "four-step split needs N2 | N1");
    constexpr bool C2R = KIND == 0 || KIND == 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PT2* Wn = reinterpret_cast<PT2*>(smem_raw);  // exp(-2 pi i k / NX), k <= NH
    PT2* TW = Wn + ((KXc + 1) & ~1);             // exp(-2 pi i k / NH), k < NH
    PT2* tile = TW + NH;
    const int tid = threadIdx.x;
    for (int k = tid; k < KXc; k += ROW4_THREADS) Wn[k] = Wg[k];
    for (int k = tid; k < NH / 2; k += ROW4_THREADS) {
        const PT2 w = Wg[2 * k];
        TW[k] = w;
        TW[k + NH / 2] = c2(-w.x, -w.y);
    }
    pdl_wait();
    const long long r0 = (long long)blockIdx.x * C;
    const int nr = (int)(rows - r0 < C ? rows - r0 : C);
    // ---- load the CTA's rows: one contiguous block ----
    if constexpr (KIND == 1) {
        const TIN* src = in + r0 * NX;
        for (int e = tid; e < nr * NX; e += ROW4_THREADS) {
            const int c = e / NX, x = e - c * NX;
            reinterpret_cast<PT*>(tile + c * CS)[x] = (PT)src[e];
        }
    } else {
        const TIN* src = in + r0 * KXc;
        for (int e = tid; e < nr * KXc; e += ROW4_THREADS) {
            const int c = e / KXc, k = e - c * KXc;
            tile[c * CS + k] = cvt2<PT2>(src[e]);
        }
    }
    __syncthreads();
    const int q = tid / T, r = tid - q * T;
    for (int c0 = 0; c0 < C; c0 += RR) {
        PT2* row = tile + (c0 + q) * CS;
        const bool act = c0 + q < nr;
        // ---- first transform ----
        {
            constexpr int SG1 = KIND == 1 ? -1 : +1;
            PT2 v[N1];
            if (act) {
#pragma unroll
                for (int j = 0; j < N1; ++j) {
                    const int n = (int)bitrev((unsigned)j, ilog2_ct(N1)) * N2 + r;
                    if constexpr (KIND == 1) {
                        v[j] = row[n];
                    } else {
                        const PT2 xk = row[n];
                        const PT2 xm = cconj(row[NH - n]);
                        const PT2 ev = cscale(cadd(xk, xm), (PT)0.5);
                        const PT2 od = cmulc(cscale(csub(xk, xm), (PT)0.5), Wn[n]);
                        v[j] = cadd(ev, cmuli(od));
                    }
                }
                reg_fft_dit<N1, N2, SG1>(v, TW);
#pragma unroll
                for (int k1 = 1; k1 < N1; ++k1) {
                    PT2 w = TW[r * k1];
                    if (SG1 > 0) w.y = -w.y;
                    v[k1] = cmul(v[k1], w);
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) row[k1 * (N2 + 1) + r] = v[k1];
            }
            __syncthreads();
            PT2 w2[P][N2];
            if (act) {
#pragma unroll
                for (int pp = 0; pp < P; ++pp) {
                    const int k1 = r + pp * T;
#pragma unroll
                    for (int j = 0; j < N2; ++j) w2[pp][j] = row[k1 * (N2 + 1) + (int)bitrev((unsigned)j, ilog2_ct(N2))];
                    reg_fft_dit<N2, N1, SG1>(w2[pp], TW);
                    if constexpr (KIND != 1) {
#pragma unroll
                        for (int k2 = 0; k2 < N2; ++k2) {
                            PT2 z = cscale(w2[pp][k2], scale);
                            if constexpr (KIND == 2) {
                                if (nonlin == EXPD_NL_ALLEN_CAHN) z = c2(nl_ac(z.x), nl_ac(z.y));
                                else z = c2((PT)0, (PT)0);
                            }
                            w2[pp][k2] = z;
                        }
                    }
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int pp = 0; pp < P; ++pp)
#pragma unroll
                    for (int k2 = 0; k2 < N2; ++k2) row[r + pp * T + N1 * k2] = w2[pp][k2];
            }
            __syncthreads();
        }
        // ---- second transform (KIND 2: forward FFT of N(u)) ----
        if constexpr (KIND == 2) {
            PT2 v[N1];
            if (act) {
#pragma unroll
                for (int j = 0; j < N1; ++j) v[j] = row[(int)bitrev((unsigned)j, ilog2_ct(N1)) * N2 + r];
                reg_fft_dit<N1, N2, -1>(v, TW);
#pragma unroll
                for (int k1 = 1; k1 < N1; ++k1) v[k1] = cmul(v[k1], TW[r * k1]);
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int k1 = 0; k1 < N1; ++k1) row[k1 * (N2 + 1) + r] = v[k1];
            }
            __syncthreads();
            PT2 w2[P][N2];
            if (act) {
#pragma unroll
                for (int pp = 0; pp < P; ++pp) {
                    const int k1 = r + pp * T;
#pragma unroll
                    for (int j = 0; j < N2; ++j) w2[pp][j] = row[k1 * (N2 + 1) + (int)bitrev((unsigned)j, ilog2_ct(N2))];
                    reg_fft_dit<N2, N1, -1>(w2[pp], TW);
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int pp = 0; pp < P; ++pp)
#pragma unroll
                    for (int k2 = 0; k2 < N2; ++k2) row[r + pp * T + N1 * k2] = w2[pp][k2];
            }
            __syncthreads();
        }
    }
    // ---- store: one contiguous block ----
    if constexpr (C2R) {
        TOUT* dst = out + r0 * NX;
        for (int e = tid; e < nr * NX; e += ROW4_THREADS) {
            const int c = e / NX, x = e - c * NX;
            const TOUT v = (TOUT)reinterpret_cast<const PT*>(tile + c * CS)[x];
            if constexpr (KIND == 3) dst[e] += v;
            else dst[e] = v;
        }
    } else {
        // even/odd split: X_k = E_k + w^k O_k from Z_k and conj(Z_{NH-k})
        TOUT* dst = out + r0 * KXc;
        for (int e = tid; e < nr * KXc; e += ROW4_THREADS) {
            const int c = e / KXc, k = e - c * KXc;
            const PT2* z = tile + c * CS;
            const PT2 zk = z[k == NH ? 0 : k];
            const PT2 zm = cconj(z[k == 0 ? 0 : NH - k]);
            const PT2 ev = cscale(cadd(zk, zm), (PT)0.5);
            const PT2 od = cscale(cmuli(csub(zm, zk)), (PT)0.5);
            dst[e] = cvt2<TOUT>(cadd(ev, cmul(Wn[k], od)));
        }
    }
}

template <typename PT, typename TIN, typename TOUT, int KIND, int N1, int N2>
expd_status launch_row4(expd_plan p, const TIN* in, TOUT* out, long long rows, PT scale, cudaStream_t s) {
    typedef typename cplx<PT>::t PT2;
    constexpr int NH = N1 * N2, KXc = NH + 1;
    constexpr int CS = row4_stride(N1, N2), C = row4_rows(N1, N2, (int)sizeof(PT2));
    const size_t smem = ((size_t)((KXc + 1) & ~1) + NH + (size_t)C * CS) * sizeof(PT2);
    auto kern = row4_kernel<PT, TIN, TOUT, KIND, N1, N2>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    const long long grid = (rows + C - 1) / C;
    const double in_row = (KIND == 1 ? 2 * NH : KXc) * (double)sizeof(TIN);
    const double out_row = (KIND == 0 ? 2 * NH : KIND == 3 ? 4 * NH : KXc) * (double)sizeof(TOUT);
    const double fl = (KIND == 2 ? 2.0 : 1.0) * 2.5 * (2 * NH) * ilog2(2 * NH) * (double)rows;
    KProf kp(p, s, sizeof(PT) == 4 ? EXPD_K_FFT_ROW32 : sizeof(PT) == 8 && !std::is_same<PT, double>::value ? EXPD_K_FFT_ROWDD : EXPD_K_FFT_ROW,
             (double)rows * (in_row + out_row), fl);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(row4_threads(N1, N2)), smem, s, in, out, rows, Wx<PT>(p),
                             scale, p->nonlin));
    return EXPD_OK;
}

template <typename PT, typename TIN, typename TOUT, int KIND>
expd_status launch_row_r4(expd_plan p, const TIN* in, TOUT* out, long long rows, PT scale, cudaStream_t s,
                          double* const* phys_slot);

template <typename PT, typename TIN, typename TOUT, int KIND>
expd_status launch_row(expd_plan p, const TIN* in, TOUT* out, long long rows, PT scale, cudaStream_t s,
                       double* const* phys_slot = nullptr) {
    typedef typename cplx<PT>::t PT2;
    const int NH = p->NX / 2;
    if constexpr (std::is_same<PT, float>::value) {
        // four-step kernel (float32): rows of 32 to 2048 points
        if (!p->no_fft4) switch (NH) {
            case 16: return launch_row4<PT, TIN, TOUT, KIND, 4, 4>(p, in, out, rows, scale, s);
            case 32: return launch_row4<PT, TIN, TOUT, KIND, 8, 4>(p, in, out, rows, scale, s);
            case 64: return launch_row4<PT, TIN, TOUT, KIND, 8, 8>(p, in, out, rows, scale, s);
            case 128: return launch_row4<PT, TIN, TOUT, KIND, 16, 8>(p, in, out, rows, scale, s);
            case 256: return launch_row4<PT, TIN, TOUT, KIND, 16, 16>(p, in, out, rows, scale, s);
            case 512: return launch_row4<PT, TIN, TOUT, KIND, 32, 16>(p, in, out, rows, scale, s);
            case 1024: return launch_row4<PT, TIN, TOUT, KIND, 32, 32>(p, in, out, rows, scale, s);
            default:
                break;
        }
    }
    if constexpr (KIND == 3) {
        return expd_fail(EXPD_ERR_UNSUPPORTED, "accumulating c2r needs a float32 row of 32..2048 points");
    } else {
        return launch_row_r4<PT, TIN, TOUT, KIND>(p, in, out, rows, scale, s, phys_slot);
    }
}

// the radix-4 shared-memory row kernel (every size and precision)
template <typename PT, typename TIN, typename TOUT, int KIND>
expd_status launch_row_r4(expd_plan p, const TIN* in, TOUT* out, long long rows, PT scale, cudaStream_t s,
                          double* const* phys_slot) {
    typedef typename cplx<PT>::t PT2;
    const int NH = p->NX / 2;
    const size_t per_row = (size_t)padded_len<(sizeof(PT2) >= 16)>(NH) * sizeof(PT2);
    int R = (int)std::max<size_t>(1, std::min<size_t>(8, (48 * 1024) / per_row));
    while (R > 1 && (rows + R - 1) / R < 2LL * p->sm_count) R >>= 1;  // small launches: more CTAs
    const size_t smem = (size_t)((NH + 2) & ~1) * sizeof(PT2) + (size_t)twp_entries(NH) * 2 * sizeof(PT2) +
                        (size_t)R * per_row;
    auto kern = row_kernel<PT, TIN, TOUT, KIND>;
    if (smem > 48 * 1024)
        EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    long long blocks = (rows + R - 1) / R;
    if (blocks > (long long)p->sm_count * 16) blocks = (long long)p->sm_count * 16;
    const double in_row = (KIND == 1 ? p->NX : NH + 1) * (double)sizeof(TIN);
    const double out_row = (KIND == 0 ? p->NX : NH + 1) * (double)sizeof(TOUT);
    const double fl = (KIND == 2 ? 2.0 : 1.0) * 2.5 * p->NX * ilog2(p->NX) * (double)rows;
    KProf kp(p, s, sizeof(PT) == 4 ? EXPD_K_FFT_ROW32 : sizeof(PT) == 8 && !std::is_same<PT, double>::value ? EXPD_K_FFT_ROWDD : EXPD_K_FFT_ROW,
             (double)rows * (in_row + out_row), fl);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)blocks), dim3(32 * R), smem, s, in, out, rows, p->NX, ilog2(NH),
                             Wx<PT>(p), scale, p->nonlin, phys_slot));
    return EXPD_OK;
}

template <typename PT, typename TIN, typename TOUT, int N1, int N2>
expd_status launch_col4(expd_plan p, const TIN* in, TOUT* out, int nslices, int sign, PT scale, cudaStream_t s) {
    typedef typename cplx<PT>::t PT2;
    constexpr int N = N1 * N2;
    constexpr int C = col4_columns(N1, N2), CS = col4_stride(N1, N2);
    const int KX = p->KX;
    const size_t smem = (size_t)N * sizeof(PT2) + (size_t)C * CS * sizeof(PT2);
    auto kern = col4_kernel<PT, TIN, TOUT, N1, N2>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    const long long ncols = (long long)nslices * KX;
    const long long grid = (ncols + C - 1) / C;
    KProf kp(p, s, sizeof(PT) == 4 ? EXPD_K_FFT_COL32 : sizeof(PT) == 8 && !std::is_same<PT, double>::value ? EXPD_K_FFT_COLDD : EXPD_K_FFT_COL,
             (double)nslices * N * KX * (sizeof(TIN) + sizeof(TOUT)), 5.0 * N * ilog2(N) * (double)KX * nslices);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(COL4_THREADS), smem, s, in, out, ncols, KX, Wy<PT>(p), sign,
                             scale));
    return EXPD_OK;
}

template <typename PT, typename TIN, typename TOUT, int N1, int N2>
expd_status launch_col4s(expd_plan p, const TIN* in, TOUT* out, int nslices, int sign, PT scale, cudaStream_t s) {
    typedef typename cplx<PT>::t PT2;
    constexpr int N = N1 * N2, CS = N + N1 + 1;
    constexpr int C = col4s_columns(N1, N2, (int)sizeof(PT2));
    const int KX = p->KX;
    const size_t smem = (size_t)N * sizeof(PT2) + (size_t)C * sizeof(long long) + (size_t)C * CS * sizeof(PT2);
    auto kern = col4s_kernel<PT, TIN, TOUT, N1, N2>;
    EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    const long long ncols = (long long)nslices * KX;
    const long long grid = (ncols + C - 1) / C;
    KProf kp(p, s, sizeof(PT) == 4 ? EXPD_K_FFT_COL32 : sizeof(PT) == 8 && !std::is_same<PT, double>::value ? EXPD_K_FFT_COLDD : EXPD_K_FFT_COL,
             (double)nslices * N * KX * (sizeof(TIN) + sizeof(TOUT)), 5.0 * N * ilog2(N) * (double)KX * nslices);
    EXPD_CUDA_TRY(launch_pdl(kern, dim3((unsigned)grid), dim3(COL4_THREADS), smem, s, in, out, ncols, KX, Wy<PT>(p), sign,
                             scale));
    return EXPD_OK;
}

template <typename PT, typename TIN, typename TOUT>
expd_status launch_col(expd_plan p, const TIN* in, TOUT* out, int nslices, int sign, PT scale, cudaStream_t s) {
    typedef typename cplx<PT>::t PT2;
    const int NY = p->NY, KX = p->KX;
    if constexpr (std::is_same<PT, dd>::value) {
        // four-step kernel (double-float, tile-staged): 16 to 256 rows (the row
        // pass stays on the radix-4 kernel: its double-float four-step variant
        // measured slower).  Launches too small to give every SM a CTA of 16
        // columns (a start-up slice) take the radix-4 kernel with one column
        // per warp instead.
        const long long ctas4 = ((long long)nslices * KX + 15) / 16;
        if (!p->no_fft4 && ctas4 >= p->sm_count) switch (NY) {
            case 16: return launch_col4s<PT, TIN, TOUT, 4, 4>(p, in, out, nslices, sign, scale, s);
            case 32: return launch_col4s<PT, TIN, TOUT, 8, 4>(p, in, out, nslices, sign, scale, s);
            case 64: return launch_col4s<PT, TIN, TOUT, 8, 8>(p, in, out, nslices, sign, scale, s);
            case 128: return launch_col4s<PT, TIN, TOUT, 16, 8>(p, in, out, nslices, sign, scale, s);
            case 256: return launch_col4s<PT, TIN, TOUT, 16, 16>(p, in, out, nslices, sign, scale, s);
            default:
                break;
        }
    }
    if constexpr (std::is_same<PT, float>::value) {
        // four-step kernel (float32): 16 to 1024 rows
        if (!p->no_fft4) switch (NY) {
            case 16: return launch_col4<PT, TIN, TOUT, 4, 4>(p, in, out, nslices, sign, scale, s);
            case 32: return launch_col4<PT, TIN, TOUT, 8, 4>(p, in, out, nslices, sign, scale, s);
            case 64: return launch_col4<PT, TIN, TOUT, 8, 8>(p, in, out, nslices, sign, scale, s);
            case 128: return launch_col4<PT, TIN, TOUT, 16, 8>(p, in, out, nslices, sign, scale, s);
            case 256: return launch_col4<PT, TIN, TOUT, 16, 16>(p, in, out, nslices, sign, scale, s);
            case 512: return launch_col4<PT, TIN, TOUT, 32, 16>(p, in, out, nslices, sign, scale, s);
            case 1024: return launch_col4<PT, TIN, TOUT, 32, 32>(p, in, out, nslices, sign, scale, s);
            default:
                break;
        }
    }
    const size_t per_col = (size_t)(NY + 1) * sizeof(PT2);
    // 128-byte row segments: 16 float2 or 8 double2 columns per CTA
    const int cmax = sizeof(TIN) == 8 ? 16 : 8;
    int C = (int)std::max<size_t>(1, std::min<size_t>(cmax, (64 * 1024) / per_col));
    // small launches (a slice or two): fewer columns per CTA, more CTAs
    while (C > 1 && (long long)((KX + C - 1) / C) * nslices < 2LL * p->sm_count) C >>= 1;
    const size_t smem = (size_t)(((NY >> 1) + 1) & ~1) * sizeof(PT2) + (size_t)twp_entries(NY) * 2 * sizeof(PT2) +
                        (size_t)C * per_col;
    auto kern = col_kernel<PT, TIN, TOUT>;
    if (smem > 48 * 1024)
        EXPD_CUDA_TRY(smem_allow((const void*)kern, smem));
    dim3 grid((KX + C - 1) / C, nslices);
    KProf kp(p, s, sizeof(PT) == 4 ? EXPD_K_FFT_COL32 : sizeof(PT) == 8 && !std::is_same<PT, double>::value ? EXPD_K_FFT_COLDD : EXPD_K_FFT_COL,
             (double)nslices * NY * KX * (sizeof(TIN) + sizeof(TOUT)),
             5.0 * NY * ilog2(NY) * (double)KX * nslices);
    EXPD_CUDA_TRY(launch_pdl(kern, grid, dim3(32 * C), smem, s, in, out, NY, KX, ilog2(NY), C, Wy<PT>(p), sign, scale));
    return EXPD_OK;
}

expd_status dgemm(expd_plan p, const double* A, long long lda, long long sA, const double* B, long long ldb,
                  long long sB, double* C, long long ldc, long long sC, int M, int N, int K, int batch,
                  cudaStream_t s) {
    dim3 grid((N + 63) / 64, (M + 63) / 64, batch);
    const double abytes = (sA ? (double)M * K : 0.0) + (sB ? (double)K * N : 0.0);
    KProf kp(p, s, EXPD_K_DST, 8.0 * batch * (abytes + (double)M * N), 2.0 * M * N * (double)K * batch);
    dgemm_kernel<<<grid, 256, 0, s>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// Fast orthonormal DST-I along contiguous rows of length n, where N = 2(n + 1)
// is a power of two.  Two rows share one complex FFT of length N: row a's odd
// extension [0, x_1..x_n, 0, -x_n..-x_1] in the real part, row b's in the
// imaginary part.  For an odd real sequence FFT(z)_k = -2i sum_j x_j
// sin(pi jk/(n+1)), so the sine sums are -Im Z_k / 2 (row a) and Re Z_k / 2
// (row b).  One warp per row pair, its length-N buffer in shared memory.
__global__ void __launch_bounds__(128) dst_rows_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                       long long nrows, int n, int log2N,
                                                       const double2* __restrict__ tw, double scale) {
    extern __shared__ double2 dbuf[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int N = 1 << log2N;
    double2* z = dbuf + (size_t)warp * N;
    const long long npairs = (nrows + 1) / 2;
    for (long long pr = (long long)blockIdx.x * nw + warp; pr < npairs; pr += (long long)gridDim.x * nw) {
        const long long ra = 2 * pr, rb = ra + 1;
        const bool hasb = rb < nrows;
        const double* xa = in + ra * n;
        const double* xb = in + rb * n;
        for (int j = lane; j < N; j += 32) {
            double2 v = make_double2(0.0, 0.0);
            if (j >= 1 && j <= n) {
                v = make_double2(xa[j - 1], hasb ? xb[j - 1] : 0.0);
            } else if (j > n + 1) {
                const int i = N - j - 1;
                v = make_double2(-xa[i], hasb ? -xb[i] : 0.0);
            }
            z[bitrev((unsigned)j, log2N)] = v;
        }
        __syncwarp();
        fft_dit(z, log2N, tw, 1, -1, lane, 32);
        double* ya = out + ra * n;
        double* yb = out + rb * n;
        for (int k = lane + 1; k <= n; k += 32) {
            const double2 Z = z[k];
            ya[k - 1] = -0.5 * scale * Z.y;
            if (hasb) yb[k - 1] = 0.5 * scale * Z.x;
        }
        __syncwarp();
    }
}

// out[s][c][r] = in[s][r][c] for R x C slices
__global__ void __launch_bounds__(256) transpose_kernel(const double* __restrict__ in, double* __restrict__ out,
                                                        int R, int C) {
    __shared__ double t[32][33];
    const long long off = (long long)blockIdx.z * R * C;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) t[i][threadIdx.x] = in[off + (long long)r * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[off + (long long)c * R + r] = t[threadIdx.x][i];
    }
}

expd_status dst_rows(expd_plan p, const double* in, double* out, long long nrows, int n, const double2* tw,
                     cudaStream_t s) {
    const int log2N = ilog2(2 * (n + 1));
    const int N = 1 << log2N;
    const int warps = std::max(1, std::min(4, 131072 / (N * 16)));
    const size_t smem = (size_t)warps * N * sizeof(double2);
    const long long npairs = (nrows + 1) / 2;
    const long long grid = std::min<long long>((npairs + warps - 1) / warps, (long long)p->sm_count * 32);
    EXPD_CUDA_TRY(smem_allow((const void*)dst_rows_kernel, smem));
    KProf kp(p, s, EXPD_K_DST, 16.0 * nrows * n, 5.0 * N * log2N * (double)npairs);
    dst_rows_kernel<<<(int)grid, 32 * warps, smem, s>>>(in, out, nrows, n, log2N, tw, sqrt(2.0 / (n + 1)));
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status transpose(expd_plan p, const double* in, double* out, int R, int C, int ns, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 16.0 * R * C * ns, 0.0);
    transpose_kernel<<<dim3((C + 31) / 32, (R + 31) / 32, ns), dim3(32, 8), 0, s>>>(in, out, R, C);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// The real eigenbasis transforms of Dirichlet and Neumann grids.
// Orthonormal 2D DST-I: Y = Sy X Sx (S symmetric and its own inverse).  With
// n + 1 a power of two in every direction: fast sine transforms along x, a
// transpose, along y, and back; otherwise the dense products (on the tensor
// cores when the plan allows, dst_tc.cu).  Neumann grids: the orthonormal
// DCT-II by the dense products, forward (dir < 0) Y = C_y X C_x^T with the
// operands Sx = C_x^T and Sy = C_y, inverse X = C_y^T Y C_x with SxT = C_x
// and SyT = C_y^T.
expd_status dst2(expd_plan p, const double* X, double* Y, int ns, double* tmp, cudaStream_t s, int dir = -1) {
    const int NX = p->NX, NY = p->NY;
    if (p->bc == EXPD_BC_NEUMANN) {
        const double* Bx = dir < 0 ? p->Sx : p->SxT;
        const double* Ay = dir < 0 ? p->Sy : p->SyT;
        if (p->ndim == 1) return dgemm(p, X, NX, (long long)NX, Bx, NX, 0, Y, NX, 0, ns, NX, NX, 1, s);
        expd_status st = dgemm(p, X, NX, (long long)NX, Bx, NX, 0, tmp, NX, 0, ns * NY, NX, NX, 1, s);
        if (st != EXPD_OK) return st;
        return dgemm(p, Ay, NY, 0, tmp, NX, (long long)NY * NX, Y, NX, (long long)NY * NX, NY, NX, NY, ns, s);
    }
    if (p->fast_dst) {
        if (p->ndim == 1) return dst_rows(p, X, Y, ns, NX, p->Dtx, s);
        double* w1 = tmp;
        double* w2 = tmp + (size_t)ns * p->M;
        expd_status st = dst_rows(p, X, w1, (long long)ns * NY, NX, p->Dtx, s);
        if (st == EXPD_OK) st = transpose(p, w1, w2, NY, NX, ns, s);
        if (st == EXPD_OK) st = dst_rows(p, w2, w1, (long long)ns * NX, NY, p->Dty, s);
        if (st == EXPD_OK) st = transpose(p, w1, Y, NX, NY, ns, s);
        return st;
    }
    if (p->tc_dst) return dst2_tc(p, X, Y, ns, tmp, s);
    if (p->ndim == 1) return dgemm(p, X, NX, (long long)NX, p->Sx, NX, 0, Y, NX, 0, ns, NX, NX, 1, s);
    expd_status st = dgemm(p, X, NX, (long long)NX, p->Sx, NX, 0, tmp, NX, 0, ns * NY, NX, NX, 1, s);
    if (st != EXPD_OK) return st;
    return dgemm(p, p->Sy, NY, 0, tmp, NX, (long long)NY * NX, Y, NX, (long long)NY * NX, NY, NX, NY, ns, s);
}

// Complex-to-complex FFT along contiguous rows of length n (a power of two),
// for complex states on periodic grids: one warp per row, its length-n buffer
// in shared memory (loaded in bit-reversed order), sign -1 forward and +1
// inverse, the output scaled by `scale`.  A warp reads its whole row before
// writing it, so in == out is allowed.
__global__ void __launch_bounds__(128) crow_kernel(const double2* __restrict__ in, double2* __restrict__ out,
                                                   long long rows, int n, int log2n,
                                                   const double2* __restrict__ tw, int sign, double scale) {
    extern __shared__ double2 cbuf[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double2* z = cbuf + (size_t)warp * n;
    for (long long r = (long long)blockIdx.x * nw + warp; r < rows; r += (long long)gridDim.x * nw) {
        const double2* x = in + r * n;
        for (int j = lane; j < n; j += 32) z[bitrev((unsigned)j, log2n)] = x[j];
        __syncwarp();
        fft_dit(z, log2n, tw, 1, sign, lane, 32);
        double2* y = out + r * n;
        for (int k = lane; k < n; k += 32) y[k] = cscale(z[k], scale);
        __syncwarp();
    }
}

expd_status crow(expd_plan p, const double2* in, double2* out, long long rows, int sign, double scale,
                 cudaStream_t s) {
    const int n = p->NX, log2n = ilog2(n);
    const int warps = std::max(1, std::min(4, 65536 / (n * 16)));
    const size_t smem = (size_t)warps * n * sizeof(double2);
    const long long grid = std::max(1LL, std::min<long long>((rows + warps - 1) / warps, (long long)p->sm_count * 32));
    EXPD_CUDA_TRY(smem_allow((const void*)crow_kernel, smem));
    KProf kp(p, s, EXPD_K_FFT_ROW, 32.0 * rows * n, 5.0 * n * log2n * (double)rows);
    crow_kernel<<<(int)grid, 32 * warps, smem, s>>>(in, out, rows, n, log2n, p->Wx64, sign, scale);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// A complex slice of M values as two real slices (real part, then imaginary
// part), and back: the real sine transform then acts on both parts alike.
__global__ void split_complex_kernel(const double2* __restrict__ in, double* __restrict__ out, long long M,
                                     long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long sl = i / M, e = i - sl * M;
        const double2 v = in[i];
        out[2 * sl * M + e] = v.x;
        out[(2 * sl + 1) * M + e] = v.y;
    }
}

__global__ void join_complex_kernel(const double* __restrict__ in, double2* __restrict__ out, long long M,
                                    long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long sl = i / M, e = i - sl * M;
        out[i] = make_double2(in[2 * sl * M + e], in[(2 * sl + 1) * M + e]);
    }
}

// Complex states (float64): forward (dir = -1) or inverse (dir = +1) spatial
// transform of nslices complex slices.  Periodic grids: complex FFTs along
// rows and columns, the full spectrum.  Dirichlet grids: split, the real
// orthonormal sine transform of the 2 ns real slices (its own inverse), join.
expd_status spatial_complex64(expd_plan p, const double* in, double* out, int nslices, int dir, cudaStream_t s) {
    const long long M = p->M;
    if (p->bc == EXPD_BC_PERIODIC) {
        const int chunk = p->Ns;
        for (int b0 = 0; b0 < nslices; b0 += chunk) {
            const int ns = std::min(chunk, nslices - b0);
            const double2* x = reinterpret_cast<const double2*>(in) + (long long)b0 * M;
            double2* y = reinterpret_cast<double2*>(out) + (long long)b0 * M;
            double2* w = static_cast<double2*>(p->work64);
            expd_status st;
            if (dir < 0) {
                if (p->ndim == 1) {
                    st = crow(p, x, y, ns, -1, 1.0, s);
                } else {
                    st = crow(p, x, w, (long long)ns * p->NY, -1, 1.0, s);
                    if (st == EXPD_OK) st = launch_col<double, double2, double2>(p, w, y, ns, -1, 1.0, s);
                }
            } else {
                const double sx = 1.0 / p->NX;
                if (p->ndim == 1) {
                    st = crow(p, x, y, ns, +1, sx, s);
                } else {
                    st = launch_col<double, double2, double2>(p, x, w, ns, +1, 1.0 / p->NY, s);
                    if (st == EXPD_OK) st = crow(p, w, y, (long long)ns * p->NY, +1, sx, s);
                }
            }
            if (st != EXPD_OK) return st;
        }
        return EXPD_OK;
    }
    // work64 holds 2 max(Ns, 4) M doubles: the split slices, the transformed
    // ones and the sine transform's scratch, 8 M doubles per complex slice
    const int chunk = std::max(1, p->Ns / 4);
    double* P = static_cast<double*>(p->work64);
    double* Q = P + 2LL * chunk * M;
    double* tmp = Q + 2LL * chunk * M;
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        const long long total = (long long)ns * M;
        const int blocks = grid_for(total, 256);
        {
            KProf kp(p, s, EXPD_K_POINTWISE, 32.0 * total, 0.0);
            split_complex_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2*>(in) + (long long)b0 * M, P,
                                                        M, total);
            EXPD_CUDA_TRY(cudaGetLastError());
        }
        expd_status st = dst2(p, P, Q, 2 * ns, tmp, s, dir);
        if (st != EXPD_OK) return st;
        {
            KProf kp(p, s, EXPD_K_POINTWISE, 32.0 * total, 0.0);
            join_complex_kernel<<<blocks, 256, 0, s>>>(Q, reinterpret_cast<double2*>(out) + (long long)b0 * M, M,
                                                       total);
            EXPD_CUDA_TRY(cudaGetLastError());
        }
    }
    return EXPD_OK;
}

}  // namespace

// ------------------------------------------------------------ launchers ----
expd_status spatial_forward64(expd_plan p, const double* phys, void* eig, int nslices, cudaStream_t s) {
    if (p->cplx) return spatial_complex64(p, phys, static_cast<double*>(eig), nslices, -1, s);
    const int chunk = p->Ns;
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        const double* x = phys + (long long)b0 * p->M;
        expd_status st;
        if (p->bc != EXPD_BC_PERIODIC) {
            double* y = static_cast<double*>(eig) + (long long)b0 * p->Mcol;
            st = dst2(p, x, y, ns, static_cast<double*>(p->work64), s, -1);
        } else {
            double2* y = static_cast<double2*>(eig) + (long long)b0 * p->Mcol;
            if (p->ndim == 1) {
                st = launch_row<double, double, double2, 1>(p, x, y, ns, 1.0, s);
            } else {
                double2* w = static_cast<double2*>(p->work64);
                st = launch_row<double, double, double2, 1>(p, x, w, (long long)ns * p->NY, 1.0, s);
                if (st == EXPD_OK) st = launch_col<double, double2, double2>(p, w, y, ns, -1, 1.0, s);
            }
        }
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

expd_status spatial_inverse64(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s) {
    if (p->cplx) return spatial_complex64(p, static_cast<const double*>(eig), phys, nslices, +1, s);
    const int chunk = p->Ns;
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        double* x = phys + (long long)b0 * p->M;
        expd_status st;
        if (p->bc != EXPD_BC_PERIODIC) {
            const double* y = static_cast<const double*>(eig) + (long long)b0 * p->Mcol;
            st = dst2(p, y, x, ns, static_cast<double*>(p->work64), s, +1);
        } else {
            const double2* y = static_cast<const double2*>(eig) + (long long)b0 * p->Mcol;
            const double sx = 1.0 / (p->NX / 2);
            if (p->ndim == 1) {
                st = launch_row<double, double2, double, 0>(p, y, x, ns, sx, s);
            } else {
                double2* w = static_cast<double2*>(p->work64);
                st = launch_col<double, double2, double2>(p, y, w, ns, +1, 1.0 / p->NY, s);
                if (st == EXPD_OK) st = launch_row<double, double2, double, 0>(p, w, x, (long long)ns * p->NY, sx, s);
            }
        }
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

expd_status nonlinear_eval(expd_plan p, const void* Uh, void* out, int f32, cudaStream_t s, int in32) {
    const int Ns = p->Ns;
    if (in32) {
        // float32 iterate (periodic grids only): float32 transforms throughout
        if (p->bc != EXPD_BC_PERIODIC || !f32) return expd_fail(EXPD_ERR_INVALID_ARG, "float32 N needs a periodic grid");
        const float2* U = static_cast<const float2*>(Uh);
        float2* o = static_cast<float2*>(out);
        const long long rows = (long long)Ns * p->NY;
        const float sx = 1.0f / (p->NX / 2);
        if (p->ndim == 1) return launch_row<float, float2, float2, 2>(p, U, o, rows, sx, s);
        float2* w = static_cast<float2*>(p->work32);
        expd_status st = launch_col<float, float2, float2>(p, U, w, Ns, +1, 1.0f / p->NY, s);
        if (st == EXPD_OK) st = launch_row<float, float2, float2, 2>(p, w, w, rows, sx, s);
        if (st == EXPD_OK) st = launch_col<float, float2, float2>(p, w, o, Ns, -1, 1.0f, s);
        return st;
    }
    if (p->bc != EXPD_BC_PERIODIC) {
        // float64 only: inverse sine / cosine transform, N(u), forward transform
        double* phys = static_cast<double*>(p->work64) + (long long)Ns * p->M;
        expd_status st = spatial_inverse64(p, Uh, phys, Ns, s);
        if (st != EXPD_OK) return st;
        const long long n = (long long)Ns * p->M;
        KProf kp(p, s, EXPD_K_POINTWISE, 16.0 * n, 3.0 * n);
        nl_pointwise_kernel<<<grid_for(n, 256), 256, 0, s>>>(phys, n, p->nonlin);
        EXPD_CUDA_TRY(cudaGetLastError());
        return spatial_forward64(p, phys, out, Ns, s);
    }
    const double2* U = static_cast<const double2*>(Uh);
    const long long rows = (long long)Ns * p->NY;
    if (f32) {
        const float sx = 1.0f / (p->NX / 2);
        float2* o = static_cast<float2*>(out);
        if (p->ndim == 1) return launch_row<float, double2, float2, 2>(p, U, o, rows, sx, s);
        float2* w = static_cast<float2*>(p->work32);
        expd_status st = launch_col<float, double2, float2>(p, U, w, Ns, +1, 1.0f / p->NY, s);
        if (st == EXPD_OK) st = launch_row<float, float2, float2, 2>(p, w, w, rows, sx, s);
        if (st == EXPD_OK) st = launch_col<float, float2, float2>(p, w, o, Ns, -1, 1.0f, s);
        return st;
    }
    const double sx = 1.0 / (p->NX / 2);
    double2* o = static_cast<double2*>(out);
    if (p->ndim == 1) return launch_row<double, double2, double2, 2>(p, U, o, rows, sx, s);
    double2* w = static_cast<double2*>(p->work64);
    expd_status st = launch_col<double, double2, double2>(p, U, w, Ns, +1, 1.0 / p->NY, s);
    if (st == EXPD_OK) st = launch_row<double, double2, double2, 2>(p, w, w, rows, sx, s);
    if (st == EXPD_OK) st = launch_col<double, double2, double2>(p, w, o, Ns, -1, 1.0, s);
    return st;
}

expd_status convert_f64_to_f32(expd_plan p, const double* in, float* out, long long n, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 12.0 * n, 0.0);
    f64_to_f32_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status convert_f64_to_dd_inplace(expd_plan p, double* a, long long n, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 16.0 * n, 0.0);
    f64_to_dd_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, n);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status convert_f32_to_dd(expd_plan p, const float* in, void* out, long long n, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 12.0 * n, 0.0);
    EXPD_CUDA_TRY(launch_pdl(f32_to_dd_kernel, dim3(grid_for((n + 3) / 4, 256)), dim3(256), 0, s, in, static_cast<dd*>(out), n));
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status convert_f32_to_f64(expd_plan p, const float* in, double* out, long long n, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 12.0 * n, 0.0);
    f32_to_f64_kernel<<<grid_for(n, 256), 256, 0, s>>>(in, out, n);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status nonlinear_eval_dd(expd_plan p, const void* Uh, void* out, cudaStream_t s, double* const* phys_slot,
                              int x32) {
    if (p->bc != EXPD_BC_PERIODIC) return expd_fail(EXPD_ERR_INVALID_ARG, "double-float N needs a periodic grid");
    const dd2* U = static_cast<const dd2*>(Uh);
    const float2* U32 = static_cast<const float2*>(Uh);
    dd2* o = static_cast<dd2*>(out);
    const long long rows = (long long)p->Ns * p->NY;
    const dd sx(1.0 / (p->NX / 2));
    if (p->ndim == 1)
        return x32 ? launch_row<dd, float2, dd2, 2>(p, U32, o, rows, sx, s, phys_slot)
                   : launch_row<dd, dd2, dd2, 2>(p, U, o, rows, sx, s, phys_slot);
    dd2* w = static_cast<dd2*>(p->work64);
    expd_status st = x32 ? launch_col<dd, float2, dd2>(p, U32, w, p->Ns, +1, dd(1.0 / p->NY), s)
                         : launch_col<dd, dd2, dd2>(p, U, w, p->Ns, +1, dd(1.0 / p->NY), s);
    if (st == EXPD_OK) st = launch_row<dd, dd2, dd2, 2>(p, w, w, rows, sx, s, phys_slot);
    if (st == EXPD_OK) st = launch_col<dd, dd2, dd2>(p, w, o, p->Ns, -1, dd(1.0), s);
    return st;
}

bool inverse32_accum_supported(expd_plan p) {
    if (p->bc != EXPD_BC_PERIODIC || p->no_fft4 || !p->work32) return false;
    auto pow2 = [](int n) { return n >= 16 && n <= 1024 && (n & (n - 1)) == 0; };
    return p->NX >= 32 && p->NX <= 2048 && ((p->NX / 2) & (p->NX / 2 - 1)) == 0 && (p->ndim == 1 || pow2(p->NY));
}

expd_status spatial_inverse32_accum(expd_plan p, const void* eig, double* phys, cudaStream_t s) {
    if (!inverse32_accum_supported(p)) return expd_fail(EXPD_ERR_UNSUPPORTED, "float32 accumulating inverse transform");
    const float2* y = static_cast<const float2*>(eig);
    const float sx = 1.0f / (float)(p->NX / 2);
    const long long rows = (long long)p->Ns * p->NY;
    if (p->ndim == 1) return launch_row<float, float2, double, 3>(p, y, phys, rows, sx, s);
    float2* w = static_cast<float2*>(p->work32);
    expd_status st = launch_col<float, float2, float2>(p, y, w, p->Ns, +1, 1.0f / (float)p->NY, s);
    if (st == EXPD_OK) st = launch_row<float, float2, double, 3>(p, w, phys, rows, sx, s);
    return st;
}

expd_status spatial_inverse_dd(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s) {
    if (p->bc != EXPD_BC_PERIODIC) return expd_fail(EXPD_ERR_INVALID_ARG, "double-float transforms need a periodic grid");
    const int chunk = p->Ns;
    const dd sx(1.0 / (p->NX / 2));
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        double* x = phys + (long long)b0 * p->M;
        const dd2* y = static_cast<const dd2*>(eig) + (long long)b0 * p->Mcol;
        expd_status st;
        if (p->ndim == 1) {
            st = launch_row<dd, dd2, double, 0>(p, y, x, ns, sx, s);
        } else {
            dd2* w = static_cast<dd2*>(p->work64);
            st = launch_col<dd, dd2, dd2>(p, y, w, ns, +1, dd(1.0 / p->NY), s);
            if (st == EXPD_OK) st = launch_row<dd, dd2, double, 0>(p, w, x, (long long)ns * p->NY, sx, s);
        }
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

// float64 data transformed with double-float arithmetic on the float32
// pipes (2^-48 unit roundoff), for the start-up transforms of the mixed path
expd_status spatial_forward_dd64(expd_plan p, const double* phys, void* eig, int nslices, cudaStream_t s) {
    if (p->bc != EXPD_BC_PERIODIC || !p->Wxdd) return spatial_forward64(p, phys, eig, nslices, s);
    const int chunk = p->Ns;
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        const double* x = phys + (long long)b0 * p->M;
        double2* y = static_cast<double2*>(eig) + (long long)b0 * p->Mcol;
        expd_status st;
        if (p->ndim == 1) {
            st = launch_row<dd, double, double2, 1>(p, x, y, ns, dd(1.0), s);
        } else {
            dd2* w = static_cast<dd2*>(p->work64);
            st = launch_row<dd, double, dd2, 1>(p, x, w, (long long)ns * p->NY, dd(1.0), s);
            if (st == EXPD_OK) st = launch_col<dd, dd2, double2>(p, w, y, ns, -1, dd(1.0), s);
        }
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

expd_status spatial_inverse_dd64(expd_plan p, const void* eig, double* phys, int nslices, cudaStream_t s) {
    if (p->bc != EXPD_BC_PERIODIC || !p->Wxdd) return spatial_inverse64(p, eig, phys, nslices, s);
    const int chunk = p->Ns;
    const dd sx(1.0 / (p->NX / 2));
    for (int b0 = 0; b0 < nslices; b0 += chunk) {
        const int ns = std::min(chunk, nslices - b0);
        double* x = phys + (long long)b0 * p->M;
        const double2* y = static_cast<const double2*>(eig) + (long long)b0 * p->Mcol;
        expd_status st;
        if (p->ndim == 1) {
            st = launch_row<dd, double2, double, 0>(p, y, x, ns, sx, s);
        } else {
            dd2* w = static_cast<dd2*>(p->work64);
            st = launch_col<dd, double2, dd2>(p, y, w, ns, +1, dd(1.0 / p->NY), s);
            if (st == EXPD_OK) st = launch_row<dd, dd2, double, 0>(p, w, x, (long long)ns * p->NY, sx, s);
        }
        if (st != EXPD_OK) return st;
    }
    return EXPD_OK;
}

expd_status sum_squares(expd_plan p, const double* x, long long n, double* out_dev, double* scratch, cudaStream_t s) {
    const int nb = 64;
    KProf kp(p, s, EXPD_K_POINTWISE, 8.0 * n, 2.0 * n);
    sumsq_partial_kernel<<<nb, 256, 0, s>>>(x, n, scratch);
    EXPD_CUDA_TRY(cudaGetLastError());
    sumsq_final_kernel<<<1, 32, 0, s>>>(scratch, nb, out_dev);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status pointwise_solve(expd_plan p, const double* w, double* u, long long n, double bdt, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 16.0 * n, 30.0 * n);
    newton_kernel<<<grid_for(n, 256), 256, 0, s>>>(w, u, n, bdt, p->nonlin);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status etd_shift(expd_plan p, void* NL, int kind, cudaStream_t s) {
    const int eshift = p->realcol ? 0 : 1;
    const long long nelem = p->Mcol << eshift;
    const double esz = kind == 1 ? 4.0 : 8.0;
    KProf kp(p, s, EXPD_K_POINTWISE, 2.0 * esz * nelem * (p->Ns - 1), (double)nelem * p->Ns);
    const int grid = (int)std::min<long long>((nelem + 255) / 256, (long long)p->sm_count * 16);
    if (kind == 0)
        etd_shift_kernel<double, double><<<grid, 256, 0, s>>>(static_cast<double*>(NL), p->PHI64, nelem, eshift, p->Ns);
    else if (kind == 1)
        etd_shift_kernel<float, float><<<grid, 256, 0, s>>>(static_cast<float*>(NL), p->PHI32, nelem, eshift, p->Ns);
    else
        etd_shift_kernel<dd, dd><<<grid, 256, 0, s>>>(static_cast<dd*>(NL), static_cast<const dd*>(p->PHIdd), nelem,
                                                      eshift, p->Ns);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status etd_step(expd_plan p, void* out, const void* prev, const void* nl, cudaStream_t s) {
    const int eshift = p->realcol ? 0 : 1;
    const long long nelem = p->Mcol << eshift;
    KProf kp(p, s, EXPD_K_POINTWISE, 24.0 * nelem, 3.0 * nelem);
    etd_step_kernel<<<grid_for(nelem, 256), 256, 0, s>>>(static_cast<double*>(out), static_cast<const double*>(prev),
                                                        static_cast<const double*>(nl), p->E, p->PHI64, nelem, eshift);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status nonlinearity_eval_phys(expd_plan p, const double* u, double* out, long long n, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_POINTWISE, 16.0 * n, 3.0 * n);
    nl_eval_kernel<<<grid_for(n, 256), 256, 0, s>>>(u, out, n, p->nonlin);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status eigen_combine(expd_plan p, void* out, const void* const* in, const double* coef, int q,
                          const void* src, double g, cudaStream_t s) {
    CombineArgs a;
    for (int j = 0; j < 6; ++j) {
        a.in[j] = j < q ? static_cast<const double*>(in[j]) : nullptr;
        a.coef[j] = j < q ? coef[j] : 0.0;
    }
    a.q = q;
    a.src = static_cast<const double*>(src);
    a.g = g;
    a.out = static_cast<double*>(out);
    a.E = p->E;
    a.adv = p->adv;
    a.eshift = p->realcol ? 0 : 1;
    a.nelem = p->Mcol << a.eshift;
    KProf kp(p, s, EXPD_K_POINTWISE, 8.0 * a.nelem * (q + (src ? 2 : 1)), 2.0 * a.nelem * q);
    combine_kernel<<<grid_for(a.nelem, 256), 256, 0, s>>>(a);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status linear_guess(expd_plan p, void* X, int x32, cudaStream_t s) {
    const double* S = reinterpret_cast<const double*>(static_cast<const char*>(p->Sh) +
                                                      (size_t)(p->order - 1) * p->Mcol * p->esz);
    const int threads = 256;
    const long long blocks = std::max(1LL, std::min<long long>((p->Mcol + threads - 1) / threads, 32LL * p->sm_count));
    const double esz = (p->realcol ? 1.0 : 2.0) * (x32 ? 4.0 : 8.0);
    KProf kp(p, s, EXPD_K_POINTWISE, (double)p->Mcol * (p->esz + esz * p->Ns), 2.0 * (double)p->Mcol * p->Ns);
    if (x32) {
        float* Xf = static_cast<float*>(X);
        if (p->realcol) linear_guess_kernel<float, true, false><<<(int)blocks, threads, 0, s>>>(p->E, S, Xf, p->Mcol, p->Ns);
        else if (p->adv) linear_guess_kernel<float, false, true><<<(int)blocks, threads, 0, s>>>(p->E, S, Xf, p->Mcol, p->Ns);
        else linear_guess_kernel<float, false, false><<<(int)blocks, threads, 0, s>>>(p->E, S, Xf, p->Mcol, p->Ns);
    } else {
        double* Xd = static_cast<double*>(X);
        if (p->realcol) linear_guess_kernel<double, true, false><<<(int)blocks, threads, 0, s>>>(p->E, S, Xd, p->Mcol, p->Ns);
        else if (p->adv) linear_guess_kernel<double, false, true><<<(int)blocks, threads, 0, s>>>(p->E, S, Xd, p->Mcol, p->Ns);
        else linear_guess_kernel<double, false, false><<<(int)blocks, threads, 0, s>>>(p->E, S, Xd, p->Mcol, p->Ns);
    }
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status assemble_rhs(expd_plan p, const void* fh, cudaStream_t s, float* F32, int fh_dd, const void* nl0) {
    RhsArgs r;
    r.nl0 = static_cast<const double*>(nl0);
    r.phi = p->PHI64;
    r.fh = static_cast<const double*>(fh);
    r.Sh = static_cast<const double*>(p->Sh);
    r.Fh = static_cast<double*>(p->Fh);
    r.F32 = F32;
    r.fh_dd = fh_dd;
    r.E = p->E;
    r.adv = p->adv;
    for (int j = 0; j < 7; ++j) r.a[j] = p->acoef[p->order][j];
    r.bdt = p->beta[p->order] * p->dt;
    r.eshift = p->realcol ? 0 : 1;
    r.nelem = p->Mcol << r.eshift;
    r.s = p->order;
    r.Ns = p->Ns;
    KProf kp(p, s, EXPD_K_POINTWISE, 8.0 * r.nelem * ((fh ? 2.0 : 1.0) * r.Ns + r.s), 2.0 * r.nelem * r.s * r.s);
    // without a source only the first s slices (the start-up terms) are
    // nonzero: the time kernels read F as zero beyond them, so only those are
    // written
    const int ny = fh ? r.Ns : std::min(r.s, r.Ns);
    p->f_slices = ny;
    const long long bx = std::max(1LL, std::min<long long>((r.nelem + 255) / 256, (4LL * p->sm_count * 8) / ny + 1));
    rhs_kernel<<<dim3((unsigned)bx, (unsigned)ny), 256, 0, s>>>(r);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}
