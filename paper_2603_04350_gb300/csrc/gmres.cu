// Vector kernels of the GMRES outer solver (Sec. 3.2): weighted multi-dot
// products and multi-axpy over space-time vectors held in L_h's eigenbasis.
//
// The inner product is the physical one: for the periodic half spectrum a
// mode with 0 < kx < NX/2 stands for itself and its conjugate and weighs 2
// (Parseval), so GMRES in the eigenbasis reproduces physical-space GMRES.
// Reductions are two-level with a fixed grid and fixed order (deterministic).
#include <algorithm>

#include "common.cuh"
#include "plan.h"

namespace {

constexpr int GM_THREADS = 256;
constexpr int GM_PER_THREAD = 4;
constexpr int GM_CHUNK = GM_THREADS * GM_PER_THREAD;

__device__ __forceinline__ double elem_weight(long long e, long long Mcol, int KX, int NX, int realcol) {
    if (realcol || KX == NX) return 1.0;  // real columns, or a complex state's full spectrum
    const long long m = (e >> 1) % Mcol;
    const int kx = (int)(m % KX);
    return (kx == 0 || 2 * kx == NX) ? 1.0 : 2.0;
}

// partial[i][block] = sum over this block's elements of w_e V_i[e] x[e], for
// the K (compile-time) vectors V_0..V_{K-1}: x is read once for all of them,
// the elements visited in a fixed order (deterministic).
constexpr int GM_DOTS = 8;

template <int K>
__global__ void __launch_bounds__(GM_THREADS) dots_kernel(const double* __restrict__ V, long long ld,
                                                          const double* __restrict__ x, long long n,
                                                          long long Mcol, int KX, int NX, int realcol,
                                                          double* __restrict__ partial) {
    __shared__ double red[K][GM_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc[K];
#pragma unroll
    for (int i = 0; i < K; ++i) acc[i] = 0.0;
    for (long long base = (long long)blockIdx.x * GM_CHUNK; base < n; base += (long long)gridDim.x * GM_CHUNK) {
#pragma unroll
        for (int t = 0; t < GM_PER_THREAD; ++t) {
            const long long e = base + t * GM_THREADS + threadIdx.x;
            if (e < n) {
                const double xe = elem_weight(e, Mcol, KX, NX, realcol) * x[e];
#pragma unroll
                for (int i = 0; i < K; ++i) acc[i] = fma(V[(long long)i * ld + e], xe, acc[i]);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        double a = acc[i];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) red[i][warp] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double t = 0.0;
        for (int w = 0; w < GM_THREADS / 32; ++w) t += red[threadIdx.x][w];
        partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// w = scale (w - sum_{i<k} c[i] V_i), partial[block] = sum of w_e (new w)^2
// over this block's elements (fixed order): the next Krylov basis vector and
// its norm in one pass.
__global__ void __launch_bounds__(GM_THREADS) update_norm_kernel(const double* __restrict__ V, long long ld, int k,
                                                                 const double* __restrict__ c, double scale,
                                                                 double* __restrict__ w, long long n, long long Mcol,
                                                                 int KX, int NX, int realcol,
                                                                 double* __restrict__ partial) {
    __shared__ double red[GM_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double acc = 0.0;
    for (long long base = (long long)blockIdx.x * GM_CHUNK; base < n; base += (long long)gridDim.x * GM_CHUNK) {
#pragma unroll
        for (int t = 0; t < GM_PER_THREAD; ++t) {
            const long long e = base + t * GM_THREADS + threadIdx.x;
            if (e < n) {
                double v = w[e];
                for (int i = 0; i < k; ++i) v = fma(-c[i], V[(long long)i * ld + e], v);
                v *= scale;
                w[e] = v;
                acc = fma(elem_weight(e, Mcol, KX, NX, realcol) * v, v, acc);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < GM_THREADS / 32; ++q) t += red[q];
        partial[blockIdx.x] = t;
    }
}

__global__ void dots_final(const double* __restrict__ partial, int grid, int k, double* __restrict__ h) {
    const int i = blockIdx.x;
    if (i >= k) return;
    __shared__ double red[32];
    double acc = 0.0;
    for (int g = threadIdx.x; g < grid; g += blockDim.x) acc += partial[(long long)i * grid + g];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        h[i] = s;
    }
}

__global__ void update_kernel(const double* __restrict__ V, long long ld, int k, const double* __restrict__ h,
                              double* __restrict__ x, long long n) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double acc = x[e];
        for (int i = 0; i < k; ++i) acc = fma(-h[i], V[(long long)i * ld + e], acc);
        x[e] = acc;
    }
}

// The same on 16-byte elements, two per thread and iteration (more loads in
// flight per thread), for an even element count and 16-byte-aligned vectors.
__global__ void __launch_bounds__(256) update_kernel_v(const double2* __restrict__ V, long long ld2, int k,
                                                       const double* __restrict__ h, double2* __restrict__ x,
                                                       long long n2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2; e += 2 * stride) {
        const long long e1 = e + stride;
        const bool two = e1 < n2;
        double2 a = x[e];
        double2 b = two ? x[e1] : make_double2(0.0, 0.0);
        for (int i = 0; i < k; ++i) {
            const double c = -h[i];
            const double2 va = __ldg(V + (long long)i * ld2 + e);
            a.x = fma(c, va.x, a.x);
            a.y = fma(c, va.y, a.y);
            if (two) {
                const double2 vb = __ldg(V + (long long)i * ld2 + e1);
                b.x = fma(c, vb.x, b.x);
                b.y = fma(c, vb.y, b.y);
            }
        }
        x[e] = a;
        if (two) x[e1] = b;
    }
}

// y = a x + b y; with b = 0, y is output only (it is not read: 0 * y would be
// NaN where y holds a non-finite value left by an earlier use of the buffer)
__global__ void axpby_kernel(long long n, double a, const double* x, double b, double* y) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = b == 0.0 ? a * x[e] : fma(a, x[e], b * y[e]);
}

// Complex states: partial[2i][block] and partial[2i+1][block] = real and
// imaginary parts of this block's share of <V_i, x> = sum conj(V_i) x over
// the complex elements (interleaved re, im doubles), fixed order.
template <int K>
__global__ void __launch_bounds__(GM_THREADS) cdots_kernel(const double2* __restrict__ V, long long ld2,
                                                           const double2* __restrict__ x, long long n2,
                                                           double* __restrict__ partial) {
    __shared__ double red[2 * K][GM_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double re[K], im[K];
#pragma unroll
    for (int i = 0; i < K; ++i) re[i] = im[i] = 0.0;
    for (long long base = (long long)blockIdx.x * GM_CHUNK; base < n2; base += (long long)gridDim.x * GM_CHUNK) {
#pragma unroll
        for (int t = 0; t < GM_PER_THREAD; ++t) {
            const long long e = base + t * GM_THREADS + threadIdx.x;
            if (e < n2) {
                const double2 xe = x[e];
#pragma unroll
                for (int i = 0; i < K; ++i) {
                    const double2 v = V[(long long)i * ld2 + e];
                    re[i] = fma(v.x, xe.x, fma(v.y, xe.y, re[i]));
                    im[i] = fma(v.x, xe.y, fma(-v.y, xe.x, im[i]));
                }
            }
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
        double a = re[i], b = im[i];
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_xor_sync(0xffffffffu, a, o);
            b += __shfl_xor_sync(0xffffffffu, b, o);
        }
        if (lane == 0) {
            red[2 * i][warp] = a;
            red[2 * i + 1][warp] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * K) {
        double t = 0.0;
        for (int w = 0; w < GM_THREADS / 32; ++w) t += red[threadIdx.x][w];
        partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// x -= sum_{i<k} h_i V_i with complex h_i = (h[2i], h[2i+1])
__global__ void cupdate_kernel(const double2* __restrict__ V, long long ld2, int k, const double* __restrict__ h,
                               double2* __restrict__ x, long long n2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n2;
         e += (long long)gridDim.x * blockDim.x) {
        double2 acc = x[e];
        for (int i = 0; i < k; ++i) {
            const double2 v = V[(long long)i * ld2 + e];
            const double hr = h[2 * i], hi = h[2 * i + 1];
            acc.x = fma(-hr, v.x, fma(hi, v.y, acc.x));
            acc.y = fma(-hr, v.y, fma(-hi, v.x, acc.y));
        }
        x[e] = acc;
    }
}

}  // namespace

long long eigen_elems(expd_plan p) { return (long long)p->Ns * p->Mcol * (p->realcol ? 1 : 2); }

// The dots partial buffer lives at the end of the GMRES block (see api.cu).
expd_status gm_dots(expd_plan p, const double* V, long long ld, int k, const double* w, double* h_dev,
                    cudaStream_t s) {
    const long long n = eigen_elems(p);
    const int grid = p->sm_count * 4;
    double* partial = h_dev + 128;  // caller reserves 128 + 65 * grid doubles
    KProf kp(p, s, EXPD_K_GMRES, 8.0 * (k + (k + GM_DOTS - 1) / GM_DOTS) * (double)n, 3.0 * k * (double)n);
    // chunks of up to GM_DOTS vectors per pass of x
    for (int i0 = 0; i0 < k; i0 += GM_DOTS) {
        const int kk = std::min(GM_DOTS, k - i0);
        const double* Vc = V + (long long)i0 * ld;
        double* pc = partial + (long long)i0 * grid;
        switch (kk) {
#define EXPD_DOTS_CASE(K)                                                                                      \
    case K:                                                                                                    \
        dots_kernel<K><<<grid, GM_THREADS, 0, s>>>(Vc, ld, w, n, p->Mcol, p->KX, p->NX, p->realcol, pc);     \
        break;
            EXPD_DOTS_CASE(1)
            EXPD_DOTS_CASE(2)
            EXPD_DOTS_CASE(3)
            EXPD_DOTS_CASE(4)
            EXPD_DOTS_CASE(5)
            EXPD_DOTS_CASE(6)
            EXPD_DOTS_CASE(7)
            EXPD_DOTS_CASE(8)
#undef EXPD_DOTS_CASE
        }
        EXPD_CUDA_TRY(cudaGetLastError());
    }
    dots_final<<<k, 256, 0, s>>>(partial, grid, k, h_dev);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status gm_update_norm(expd_plan p, const double* V, long long ld, int k, const double* c_dev, double scale,
                           double* w, double* h_dev, cudaStream_t s) {
    const long long n = eigen_elems(p);
    const int grid = p->sm_count * 4;
    double* partial = h_dev + 128;
    KProf kp(p, s, EXPD_K_GMRES, 8.0 * (k + 2) * (double)n, (2.0 * k + 3.0) * (double)n);
    update_norm_kernel<<<grid, GM_THREADS, 0, s>>>(V, ld, k, c_dev, scale, w, n, p->Mcol, p->KX, p->NX, p->realcol,
                                                   partial);
    EXPD_CUDA_TRY(cudaGetLastError());
    dots_final<<<1, 256, 0, s>>>(partial, grid, 1, h_dev);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status gm_update(expd_plan p, const double* V, long long ld, int k, const double* h_dev, double* w,
                      cudaStream_t s) {
    const long long n = eigen_elems(p);
    KProf kp(p, s, EXPD_K_GMRES, 8.0 * (k + 2) * (double)n, 2.0 * k * (double)n);
    const bool vec = (n % 2 == 0) && (ld % 2 == 0) && ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0;
    if (vec)
        update_kernel_v<<<p->sm_count * 8, 256, 0, s>>>(reinterpret_cast<const double2*>(V), ld / 2, k, h_dev,
                                                        reinterpret_cast<double2*>(w), n / 2);
    else
        update_kernel<<<p->sm_count * 8, 256, 0, s>>>(V, ld, k, h_dev, w, n);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status gm_axpby(expd_plan p, long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
    KProf kp(p, s, EXPD_K_GMRES, 24.0 * (double)n, 3.0 * (double)n);
    axpby_kernel<<<p->sm_count * 8, 256, 0, s>>>(n, a, x, b, y);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

// Complex states: h_dev[2i], h_dev[2i+1] = <V_i, w> = sum conj(V_i) w for
// i < k (k <= 65); per-block partials after the 256 result slots.
expd_status gm_cdots(expd_plan p, const double* V, long long ld, int k, const double* w, double* h_dev,
                     cudaStream_t s) {
    const long long n2 = eigen_elems(p) / 2;
    const int grid = p->sm_count * 4;
    double* partial = h_dev + 256;  // caller reserves 256 + 131 * grid doubles
    KProf kp(p, s, EXPD_K_GMRES, 16.0 * (k + (k + GM_DOTS - 1) / GM_DOTS) * (double)n2, 8.0 * k * (double)n2);
    const double2* V2 = reinterpret_cast<const double2*>(V);
    const double2* w2 = reinterpret_cast<const double2*>(w);
    for (int i0 = 0; i0 < k; i0 += GM_DOTS) {
        const int kk = std::min(GM_DOTS, k - i0);
        const double2* Vc = V2 + (long long)i0 * (ld / 2);
        double* pc = partial + 2LL * i0 * grid;
        switch (kk) {
#define EXPD_CDOTS_CASE(K)                                                                 \
    case K:                                                                                \
        cdots_kernel<K><<<grid, GM_THREADS, 0, s>>>(Vc, ld / 2, w2, n2, pc);               \
        break;
            EXPD_CDOTS_CASE(1)
            EXPD_CDOTS_CASE(2)
            EXPD_CDOTS_CASE(3)
            EXPD_CDOTS_CASE(4)
            EXPD_CDOTS_CASE(5)
            EXPD_CDOTS_CASE(6)
            EXPD_CDOTS_CASE(7)
            EXPD_CDOTS_CASE(8)
#undef EXPD_CDOTS_CASE
        }
        EXPD_CUDA_TRY(cudaGetLastError());
    }
    dots_final<<<2 * k, 256, 0, s>>>(partial, grid, 2 * k, h_dev);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}

expd_status gm_cupdate(expd_plan p, const double* V, long long ld, int k, const double* h_dev, double* x,
                       cudaStream_t s) {
    const long long n2 = eigen_elems(p) / 2;
    KProf kp(p, s, EXPD_K_GMRES, 16.0 * (k + 2) * (double)n2, 8.0 * k * (double)n2);
    cupdate_kernel<<<p->sm_count * 8, 256, 0, s>>>(reinterpret_cast<const double2*>(V), ld / 2, k, h_dev,
                                                   reinterpret_cast<double2*>(x), n2);
    EXPD_CUDA_TRY(cudaGetLastError());
    return EXPD_OK;
}
