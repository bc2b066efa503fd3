// Shared device helpers: complex arithmetic on double2/float2 and the
// warp-cooperative radix-2 FFTs on shared-memory buffers used by both the
// spatial transforms and the time-direction preconditioner.
//
// The FFT routines are __host__ __device__: on the GPU one warp runs them with
// `lane`/`nlanes` = lane id / 32, on the host a self-test runs them with
// lane 0 of 1 to check the index arithmetic without a GPU.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#ifdef __CUDA_ARCH__
#define EXPD_SYNCWARP() __syncwarp()
#else
#define EXPD_SYNCWARP() \
    do {                \
    } while (0)
#endif

#define EXPD_HD __host__ __device__ __forceinline__

// ---------------------------------------------------------------- complex ---
EXPD_HD double2 c2(double x, double y) { return make_double2(x, y); }
EXPD_HD float2 c2(float x, float y) { return make_float2(x, y); }

EXPD_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
EXPD_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
EXPD_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
EXPD_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
EXPD_HD double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
EXPD_HD float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
EXPD_HD double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
EXPD_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
EXPD_HD double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
EXPD_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// a * conj(b)
EXPD_HD double2 cmulc(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
EXPD_HD float2 cmulc(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// a / b
EXPD_HD double2 cdiv(double2 a, double2 b) {
    const double inv = 1.0 / fma(b.x, b.x, b.y * b.y);
    return cscale(cmulc(a, b), inv);
}
EXPD_HD float2 cdiv(float2 a, float2 b) {
    const float inv = 1.0f / fmaf(b.x, b.x, b.y * b.y);
    return cscale(cmulc(a, b), inv);
}
// i * a
EXPD_HD double2 cmuli(double2 a) { return make_double2(-a.y, a.x); }
EXPD_HD float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

EXPD_HD double2 to_c64(double2 a) { return a; }
EXPD_HD double2 to_c64(float2 a) { return make_double2((double)a.x, (double)a.y); }
template <typename T2>
EXPD_HD T2 from_c64(double2 a);
template <>
EXPD_HD double2 from_c64<double2>(double2 a) { return a; }
template <>
EXPD_HD float2 from_c64<float2>(double2 a) { return make_float2((float)a.x, (float)a.y); }

template <typename T>
struct cplx;
template <>
struct cplx<double> {
    typedef double2 t;
};
template <>
struct cplx<float> {
    typedef float2 t;
};

EXPD_HD unsigned bitrev(unsigned x, int log2n) {
#ifdef __CUDA_ARCH__
    return log2n == 0 ? 0u : (__brev(x) >> (32 - log2n));
#else
    unsigned r = 0;
    for (int i = 0; i < log2n; ++i) r |= ((x >> i) & 1u) << (log2n - 1 - i);
    return r;
#endif
}

EXPD_HD int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// ------------------------------------------------------------------- FFTs ---
// Twiddle convention: tw[k * ts] = exp(-2 pi i k / n) for 0 <= k < n/2, where
// ts is the stride of the table for this length (tables are shared between a
// length and its divisors).  sign = -1 transforms with exp(-2 pi i jk/n),
// sign = +1 with exp(+2 pi i jk/n); no normalisation.

// Decimation in time: x in bit-reversed order -> X in natural order.
template <typename T2>
EXPD_HD void fft_dit(T2* x, int log2n, const T2* tw, int ts, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    for (int s = 0; s < log2n; ++s) {
        const int h = 1 << s;
        const int tstep = (n >> (s + 1)) * ts;
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const int k = b & (h - 1);
            const int i = ((b >> s) << (s + 1)) + k;
            T2 w = tw[k * tstep];
            if (sign > 0) w.y = -w.y;
            const T2 u = x[i];
            const T2 v = cmul(x[i + h], w);
            x[i] = cadd(u, v);
            x[i + h] = csub(u, v);
        }
        EXPD_SYNCWARP();
    }
}

// Decimation in frequency: x in natural order -> X in bit-reversed order.
template <typename T2>
EXPD_HD void fft_dif(T2* x, int log2n, const T2* tw, int ts, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    for (int s = log2n - 1; s >= 0; --s) {
        const int h = 1 << s;
        const int tstep = (n >> (s + 1)) * ts;
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const int k = b & (h - 1);
            const int i = ((b >> s) << (s + 1)) + k;
            T2 w = tw[k * tstep];
            if (sign > 0) w.y = -w.y;
            const T2 u = x[i];
            const T2 v = x[i + h];
            x[i] = cadd(u, v);
            x[i + h] = cmul(csub(u, v), w);
        }
        EXPD_SYNCWARP();
    }
}

// Error checking used by every host launcher.
#define EXPD_CUDA_TRY(expr)                                                    \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) return expd_cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)
