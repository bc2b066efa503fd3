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
//
// Both routines fuse pairs of radix-2 stages: the four elements a pair of
// stages combines are held in registers, so each shared-memory round trip
// (and each warp synchronisation) covers two stages; an odd leftover stage has
// trivial twiddles.

// -i*a (sign < 0) or +i*a (sign > 0): the twiddle W_{4h}^h of a fused stage pair.
template <typename T2>
EXPD_HD T2 cmul_quarter(T2 a, int sign) {
    T2 r;
    if (sign > 0) {
        r.x = -a.y;
        r.y = a.x;
    } else {
        r.x = a.y;
        r.y = -a.x;
    }
    return r;
}

// Optional shared-memory padding for 16-byte elements: element i lives at
// i + 2 (i >> 3).  The radix-4 passes touch elements 0, 1, 8, 9, 16, 17, ...
// from consecutive lanes; unpadded, a quarter-warp's eight 16-byte accesses
// then fall on two bank groups (4-way conflicts), padded on eight.
// Shared-memory index maps of the warp FFT buffers.  PAD 1: two 16-byte slots
// of padding per eight elements (16-byte elements).  PAD 2: an XOR swizzle of
// the low four index bits by bits 4-5, i ^ 5 ((i >> 4) & 3), a bijection on
// every aligned block of 16 elements that keeps all radix-4 passes and the
// natural-order sweeps of lengths 64..1024 free of bank conflicts for 8-byte
// elements (at most two-way for 16-byte ones).
template <int PAD>
EXPD_HD int padi(int i) {
    if (PAD == 2) return i ^ (5 * ((i >> 4) & 3));
    return PAD ? i + ((i >> 3) << 1) : i;
}
template <int PAD>
EXPD_HD int padded_len(int n) { return PAD == 1 ? n + ((n >> 3) << 1) : n; }

// Decimation in time: x in bit-reversed order -> X in natural order.
template <typename T2, int PAD = 0>
EXPD_HD void fft_dit(T2* x, int log2n, const T2* tw, int ts, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    int s = 0;
    if (log2n & 1) {
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
            x[padi<PAD>(2 * b)] = cadd(u, v);
            x[padi<PAD>(2 * b + 1)] = csub(u, v);
        }
        EXPD_SYNCWARP();
        s = 1;
    }
    for (; s < log2n; s += 2) {
        const int h = 1 << s;
        const int t2 = (n >> (s + 1)) * ts;  // W_{2h}^k = tw[k * t2]
        const int t4 = (n >> (s + 2)) * ts;  // W_{4h}^k = tw[k * t4]
        for (int g = lane; g < (n >> 2); g += nlanes) {
            const int k = g & (h - 1);
            const int i = ((g >> s) << (s + 2)) + k;
            T2 w2 = tw[k * t2], w4 = tw[k * t4];
            if (sign > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<PAD>(i)], x1 = cmul(x[padi<PAD>(i + h)], w2);
            const T2 x2 = x[padi<PAD>(i + 2 * h)], x3 = cmul(x[padi<PAD>(i + 3 * h)], w2);
            const T2 a0 = cadd(x0, x1), a1 = csub(x0, x1);
            const T2 a2 = cmul(cadd(x2, x3), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x2, x3), w4), sign);
            x[padi<PAD>(i)] = cadd(a0, a2);
            x[padi<PAD>(i + 2 * h)] = csub(a0, a2);
            x[padi<PAD>(i + h)] = cadd(a1, a3);
            x[padi<PAD>(i + 3 * h)] = csub(a1, a3);
        }
        EXPD_SYNCWARP();
    }
}

// Decimation in frequency: x in natural order -> X in bit-reversed order.
template <typename T2, int PAD = 0>
EXPD_HD void fft_dif(T2* x, int log2n, const T2* tw, int ts, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    int s = log2n - 1;
    for (; s >= 1; s -= 2) {
        // stages s (span 2h) and s-1 (span h), h = 2^(s-1)
        const int h = 1 << (s - 1);
        const int t4 = (n >> (s + 1)) * ts;  // W_{4h}^k
        const int t2 = (n >> s) * ts;        // W_{2h}^k
        for (int g = lane; g < (n >> 2); g += nlanes) {
            const int k = g & (h - 1);
            const int i = ((g >> (s - 1)) << (s + 1)) + k;
            T2 w2 = tw[k * t2], w4 = tw[k * t4];
            if (sign > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<PAD>(i)], x1 = x[padi<PAD>(i + h)], x2 = x[padi<PAD>(i + 2 * h)],
                     x3 = x[padi<PAD>(i + 3 * h)];
            const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
            const T2 a2 = cmul(csub(x0, x2), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x1, x3), w4), sign);
            x[padi<PAD>(i)] = cadd(a0, a1);
            x[padi<PAD>(i + h)] = cmul(csub(a0, a1), w2);
            x[padi<PAD>(i + 2 * h)] = cadd(a2, a3);
            x[padi<PAD>(i + 3 * h)] = cmul(csub(a2, a3), w2);
        }
        EXPD_SYNCWARP();
    }
    if (s == 0) {
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
            x[padi<PAD>(2 * b)] = cadd(u, v);
            x[padi<PAD>(2 * b + 1)] = csub(u, v);
        }
        EXPD_SYNCWARP();
    }
}

// Twiddle pairs of the radix-4 passes, one table per pass span h: entry k < h
// holds (w4, w2) = (e^{-2 pi i k/(4h)}, e^{-2 pi i k/(2h)}), the two twiddles
// a butterfly of that span reads, so one load fetches both and consecutive
// lanes read consecutive entries (a strided read of the length-n table puts
// up to 8 lanes of a half-warp on one bank in the middle passes).  The spans
// are n/4, n/16, ... (both directions use the same set); the tables are stored
// largest span first.
template <typename T2>
struct __align__(2 * sizeof(T2)) TwPair {
    T2 w4, w2;
};

// offset of span h's table: the sizes of the larger spans before it
__host__ __device__ constexpr int twp_offset(int n, int h) {
    int off = 0;
    for (int q = n >> 2; q > h; q >>= 2) off += q;
    return off;
}
// entries of all the tables of length n
__host__ __device__ constexpr int twp_entries(int n) {
    int e = 0;
    for (int q = n >> 2; q >= 1; q >>= 2) e += q;
    return e;
}

// Fills the per-pass tables of length n (threads tid of nth) from a table
// with tw[j * ts] = e^{-2 pi i j/n}.
template <typename T2>
EXPD_HD void twp_build(TwPair<T2>* twp, const T2* tw, int ts, int n, int tid, int nth) {
    for (int h = n >> 2; h >= 1; h >>= 2)
        for (int k = tid; k < h; k += nth) {
            TwPair<T2> tp;
            tp.w4 = tw[k * (n / (4 * h)) * ts];
            tp.w2 = tw[k * (n / (2 * h)) * ts];
            twp[twp_offset(n, h) + k] = tp;
        }
}

// fft_dit / fft_dif reading their twiddles from the per-pass pair tables
// (the same arithmetic in the same order)
template <typename T2, int PAD = 0>
EXPD_HD void fft_dit_tp(T2* x, int log2n, const TwPair<T2>* twp, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    int s = 0;
    if (log2n & 1) {
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
            x[padi<PAD>(2 * b)] = cadd(u, v);
            x[padi<PAD>(2 * b + 1)] = csub(u, v);
        }
        EXPD_SYNCWARP();
        s = 1;
    }
    for (; s < log2n; s += 2) {
        const int h = 1 << s;
        const TwPair<T2>* tph = twp + twp_offset(n, h);
        for (int g = lane; g < (n >> 2); g += nlanes) {
            const int k = g & (h - 1);
            const int i = ((g >> s) << (s + 2)) + k;
            const TwPair<T2> tp = tph[k];
            T2 w2 = tp.w2, w4 = tp.w4;
            if (sign > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<PAD>(i)], x1 = cmul(x[padi<PAD>(i + h)], w2);
            const T2 x2 = x[padi<PAD>(i + 2 * h)], x3 = cmul(x[padi<PAD>(i + 3 * h)], w2);
            const T2 a0 = cadd(x0, x1), a1 = csub(x0, x1);
            const T2 a2 = cmul(cadd(x2, x3), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x2, x3), w4), sign);
            x[padi<PAD>(i)] = cadd(a0, a2);
            x[padi<PAD>(i + 2 * h)] = csub(a0, a2);
            x[padi<PAD>(i + h)] = cadd(a1, a3);
            x[padi<PAD>(i + 3 * h)] = csub(a1, a3);
        }
        EXPD_SYNCWARP();
    }
}

template <typename T2, int PAD = 0>
EXPD_HD void fft_dif_tp(T2* x, int log2n, const TwPair<T2>* twp, int sign, int lane, int nlanes) {
    const int n = 1 << log2n;
    int s = log2n - 1;
    for (; s >= 1; s -= 2) {
        const int h = 1 << (s - 1);
        const TwPair<T2>* tph = twp + twp_offset(n, h);
        for (int g = lane; g < (n >> 2); g += nlanes) {
            const int k = g & (h - 1);
            const int i = ((g >> (s - 1)) << (s + 1)) + k;
            const TwPair<T2> tp = tph[k];
            T2 w2 = tp.w2, w4 = tp.w4;
            if (sign > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<PAD>(i)], x1 = x[padi<PAD>(i + h)], x2 = x[padi<PAD>(i + 2 * h)],
                     x3 = x[padi<PAD>(i + 3 * h)];
            const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
            const T2 a2 = cmul(csub(x0, x2), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x1, x3), w4), sign);
            x[padi<PAD>(i)] = cadd(a0, a1);
            x[padi<PAD>(i + h)] = cmul(csub(a0, a1), w2);
            x[padi<PAD>(i + 2 * h)] = cadd(a2, a3);
            x[padi<PAD>(i + 3 * h)] = cmul(csub(a2, a3), w2);
        }
        EXPD_SYNCWARP();
    }
    if (s == 0) {
        for (int b = lane; b < (n >> 1); b += nlanes) {
            const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
            x[padi<PAD>(2 * b)] = cadd(u, v);
            x[padi<PAD>(2 * b + 1)] = csub(u, v);
        }
        EXPD_SYNCWARP();
    }
}

// The same radix-4 passes for one warp of 32 lanes with the length known at
// compile time (LOG2N) and the direction a template parameter: every pass and
// lane loop unrolls and the strides, spans and twiddle steps become constants.
// The arithmetic, and its order, is that of fft_dif / fft_dit.
template <typename T2, int PAD, int LOG2N, int SIGN>
EXPD_HD void wfft_dif(T2* x, const T2* tw, int lane) {
    constexpr int n = 1 << LOG2N;
#pragma unroll
    for (int s = LOG2N - 1; s >= 1; s -= 2) {
        const int h = 1 << (s - 1);
        const int t4 = n >> (s + 1);
        const int t2 = n >> s;
#pragma unroll 2
        for (int g0 = 0; g0 < (n >> 2); g0 += 32) {
            const int g = g0 + lane;
            if ((n >> 2) >= 32 || g < (n >> 2)) {
                const int k = g & (h - 1);
                const int i = ((g >> (s - 1)) << (s + 1)) + k;
                T2 w2 = tw[k * t2], w4 = tw[k * t4];
                if (SIGN > 0) {
                    w2.y = -w2.y;
                    w4.y = -w4.y;
                }
                const T2 x0 = x[padi<PAD>(i)], x1 = x[padi<PAD>(i + h)], x2 = x[padi<PAD>(i + 2 * h)],
                         x3 = x[padi<PAD>(i + 3 * h)];
                const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
                const T2 a2 = cmul(csub(x0, x2), w4);
                const T2 a3 = cmul_quarter(cmul(csub(x1, x3), w4), SIGN);
                x[padi<PAD>(i)] = cadd(a0, a1);
                x[padi<PAD>(i + h)] = cmul(csub(a0, a1), w2);
                x[padi<PAD>(i + 2 * h)] = cadd(a2, a3);
                x[padi<PAD>(i + 3 * h)] = cmul(csub(a2, a3), w2);
            }
        }
        EXPD_SYNCWARP();
    }
    if (LOG2N & 1) {
#pragma unroll
        for (int b0 = 0; b0 < (n >> 1); b0 += 32) {
            const int b = b0 + lane;
            if ((n >> 1) >= 32 || b < (n >> 1)) {
                const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
                x[padi<PAD>(2 * b)] = cadd(u, v);
                x[padi<PAD>(2 * b + 1)] = csub(u, v);
            }
        }
        EXPD_SYNCWARP();
    }
}

template <typename T2, int PAD, int LOG2N, int SIGN>
EXPD_HD void wfft_dit(T2* x, const T2* tw, int lane) {
    constexpr int n = 1 << LOG2N;
    if (LOG2N & 1) {
#pragma unroll
        for (int b0 = 0; b0 < (n >> 1); b0 += 32) {
            const int b = b0 + lane;
            if ((n >> 1) >= 32 || b < (n >> 1)) {
                const T2 u = x[padi<PAD>(2 * b)], v = x[padi<PAD>(2 * b + 1)];
                x[padi<PAD>(2 * b)] = cadd(u, v);
                x[padi<PAD>(2 * b + 1)] = csub(u, v);
            }
        }
        EXPD_SYNCWARP();
    }
#pragma unroll
    for (int s = (LOG2N & 1); s < LOG2N; s += 2) {
        const int h = 1 << s;
        const int t2 = n >> (s + 1);
        const int t4 = n >> (s + 2);
#pragma unroll 2
        for (int g0 = 0; g0 < (n >> 2); g0 += 32) {
            const int g = g0 + lane;
            if ((n >> 2) >= 32 || g < (n >> 2)) {
                const int k = g & (h - 1);
                const int i = ((g >> s) << (s + 2)) + k;
                T2 w2 = tw[k * t2], w4 = tw[k * t4];
                if (SIGN > 0) {
                    w2.y = -w2.y;
                    w4.y = -w4.y;
                }
                const T2 x0 = x[padi<PAD>(i)], x1 = cmul(x[padi<PAD>(i + h)], w2);
                const T2 x2 = x[padi<PAD>(i + 2 * h)], x3 = cmul(x[padi<PAD>(i + 3 * h)], w2);
                const T2 a0 = cadd(x0, x1), a1 = csub(x0, x1);
                const T2 a2 = cmul(cadd(x2, x3), w4);
                const T2 a3 = cmul_quarter(cmul(csub(x2, x3), w4), SIGN);
                x[padi<PAD>(i)] = cadd(a0, a2);
                x[padi<PAD>(i + 2 * h)] = csub(a0, a2);
                x[padi<PAD>(i + h)] = cadd(a1, a3);
                x[padi<PAD>(i + 3 * h)] = csub(a1, a3);
            }
        }
        EXPD_SYNCWARP();
    }
}

// ---- coefficient helpers: real a_j E^j (diffusion) or complex (advection) ----
// acc + c, and r - c x, for a real or a complex coefficient c
EXPD_HD float2 acc_add(float2 a, float c) { return make_float2(a.x + c, a.y); }
EXPD_HD float2 acc_add(float2 a, float2 c) { return cadd(a, c); }
EXPD_HD double2 acc_add(double2 a, double c) { return make_double2(a.x + c, a.y); }
EXPD_HD double2 acc_add(double2 a, double2 c) { return cadd(a, c); }
EXPD_HD float2 sub_cx(float2 r, float c, float2 x) { return make_float2(fmaf(-c, x.x, r.x), fmaf(-c, x.y, r.y)); }
EXPD_HD float2 sub_cx(float2 r, float2 c, float2 x) { return csub(r, cmul(c, x)); }
EXPD_HD double2 sub_cx(double2 r, double c, double2 x) { return make_double2(fma(-c, x.x, r.x), fma(-c, x.y, r.y)); }
EXPD_HD double2 sub_cx(double2 r, double2 c, double2 x) { return csub(r, cmul(c, x)); }
template <typename C>
EXPD_HD C coef_zero();
template <>
EXPD_HD float coef_zero<float>() { return 0.0f; }
template <>
EXPD_HD double coef_zero<double>() { return 0.0; }
template <>
EXPD_HD float2 coef_zero<float2>() { return make_float2(0.0f, 0.0f); }
template <>
EXPD_HD double2 coef_zero<double2>() { return make_double2(0.0, 0.0); }

// ------------------------------------------------------- register FFTs ---
// Length-R FFTs on a register array (compile-time indices, fully unrolled).
// tw[k * TS] = exp(-2 pi i k / R) for k < R/2 (a table of a longer length,
// read at stride TS); the quarter-turn twiddle is applied as a swap.
// SIGN < 0: exp(-2 pi i jk/R); SIGN > 0: exp(+2 pi i jk/R).
constexpr int ilog2_ct(int n) { return n <= 1 ? 0 : 1 + ilog2_ct(n >> 1); }

// DIT: bit-reversed in -> natural out
template <int R, int TS, int SIGN, typename T2>
EXPD_HD void reg_fft_dit(T2 (&v)[R], const T2* tw) {
#pragma unroll
    for (int st = 0; st < ilog2_ct(R); ++st) {
        const int h = 1 << st;
#pragma unroll
        for (int b = 0; b < R / 2; ++b) {
            const int k = b & (h - 1);
            const int i = ((b >> st) << (st + 1)) + k;
            T2 t = v[i + h];
            if (2 * k == h) {
                t = cmul_quarter(t, SIGN);  // exp(-+ i pi/2) = -+i, no table read
            } else if (k != 0) {
                T2 w = tw[k * (R / (2 * h)) * TS];
                if (SIGN > 0) w.y = -w.y;
                t = cmul(t, w);
            }
            v[i + h] = csub(v[i], t);
            v[i] = cadd(v[i], t);
        }
    }
}

// DIF: natural in -> bit-reversed out
template <int R, int TS, int SIGN, typename T2>
EXPD_HD void reg_fft_dif(T2 (&v)[R], const T2* tw) {
#pragma unroll
    for (int st = ilog2_ct(R) - 1; st >= 0; --st) {
        const int h = 1 << st;
#pragma unroll
        for (int b = 0; b < R / 2; ++b) {
            const int k = b & (h - 1);
            const int i = ((b >> st) << (st + 1)) + k;
            const T2 u = v[i], t = v[i + h];
            v[i] = cadd(u, t);
            T2 d = csub(u, t);
            if (2 * k == h) {
                d = cmul_quarter(d, SIGN);
            } else if (k != 0) {
                T2 w = tw[k * (R / (2 * h)) * TS];
                if (SIGN > 0) w.y = -w.y;
                d = cmul(d, w);
            }
            v[i + h] = d;
        }
    }
}

// ---- programmatic dependent launch ----
// Kernels of a sweep are launched so that each may start (load its constant
// tables into shared memory) while the previous one drains; pdl_wait() then
// blocks until the previous grid has completed and its writes are visible.
// Without a programmatic dependency (an ordinary launch) it returns at once.
__device__ __forceinline__ void pdl_wait() {
#ifdef __CUDA_ARCH__
    asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// Error checking used by every host launcher.
#define EXPD_CUDA_TRY(expr)                                                    \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) return expd_cuda_fail(_e, #expr, __FILE__, __LINE__); \
    } while (0)
