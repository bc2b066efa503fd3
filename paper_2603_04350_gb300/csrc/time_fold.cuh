// Folded Bluestein passes shared by the time kernels of fixed window length
// (time_real.cu: real columns; time_cplx.cu: complex columns): radix-4 passes
// of one warp over a buffer of length 2^LOG2N in the swizzled index map
// padi<2>, with the chirp-z steps of the preconditioner solve folded into the
// first and last passes, and the per-pass twiddle-pair tables they read.
#pragma once

#include "common.cuh"

namespace expd_time {

// Bluestein passes of the real kernel (one warp, length 2^LOG2N, the
// swizzled buffer map padi<2>), with the pointwise steps of precond_step_a /
// precond_step_c folded in.  A Bluestein input is zero from Ns <= L/2 on, so
// the first DIF pass reads only the lower half; the kernel spectrum (bp or bm,
// stored in the DIF's bit-reversed output order) multiplies the last DIF
// pass's results; the last DIT pass stores only the lower half, the outputs
// k < Ns the solve reads.  The operations on the values kept, and their order,
// are those of fft_dif / fft_dit and the separate sweeps.
template <typename T2, int LOG2N, int SIGN>
__device__ __forceinline__ void bl_dif(T2* x, const TwPair<T2>* twp, const T2* tab, int lane) {
    constexpr int n = 1 << LOG2N;
    static_assert(LOG2N >= 6, "a warp of 32 lanes covers the radix-2 passes; the first pass is not the last");
    {  // first pass: span n/4, inputs x[i + n/2], x[i + 3n/4] are zero
        constexpr int h = n >> 2;
#pragma unroll 2
        for (int g0 = 0; g0 < h; g0 += 32) {
            const int i = g0 + lane;
            if (h < 32 && i >= h) break;
            const TwPair<T2> tp = twp[twp_offset(n, h) + i];
            T2 w2 = tp.w2, w4 = tp.w4;
            if (SIGN > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<2>(i)], x1 = x[padi<2>(i + h)];
            const T2 a2 = cmul(x0, w4);
            const T2 a3 = cmul_quarter(cmul(x1, w4), SIGN);
            x[padi<2>(i)] = cadd(x0, x1);
            x[padi<2>(i + h)] = cmul(csub(x0, x1), w2);
            x[padi<2>(i + 2 * h)] = cadd(a2, a3);
            x[padi<2>(i + 3 * h)] = cmul(csub(a2, a3), w2);
        }
        EXPD_SYNCWARP();
    }
#pragma unroll
    for (int s = LOG2N - 3; s >= 1; s -= 2) {
        const int h = 1 << (s - 1);
        const TwPair<T2>* tph = twp + twp_offset(n, h);
        const bool last = (s == 1);  // (LOG2N even: the last pass, spans 1)
#pragma unroll 2
        for (int g0 = 0; g0 < (n >> 2); g0 += 32) {
            const int g = g0 + lane;
            if ((n >> 2) < 32 && g >= (n >> 2)) break;
            const int k = g & (h - 1);
            const int i = ((g >> (s - 1)) << (s + 1)) + k;
            const TwPair<T2> tp = tph[k];
            T2 w2 = tp.w2, w4 = tp.w4;
            if (SIGN > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<2>(i)], x1 = x[padi<2>(i + h)], x2 = x[padi<2>(i + 2 * h)],
                     x3 = x[padi<2>(i + 3 * h)];
            const T2 a0 = cadd(x0, x2), a1 = cadd(x1, x3);
            const T2 a2 = cmul(csub(x0, x2), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x1, x3), w4), SIGN);
            T2 o0 = cadd(a0, a1), o1 = cmul(csub(a0, a1), w2), o2 = cadd(a2, a3), o3 = cmul(csub(a2, a3), w2);
            if (last) {
                o0 = cmul(o0, tab[i]);
                o1 = cmul(o1, tab[i + h]);
                o2 = cmul(o2, tab[i + 2 * h]);
                o3 = cmul(o3, tab[i + 3 * h]);
            }
            x[padi<2>(i)] = o0;
            x[padi<2>(i + h)] = o1;
            x[padi<2>(i + 2 * h)] = o2;
            x[padi<2>(i + 3 * h)] = o3;
        }
        EXPD_SYNCWARP();
    }
    if (LOG2N & 1) {  // the last pass is radix 2
#pragma unroll 2
        for (int b0 = 0; b0 < (n >> 1); b0 += 32) {
            const int b = b0 + lane;
            const T2 u = x[padi<2>(2 * b)], v = x[padi<2>(2 * b + 1)];
            x[padi<2>(2 * b)] = cmul(cadd(u, v), tab[2 * b]);
            x[padi<2>(2 * b + 1)] = cmul(csub(u, v), tab[2 * b + 1]);
        }
        EXPD_SYNCWARP();
    }
}

template <typename T2, int LOG2N, int SIGN>
__device__ __forceinline__ void bl_dit(T2* x, const TwPair<T2>* twp, int lane) {
    constexpr int n = 1 << LOG2N;
    if (LOG2N & 1) {
#pragma unroll 2
        for (int b0 = 0; b0 < (n >> 1); b0 += 32) {
            const int b = b0 + lane;
            const T2 u = x[padi<2>(2 * b)], v = x[padi<2>(2 * b + 1)];
            x[padi<2>(2 * b)] = cadd(u, v);
            x[padi<2>(2 * b + 1)] = csub(u, v);
        }
        EXPD_SYNCWARP();
    }
#pragma unroll
    for (int s = (LOG2N & 1); s < LOG2N; s += 2) {
        const int h = 1 << s;
        const TwPair<T2>* tph = twp + twp_offset(n, h);
        const bool last = (s == LOG2N - 2);  // span n/4: only outputs below n/2 are kept
#pragma unroll 2
        for (int g0 = 0; g0 < (n >> 2); g0 += 32) {
            const int g = g0 + lane;
            if ((n >> 2) < 32 && g >= (n >> 2)) break;
            const int k = g & (h - 1);
            const int i = ((g >> s) << (s + 2)) + k;
            const TwPair<T2> tp = tph[k];
            T2 w2 = tp.w2, w4 = tp.w4;
            if (SIGN > 0) {
                w2.y = -w2.y;
                w4.y = -w4.y;
            }
            const T2 x0 = x[padi<2>(i)], x1 = cmul(x[padi<2>(i + h)], w2);
            const T2 x2 = x[padi<2>(i + 2 * h)], x3 = cmul(x[padi<2>(i + 3 * h)], w2);
            const T2 a0 = cadd(x0, x1), a1 = csub(x0, x1);
            const T2 a2 = cmul(cadd(x2, x3), w4);
            const T2 a3 = cmul_quarter(cmul(csub(x2, x3), w4), SIGN);
            x[padi<2>(i)] = cadd(a0, a2);
            x[padi<2>(i + h)] = cadd(a1, a3);
            if (!last) {
                x[padi<2>(i + 2 * h)] = csub(a0, a2);
                x[padi<2>(i + 3 * h)] = csub(a1, a3);
            }
        }
        EXPD_SYNCWARP();
    }
}

}  // namespace expd_time
