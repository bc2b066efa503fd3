// Steps (a)-(c) of the preconditioner solve (Eq. (3.3) / Eq. (4.5)) on one
// time column of length Ns held in a buffer w of length L, executed by one warp
// (or, on the host self-test, by a single "lane").
//
// On entry w holds y_n = alpha^(n/Ns) q_n at position n (Bluestein, Ns not a
// power of two) or at position bitrev(n) (Ns = L a power of two).
// On exit position pos(n) (same rule) holds v_n with
//     s_n = v_n * scale / alpha^(n/Ns),
//     s   = Gamma^{-1} F^* diag(1/d) F Gamma q   (F: omega = e^{+2 pi i/Ns})
// where d_k = one - sum_{j=1..order} cj[j] lambda_k^j and cj[j] = a_j E^j
// (cj[1..6] valid, entries beyond `order` ignored; real, or complex with
// advection; one = 1 except for the shifted solve of the inexact Newton
// variant).
#pragma once

#include "common.cuh"

// Step (a): on exit w[k] holds Y_k (radix-2) or L Y_k (Bluestein), natural order.
// PAD selects the buffer's index map (padi): every access to w goes through it.
template <typename PT, typename PT2, int PAD = 0, int LOG2L = 0>
EXPD_HD void precond_step_a(PT2* w, int Ns, int L, int log2L, int bluestein, const PT2* tw, const PT2* chirp,
                            const PT2* bp, int lane, int nlanes) {
    if (bluestein) {
        for (int n = lane; n < Ns; n += nlanes) w[padi<PAD>(n)] = cmul(w[padi<PAD>(n)], chirp[n]);
        for (int n = Ns + lane; n < L; n += nlanes) w[padi<PAD>(n)] = c2((PT)0, (PT)0);
        EXPD_SYNCWARP();
        // Step (a) by chirp-z: Y_k = c_k sum_n (y_n c_n) conj(c_{k-n}),
        // the convolution as FFT_L^{-1}(FFT_L(.) * FFT_L(kernel)).
        if constexpr (LOG2L > 0) wfft_dif<PT2, PAD, LOG2L, -1>(w, tw, lane);
        else fft_dif<PT2, PAD>(w, log2L, tw, 1, -1, lane, nlanes);
        for (int k = lane; k < L; k += nlanes) w[padi<PAD>(k)] = cmul(w[padi<PAD>(k)], bp[k]);
        EXPD_SYNCWARP();
        if constexpr (LOG2L > 0) wfft_dit<PT2, PAD, LOG2L, +1>(w, tw, lane);
        else fft_dit<PT2, PAD>(w, log2L, tw, 1, +1, lane, nlanes);
        for (int k = lane; k < Ns; k += nlanes) w[padi<PAD>(k)] = cmul(w[padi<PAD>(k)], chirp[k]);  // = L * Y_k
        EXPD_SYNCWARP();
    } else {
        if constexpr (LOG2L > 0) wfft_dit<PT2, PAD, LOG2L, +1>(w, tw, lane);  // natural Y_k
        else fft_dit<PT2, PAD>(w, log2L, tw, 1, +1, lane, nlanes);
    }
}

// d_k = one - sum_{j=1..order} cp[j] lambda_k^j (Horner, unrolled over the at
// most six coefficients so they stay in registers)
template <typename PT, typename PT2, typename CJ>
EXPD_HD PT2 precond_divisor(PT2 lk, const CJ* cp, int order, PT one) {
    PT2 acc = c2((PT)0, (PT)0);
#pragma unroll
    for (int j = 6; j >= 1; --j) {
        if (j <= order) {
            acc = cmul(lk, acc);
            acc = acc_add(acc, cp[j]);
        }
    }
    acc = cmul(lk, acc);
    return c2(one - acc.x, -acc.y);
}

// Step (c) from Z_k in natural order (Bluestein: already times conj(c_k));
// returns the output scale.
template <typename PT, typename PT2, int PAD = 0, int LOG2L = 0>
EXPD_HD double precond_step_c(PT2* w, int Ns, int L, int log2L, int bluestein, const PT2* tw, const PT2* chirp,
                              const PT2* bm, int lane, int nlanes) {
    if (bluestein)
        for (int k = Ns + lane; k < L; k += nlanes) w[padi<PAD>(k)] = c2((PT)0, (PT)0);
    EXPD_SYNCWARP();
    // Step (c): z_n = sum_k Z_k e^{-2 pi i kn/Ns}
    if constexpr (LOG2L > 0) wfft_dif<PT2, PAD, LOG2L, -1>(w, tw, lane);
    else fft_dif<PT2, PAD>(w, log2L, tw, 1, -1, lane, nlanes);
    if (!bluestein) return 1.0 / Ns;  // bit-reversed output
    for (int k = lane; k < L; k += nlanes) w[padi<PAD>(k)] = cmul(w[padi<PAD>(k)], bm[k]);
    EXPD_SYNCWARP();
    if constexpr (LOG2L > 0) wfft_dit<PT2, PAD, LOG2L, +1>(w, tw, lane);
    else fft_dit<PT2, PAD>(w, log2L, tw, 1, +1, lane, nlanes);
    for (int n = lane; n < Ns; n += nlanes) w[padi<PAD>(n)] = cmulc(w[padi<PAD>(n)], chirp[n]);
    EXPD_SYNCWARP();
    return 1.0 / ((double)L * (double)L * (double)Ns);
}

template <typename PT, typename PT2, typename CJ, int PAD = 0>
EXPD_HD double precond_column(PT2* w, int Ns, int L, int log2L, int bluestein, const PT2* tw, const PT2* lam,
                              const PT2* chirp, const PT2* bp, const PT2* bm, const CJ* cj, int order,
                              int lane, int nlanes, PT one = (PT)1) {
    precond_step_a<PT, PT2, PAD>(w, Ns, L, log2L, bluestein, tw, chirp, bp, lane, nlanes);
    // Step (b): Z_k = Y_k / d_k
    CJ cp[7];
#pragma unroll
    for (int j = 1; j <= 6; ++j) cp[j] = j <= order ? cj[j] : coef_zero<CJ>();
    for (int k = lane; k < Ns; k += nlanes) {
        const PT2 d = precond_divisor<PT, PT2, CJ>(lam[k], cp, order, one);
        PT2 z = cdiv(w[padi<PAD>(k)], d);
        if (bluestein) z = cmulc(z, chirp[k]);
        w[padi<PAD>(k)] = z;
    }
    return precond_step_c<PT, PT2, PAD>(w, Ns, L, log2L, bluestein, tw, chirp, bm, lane, nlanes);
}

// The same solve for two real columns at once (real coefficients cj1, cj2):
// on entry w holds y1_n + i y2_n at position pos(n), on exit v1_n + i v2_n.
// The DFT of a real sequence is conjugate-symmetric (Y_{Ns-k} = conj(Y_k)),
// and so is d_k for real coefficients (lambda_{Ns-k} = conj(lambda_k)), so
// with W = DFT(y1 + i y2): Y1_k = (W_k + conj(W_{Ns-k})) / 2,
// Y2_k = (W_k - conj(W_{Ns-k})) / 2i, and Z1 + i Z2 goes into step (c).  One
// lane handles k and Ns - k together.  Two columns for the FFT work of one.
template <typename PT, typename PT2, int PAD = 0, int LOG2L = 0>
EXPD_HD double precond_column_pair(PT2* w, int Ns, int L, int log2L, int bluestein, const PT2* tw, const PT2* lam,
                                   const PT2* chirp, const PT2* bp, const PT2* bm, const PT* cj1, const PT* cj2,
                                   int order, int lane, int nlanes, PT one = (PT)1) {
    precond_step_a<PT, PT2, PAD, LOG2L>(w, Ns, L, log2L, bluestein, tw, chirp, bp, lane, nlanes);
    PT c1[7], c2v[7];
#pragma unroll
    for (int j = 1; j <= 6; ++j) {
        c1[j] = j <= order ? cj1[j] : (PT)0;
        c2v[j] = j <= order ? cj2[j] : (PT)0;
    }
    const PT h = (PT)0.5;
    for (int k = lane; k <= Ns / 2; k += nlanes) {
        const int kk = k == 0 ? 0 : Ns - k;
        const PT2 a = w[padi<PAD>(k)], b = w[padi<PAD>(kk)];
        const PT2 y1 = c2(h * (a.x + b.x), h * (a.y - b.y));
        const PT2 y2 = c2(h * (a.y + b.y), h * (b.x - a.x));
        const PT2 z1 = cdiv(y1, precond_divisor<PT, PT2, PT>(lam[k], c1, order, one));
        const PT2 z2 = cdiv(y2, precond_divisor<PT, PT2, PT>(lam[k], c2v, order, one));
        PT2 wk = c2(z1.x - z2.y, z1.y + z2.x);     // Z1_k + i Z2_k
        PT2 wkk = c2(z1.x + z2.y, z2.x - z1.y);    // conj(Z1_k) + i conj(Z2_k)
        if (bluestein) {
            wk = cmulc(wk, chirp[k]);
            wkk = cmulc(wkk, chirp[kk]);
        }
        w[padi<PAD>(k)] = wk;
        if (kk != k) w[padi<PAD>(kk)] = wkk;
    }
    return precond_step_c<PT, PT2, PAD, LOG2L>(w, Ns, L, log2L, bluestein, tw, chirp, bm, lane, nlanes);
}

#ifndef __CUDACC_RTC__
#include <math.h>

#include <complex>
#include <vector>

// Host construction of the time-direction tables for Ns unknown slices.
// Power-of-two Ns: radix-2 FFT of length L = Ns.  Otherwise Bluestein with
// L = the smallest power of two >= 2 Ns - 1, chirp c_n = e^{+i pi n^2/Ns} and
// the two convolution kernels' FFT_L stored in bit-reversed order.
struct TimeTablesHost {
    int L = 0, log2L = 0, bluestein = 0;
    std::vector<std::complex<double>> tw, lam, chirp, bplus, bminus;
    std::vector<double> gamma;
};

inline void host_fft_inplace(std::vector<std::complex<double>>& x, int sign) {
    const size_t n = x.size();
    for (size_t i = 1, j = 0; i < n; ++i) {
        size_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) std::swap(x[i], x[j]);
    }
    for (size_t len = 2; len <= n; len <<= 1)
        for (size_t i = 0; i < n; i += len)
            for (size_t k = 0; k < len / 2; ++k) {
                const double ang = sign * 2.0 * M_PI * (double)k / (double)len;
                const std::complex<double> w(cos(ang), sin(ang));
                const std::complex<double> u = x[i + k], v = x[i + k + len / 2] * w;
                x[i + k] = u + v;
                x[i + k + len / 2] = u - v;
            }
}

inline TimeTablesHost time_tables_host(int Ns, double alpha) {
    TimeTablesHost t;
    int L = 1;
    while (L < Ns) L <<= 1;
    t.bluestein = (L != Ns);
    if (t.bluestein) {
        L = 1;
        while (L < 2 * Ns - 1) L <<= 1;
    }
    t.L = L;
    t.log2L = ilog2(L);
    t.tw.resize(L / 2 > 0 ? L / 2 : 1);
    for (int k = 0; k < L / 2; ++k) t.tw[k] = std::polar(1.0, -2.0 * M_PI * k / L);
    t.lam.resize(Ns);
    t.gamma.resize(Ns);
    const double ar = pow(alpha, 1.0 / Ns);
    for (int k = 0; k < Ns; ++k) {
        t.lam[k] = std::polar(ar, 2.0 * M_PI * k / Ns);
        t.gamma[k] = pow(alpha, (double)k / Ns);
    }
    if (t.bluestein) {
        t.chirp.resize(Ns);
        for (int n = 0; n < Ns; ++n) {
            const long long r = ((long long)n * n) % (2LL * Ns);
            t.chirp[n] = std::polar(1.0, M_PI * (double)r / Ns);
        }
        for (int pass = 0; pass < 2; ++pass) {
            std::vector<std::complex<double>> b(L, 0.0);
            for (int j = 0; j < Ns; ++j) {
                const std::complex<double> cj = pass == 0 ? std::conj(t.chirp[j]) : t.chirp[j];
                b[j] = cj;
                if (j > 0) b[L - j] = cj;
            }
            host_fft_inplace(b, -1);
            std::vector<std::complex<double>> br(L);
            for (int k = 0; k < L; ++k) br[bitrev((unsigned)k, t.log2L)] = b[k];
            (pass == 0 ? t.bplus : t.bminus) = br;
        }
    }
    return t;
}
#endif
