// Host-only self-test of the device FFT routines and of the per-column
// preconditioner solve (time_column.cuh), run without a GPU: the routines are
// __host__ __device__ and run here with a single lane.  Compared with naive
// O(n^2) DFTs.  Exit status 0 on success.  Not part of libexpd.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <complex>
#include <random>
#include <vector>

#include "common.cuh"
#include "dd.cuh"
#include "dst_digits.cuh"
#include "time_column.cuh"

typedef std::complex<double> cd;

template <typename T2, typename T>
static std::vector<T2> to_dev(const std::vector<cd>& v) {
    std::vector<T2> o(v.size());
    for (size_t i = 0; i < v.size(); ++i) {
        o[i].x = (T)v[i].real();
        o[i].y = (T)v[i].imag();
    }
    return o;
}

static std::vector<cd> naive_dft(const std::vector<cd>& x, int sign) {
    const size_t n = x.size();
    std::vector<cd> X(n);
    for (size_t k = 0; k < n; ++k) {
        cd acc = 0;
        for (size_t j = 0; j < n; ++j) {
            const long long r = (long long)((k * j) % n);
            acc += x[j] * std::polar(1.0, sign * 2.0 * M_PI * (double)r / (double)n);
        }
        X[k] = acc;
    }
    return X;
}

static int failures = 0;

static void check(const char* what, double err, double tol, int a, int b) {
    if (!(err <= tol)) {
        printf("FAIL %s (%d, %d): err %.3e > %.1e\n", what, a, b, err, tol);
        ++failures;
    }
}

template <typename T, typename T2>
static void test_fft(int log2n, int sign, double tol, std::mt19937_64& rng) {
    const int n = 1 << log2n;
    std::normal_distribution<double> N01;
    std::vector<cd> x(n), tw(n / 2 > 0 ? n / 2 : 1);
    for (auto& v : x) v = cd(N01(rng), N01(rng));
    for (int k = 0; k < n / 2; ++k) tw[k] = std::polar(1.0, -2.0 * M_PI * k / n);
    const std::vector<cd> ref = naive_dft(x, sign);
    double scale = 0;
    for (auto& v : ref) scale = std::max(scale, std::abs(v));
    std::vector<T2> twd = to_dev<T2, T>(tw);
    // DIT: bit-reversed in, natural out
    std::vector<cd> xb(n);
    for (int j = 0; j < n; ++j) xb[bitrev(j, log2n)] = x[j];
    std::vector<T2> buf = to_dev<T2, T>(xb);
    fft_dit(buf.data(), log2n, twd.data(), 1, sign, 0, 1);
    double err = 0;
    for (int k = 0; k < n; ++k) err = std::max(err, std::abs(cd(buf[k].x, buf[k].y) - ref[k]));
    check(sizeof(T) == 8 ? "fft_dit double" : "fft_dit float", err / scale, tol, n, sign);
    // DIF: natural in, bit-reversed out
    buf = to_dev<T2, T>(x);
    fft_dif(buf.data(), log2n, twd.data(), 1, sign, 0, 1);
    err = 0;
    for (int k = 0; k < n; ++k) {
        const T2 v = buf[bitrev(k, log2n)];
        err = std::max(err, std::abs(cd(v.x, v.y) - ref[k]));
    }
    check(sizeof(T) == 8 ? "fft_dif double" : "fft_dif float", err / scale, tol, n, sign);
    // strided twiddle table (table of 2n used with stride 2)
    std::vector<cd> tw2(n);
    for (int k = 0; k < n; ++k) tw2[k] = std::polar(1.0, -2.0 * M_PI * k / (2 * n));
    std::vector<T2> tw2d = to_dev<T2, T>(tw2);
    buf = to_dev<T2, T>(xb);
    fft_dit(buf.data(), log2n, tw2d.data(), 2, sign, 0, 1);
    err = 0;
    for (int k = 0; k < n; ++k) err = std::max(err, std::abs(cd(buf[k].x, buf[k].y) - ref[k]));
    check("fft_dit strided table", err / scale, tol, n, sign);
    // padded layout (element i at i + 2 (i >> 3)), both directions
    std::vector<T2> pb((size_t)padded_len<1>(n));
    for (int j = 0; j < n; ++j) pb[padi<1>(bitrev(j, log2n))] = to_dev<T2, T>({x[j]})[0];
    fft_dit<T2, 1>(pb.data(), log2n, twd.data(), 1, sign, 0, 1);
    err = 0;
    for (int k = 0; k < n; ++k) err = std::max(err, std::abs(cd(pb[padi<1>(k)].x, pb[padi<1>(k)].y) - ref[k]));
    check("fft_dit padded", err / scale, tol, n, sign);
    for (int j = 0; j < n; ++j) pb[padi<1>(j)] = to_dev<T2, T>({x[j]})[0];
    fft_dif<T2, 1>(pb.data(), log2n, twd.data(), 1, sign, 0, 1);
    err = 0;
    for (int k = 0; k < n; ++k) {
        const T2 v = pb[padi<1>(bitrev(k, log2n))];
        err = std::max(err, std::abs(cd(v.x, v.y) - ref[k]));
    }
    check("fft_dif padded", err / scale, tol, n, sign);
}

// Register FFTs (compile-time length R, twiddles from a table of length R*TS
// read at stride TS), both directions, against the naive DFT.
template <typename T, typename T2, int R, int TS, int SIGN>
static void test_reg_fft(double tol, std::mt19937_64& rng) {
    std::normal_distribution<double> N01;
    std::vector<cd> x(R), tw(R * TS / 2);
    for (auto& v : x) v = cd(N01(rng), N01(rng));
    for (int k = 0; k < R * TS / 2; ++k) tw[k] = std::polar(1.0, -2.0 * M_PI * k / (R * TS));
    const std::vector<cd> ref = naive_dft(x, SIGN);
    double scale = 0;
    for (auto& v : ref) scale = std::max(scale, std::abs(v));
    const std::vector<T2> twd = to_dev<T2, T>(tw);
    const int lg = ilog2_ct(R);
    T2 v[R];
    for (int j = 0; j < R; ++j) v[bitrev(j, lg)] = to_dev<T2, T>({x[j]})[0];
    reg_fft_dit<R, TS, SIGN>(v, twd.data());
    double err = 0;
    for (int k = 0; k < R; ++k) err = std::max(err, std::abs(cd(v[k].x, v[k].y) - ref[k]));
    check(sizeof(T) == 8 ? "reg_fft_dit double" : "reg_fft_dit float", err / scale, tol, R, SIGN * TS);
    for (int j = 0; j < R; ++j) v[j] = to_dev<T2, T>({x[j]})[0];
    reg_fft_dif<R, TS, SIGN>(v, twd.data());
    err = 0;
    for (int k = 0; k < R; ++k) {
        const T2 w = v[bitrev(k, lg)];
        err = std::max(err, std::abs(cd(w.x, w.y) - ref[k]));
    }
    check(sizeof(T) == 8 ? "reg_fft_dif double" : "reg_fft_dif float", err / scale, tol, R, SIGN * TS);
}

template <typename T, typename T2, int R>
static void test_reg_fft_all(double tol, std::mt19937_64& rng) {
    test_reg_fft<T, T2, R, 1, -1>(tol, rng);
    test_reg_fft<T, T2, R, 1, +1>(tol, rng);
    test_reg_fft<T, T2, R, 4, -1>(tol, rng);
    test_reg_fft<T, T2, R, 4, +1>(tol, rng);
}

template <typename T, typename T2>
static void test_column(int Ns, int order, double E, double alpha, double tol, std::mt19937_64& rng) {
    static const double bdf[7][7] = {{0},
                                     {0, 1.0},
                                     {0, 4.0 / 3, -1.0 / 3},
                                     {0, 18.0 / 11, -9.0 / 11, 2.0 / 11},
                                     {0, 48.0 / 25, -36.0 / 25, 16.0 / 25, -3.0 / 25},
                                     {0, 300.0 / 137, -300.0 / 137, 200.0 / 137, -75.0 / 137, 12.0 / 137},
                                     {0, 360.0 / 147, -450.0 / 147, 400.0 / 147, -225.0 / 147, 72.0 / 147, -10.0 / 147}};
    const TimeTablesHost t = time_tables_host(Ns, alpha);
    std::normal_distribution<double> N01;
    std::vector<cd> q(Ns);
    for (auto& v : q) v = cd(N01(rng), N01(rng));
    double cj[7] = {0};
    double Ej = 1.0;
    for (int j = 1; j <= order; ++j) {
        Ej *= E;
        cj[j] = bdf[order][j] * Ej;
    }
    // reference: s = Gamma^{-1} F* diag(1/d) F Gamma q
    std::vector<cd> y(Ns);
    for (int n = 0; n < Ns; ++n) y[n] = t.gamma[n] * q[n];
    std::vector<cd> Y = naive_dft(y, +1);
    for (int k = 0; k < Ns; ++k) {
        cd d = 1.0, lk = t.lam[k], lp = 1.0;
        for (int j = 1; j <= order; ++j) {
            lp *= lk;
            d -= cj[j] * lp;
        }
        Y[k] /= d;
    }
    std::vector<cd> z = naive_dft(Y, -1);
    std::vector<cd> sref(Ns);
    double scale = 0;
    for (int n = 0; n < Ns; ++n) {
        sref[n] = z[n] / ((double)Ns * t.gamma[n]);
        scale = std::max(scale, std::abs(sref[n]));
    }
    // routine under test
    std::vector<cd> w(t.L, 0.0);
    for (int n = 0; n < Ns; ++n) w[t.bluestein ? n : bitrev(n, t.log2L)] = y[n];
    std::vector<T2> wd = to_dev<T2, T>(w), twd = to_dev<T2, T>(t.tw), lamd = to_dev<T2, T>(t.lam);
    std::vector<T2> chd = to_dev<T2, T>(t.chirp), bpd = to_dev<T2, T>(t.bplus), bmd = to_dev<T2, T>(t.bminus);
    T cjT[7];
    for (int j = 0; j < 7; ++j) cjT[j] = (T)cj[j];
    const double sc = precond_column<T, T2>(wd.data(), Ns, t.L, t.log2L, t.bluestein, twd.data(), lamd.data(),
                                            t.bluestein ? chd.data() : nullptr, t.bluestein ? bpd.data() : nullptr,
                                            t.bluestein ? bmd.data() : nullptr, cjT, order, 0, 1);
    double err = 0;
    for (int n = 0; n < Ns; ++n) {
        const T2 v = wd[t.bluestein ? n : bitrev(n, t.log2L)];
        const cd s = cd(v.x, v.y) * sc / t.gamma[n];
        err = std::max(err, std::abs(s - sref[n]));
    }
    check(sizeof(T) == 8 ? "precond_column double" : "precond_column float", err / scale, tol, Ns, order);

    // two real columns (this one's real part with E, a second with E2) packed
    // into one complex column, against two single-column solves
    std::vector<double> q1(Ns), q2(Ns);
    for (int n = 0; n < Ns; ++n) {
        q1[n] = N01(rng);
        q2[n] = N01(rng);
    }
    const double E2 = 0.5 * E + 0.1;
    T cj2[7] = {0};
    double Ej2 = 1.0;
    for (int j = 1; j <= order; ++j) {
        Ej2 *= E2;
        cj2[j] = (T)(bdf[order][j] * Ej2);
    }
    auto single = [&](const std::vector<double>& qq, const T* c) {
        std::vector<cd> ww(t.L, 0.0);
        for (int n = 0; n < Ns; ++n) ww[t.bluestein ? n : bitrev(n, t.log2L)] = t.gamma[n] * qq[n];
        std::vector<T2> wv = to_dev<T2, T>(ww);
        const double s1 = precond_column<T, T2>(wv.data(), Ns, t.L, t.log2L, t.bluestein, twd.data(), lamd.data(),
                                                t.bluestein ? chd.data() : nullptr, t.bluestein ? bpd.data() : nullptr,
                                                t.bluestein ? bmd.data() : nullptr, c, order, 0, 1);
        std::vector<double> out(Ns);
        for (int n = 0; n < Ns; ++n) out[n] = (double)wv[t.bluestein ? n : bitrev(n, t.log2L)].x * s1 / t.gamma[n];
        return out;
    };
    const std::vector<double> r1 = single(q1, cjT), r2 = single(q2, cj2);
    std::vector<cd> wp(t.L, 0.0);
    for (int n = 0; n < Ns; ++n) wp[t.bluestein ? n : bitrev(n, t.log2L)] = t.gamma[n] * cd(q1[n], q2[n]);
    std::vector<T2> wpd = to_dev<T2, T>(wp);
    const double sp = precond_column_pair<T, T2>(wpd.data(), Ns, t.L, t.log2L, t.bluestein, twd.data(), lamd.data(),
                                                 t.bluestein ? chd.data() : nullptr, t.bluestein ? bpd.data() : nullptr,
                                                 t.bluestein ? bmd.data() : nullptr, cjT, cj2, order, 0, 1);
    double perr = 0, pscale = 0;
    for (int n = 0; n < Ns; ++n) {
        const T2 v = wpd[t.bluestein ? n : bitrev(n, t.log2L)];
        perr = std::max(perr, std::max(std::fabs((double)v.x * sp / t.gamma[n] - r1[n]),
                                       std::fabs((double)v.y * sp / t.gamma[n] - r2[n])));
        pscale = std::max(pscale, std::max(std::fabs(r1[n]), std::fabs(r2[n])));
    }
    check(sizeof(T) == 8 ? "precond_column_pair double" : "precond_column_pair float", perr / pscale, tol, Ns, order);

    // the same pair solve on the swizzled buffer layout (padi<2>) of the
    // real-column kernel: identical values at every logical position
    std::vector<T2> wsw(t.L);
    for (int i = 0; i < t.L; ++i) wsw[padi<2>(i)] = to_dev<T2, T>(wp)[i];
    const double ss = precond_column_pair<T, T2, 2>(wsw.data(), Ns, t.L, t.log2L, t.bluestein, twd.data(), lamd.data(),
                                                    t.bluestein ? chd.data() : nullptr,
                                                    t.bluestein ? bpd.data() : nullptr,
                                                    t.bluestein ? bmd.data() : nullptr, cjT, cj2, order, 0, 1);
    double serr = 0;
    for (int n = 0; n < Ns; ++n) {
        const int pos = t.bluestein ? n : bitrev(n, t.log2L);
        const T2 a = wsw[padi<2>(pos)], b = wpd[pos];
        serr = std::max(serr, std::max(std::fabs((double)a.x * ss - (double)b.x * sp),
                                       std::fabs((double)a.y * ss - (double)b.y * sp)));
    }
    check(sizeof(T) == 8 ? "precond_column_pair swizzled double" : "precond_column_pair swizzled float",
          serr / pscale, 0.0, Ns, order);  // the same operations in the same order: bit-identical
}

// The integer-path conversions against the hardware ones: round to nearest
// even for float32 (bit-exact), and |hi + lo - v| <= 2^-47 |v| for
// double-float, over exponents spanning float's range, zeros and NaN.
static void test_conversions(std::mt19937_64& rng) {
    std::uniform_real_distribution<double> frac(1.0, 2.0);
    std::uniform_int_distribution<int> ex(-140, 140);
    int bad = 0;
    double worst = 0;
    for (int i = 0; i < 400000; ++i) {
        double v = ldexp(frac(rng), ex(rng));
        if (i & 1) v = -v;
        if (i % 97 == 0) v = nextafter((double)(float)v, 0.0);  // near a float tie / boundary
        const float f = f32_rn_from_f64(v);
        if (f != (float)v) ++bad;
        const dd d = dd_from_f64(v);
        const double r = (double)d.hi + (double)d.lo;
        if (fabs(v) >= ldexp(1.0, -74) && fabs(v) < ldexp(1.0, 127)) worst = std::max(worst, fabs(r - v) / fabs(v));
        if (fabs(d.lo) > ldexp(fabs((double)d.hi), -23)) ++bad;  // normalised pair
    }
    const double specials[] = {0.0, -0.0, 1.0, -1.0, 3.0e38, -3.4e38, 1e-40, 1e300};
    for (double v : specials)
        if (f32_rn_from_f64(v) != (float)v) ++bad;
    // exact float -> double widening: every float, specials included
    std::uniform_int_distribution<unsigned> bits32(0u, 0xffffffffu);
    for (int i = 0; i < 400000; ++i) {
        unsigned u = bits32(rng);
        float f;
        memcpy(&f, &u, 4);
        const double a = f64_from_f32(f), b = (double)f;
        if (!(a == b || (a != a && b != b)) || (a == 0.0 && std::signbit(a) != std::signbit(b))) ++bad;
    }
    // the flushing variant: the rounding of the hardware conversion on float's
    // normal range, signed zero below it
    for (int i = 0; i < 200000; ++i) {
        double v = ldexp(frac(rng), ex(rng));
        if (i & 1) v = -v;
        const float a = f32_ftz_from_f64(v);
        const float want = fabs(v) < ldexp(1.0, -126) ? (v < 0 ? -0.0f : 0.0f) : (float)v;
        if (a != want || std::signbit(a) != std::signbit(want)) ++bad;
    }
    if (f32_ftz_from_f64(-0.0) != 0.0f || !std::signbit(f32_ftz_from_f64(-0.0)) || f32_rn_from_f64(-0.0) != 0.0f ||
        !std::signbit(f32_rn_from_f64(-0.0)))
        ++bad;
    const float fspec[] = {0.0f, -0.0f, 1.0f, -1.0f, 3.4e38f, 1e-40f, -1e-45f, INFINITY, -INFINITY};
    for (float f : fspec)
        if (f64_from_f32(f) != (double)f) ++bad;
    const dd n = dd_from_f64(NAN);
    if (!(n.hi != n.hi)) ++bad;
    const dd z = dd_from_f64(0.0);
    if (z.hi != 0.0f || z.lo != 0.0f) ++bad;
    if (bad || worst > ldexp(1.0, -47)) {
        printf("FAIL conversions: %d mismatches, worst double-float error %.3e\n", bad, worst);
        ++failures;
    }
}

// Double-float complex products (cmul, cmulc) against long double, and a
// double-float register FFT against the naive DFT.
static void test_dd_complex(std::mt19937_64& rng) {
    std::normal_distribution<double> N01;
    std::uniform_int_distribution<int> ex(-20, 20);
    double worst = 0;
    for (int i = 0; i < 200000; ++i) {
        double v[4];
        for (double& x : v) x = ldexp(N01(rng), ex(rng));
        const dd2 a = c2(dd(v[0]), dd(v[1])), b = c2(dd(v[2]), dd(v[3]));
        typedef long double ld;
        const ld ax = (ld)a.x.hi + (ld)a.x.lo, ay = (ld)a.y.hi + (ld)a.y.lo;
        const ld bx = (ld)b.x.hi + (ld)b.x.lo, by = (ld)b.y.hi + (ld)b.y.lo;
        const ld scale = (fabsl(ax) + fabsl(ay)) * (fabsl(bx) + fabsl(by));
        const dd2 m = cmul(a, b), mc = cmulc(a, b);
        const ld err[4] = {(ld)m.x.hi + (ld)m.x.lo - (ax * bx - ay * by), (ld)m.y.hi + (ld)m.y.lo - (ax * by + ay * bx),
                           (ld)mc.x.hi + (ld)mc.x.lo - (ax * bx + ay * by),
                           (ld)mc.y.hi + (ld)mc.y.lo - (ay * bx - ax * by)};
        for (ld e : err) worst = std::max(worst, (double)(fabsl(e) / scale));
    }
    check("double-float complex products", worst, ldexp(1.0, -45), 0, 0);
    // 16-point register FFT in double-float
    constexpr int R = 16;
    std::vector<cd> x(R), tw(R / 2);
    for (auto& v : x) v = cd(N01(rng), N01(rng));
    for (int k = 0; k < R / 2; ++k) tw[k] = std::polar(1.0, -2.0 * M_PI * k / R);
    std::vector<dd2> twd(R / 2);
    for (int k = 0; k < R / 2; ++k) twd[k] = c2(dd(tw[k].real()), dd(tw[k].imag()));
    const std::vector<cd> ref = naive_dft(x, -1);
    dd2 v[R];
    for (int j = 0; j < R; ++j) v[bitrev(j, 4)] = c2(dd(x[j].real()), dd(x[j].imag()));
    reg_fft_dit<R, 1, -1>(v, twd.data());
    double e = 0, sc = 0;
    for (int k = 0; k < R; ++k) {
        e = std::max(e, std::abs(cd((double)v[k].x, (double)v[k].y) - ref[k]));
        sc = std::max(sc, std::abs(ref[k]));
    }
    check("reg_fft_dit double-float", e / sc, 1e-13, R, -1);
}

// ---- tensor-core DST: digits, packed operands, MMA descriptors ----------------
static uint16_t bf16_bits_of_int(int d) {
    const float f = (float)d;  // |d| <= 128: exact, and exact in bf16
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}
static double bf16_value(uint16_t h) {
    const uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return (double)f;
}
static unsigned long long bits_of(double v) {
    unsigned long long b;
    memcpy(&b, &v, 8);
    return b;
}

// the split kernel, row by row: exponents and packed digit slices
static void split_host(const std::vector<double>& x, long long rows, int K, int nsl, std::vector<uint16_t>& pack,
                       std::vector<int>& ex, int fixed_e) {
    pack.assign((size_t)nsl * rows * K, 0);
    ex.assign((size_t)rows, 0);
    for (long long r = 0; r < rows; ++r) {
        unsigned long long mx = 0;
        for (int k = 0; k < K; ++k) mx = std::max(mx, bits_of(x[r * K + k]) & 0x7FFFFFFFFFFFFFFFull);
        const int e = fixed_e != INT_MIN ? fixed_e : digit_row_exponent(mx);
        if (fixed_e != INT_MIN && mx >= bits_of(ldexp(1.0, e))) ++failures;  // the given exponent must bound the row
        ex[r] = e;
        for (int k = 0; k < K; ++k) {
            unsigned neg;
            unsigned long long Y = digit_magnitude(bits_of(x[r * K + k]), e, nsl, &neg);
            const unsigned long long Yo = Y + digit_offset(nsl);
            for (int i = nsl - 1; i >= 0; --i) {
                int d = digit_next(&Y, i);
                if (d != digit_at(Yo, i, nsl)) ++failures;  // the kernels' carry-free extraction
                if (i == 0 && (d < 0 || d > 128)) ++failures;
                if (i > 0 && (d < -64 || d > 63)) ++failures;
                if (neg) d = -d;
                pack[(size_t)i * rows * K + packed_offset(r, k, K / 64)] = bf16_bits_of_int(d);
            }
        }
    }
}

// One M = N = 128, K = 16 MMA with K-major operands, reading shared memory the
// way the descriptor fields say: element (m, k) at start + (m / 8) SBO +
// (m % 8) 16 + (k / 8) LBO + 2 (k % 8).
static void mma_emulate(const uint8_t* smem, uint64_t adesc, uint64_t bdesc, std::vector<double>& D, bool acc) {
    auto elem = [&](uint64_t desc, int m, int k) {
        const size_t start = (size_t)(desc & 0x3FFF) << 4, lbo = (size_t)((desc >> 16) & 0x3FFF) << 4,
                     sbo = (size_t)((desc >> 32) & 0x3FFF) << 4;
        uint16_t h;
        memcpy(&h, smem + start + (m / 8) * sbo + (m % 8) * 16 + (k / 8) * lbo + 2 * (k % 8), 2);
        return bf16_value(h);
    };
    if (((adesc >> 46) & 7) != 1 || ((bdesc >> 46) & 7) != 1 || (adesc >> 61) != 0) ++failures;
    for (int m = 0; m < 128; ++m)
        for (int n = 0; n < 128; ++n) {
            double s = acc ? D[m * 128 + n] : 0.0;
            for (int k = 0; k < 16; ++k) s += elem(adesc, m, k) * elem(bdesc, n, k);
            D[m * 128 + n] = s;
        }
}

// One pass of the tensor-core DST as the kernel schedules it: out (transposed
// within slices of R rows) = A B^T over the digit pairs i + j < nsl, B's
// digits with the one exponent eB, the pairs summed group by group.
static void tc_pass_host(const std::vector<double>& A, long long rows, int R, const std::vector<double>& B, int N, int K,
                         int nsl, int eB, std::vector<double>& out) {
    std::vector<uint16_t> pa, pb;
    std::vector<int> ea, eb;
    split_host(A, rows, K, nsl, pa, ea, INT_MIN);
    split_host(B, N, K, nsl, pb, eb, eB);
    int np = 0, ng = 0;
    unsigned char pi[32], pj[32], gstart[33], gw[32];
    tc_groups(nsl, K, &np, &ng, pi, pj, gstart, gw);
    if (np != nsl * (nsl + 1) / 2) ++failures;
    const int KB = K / 64;
    std::vector<uint8_t> smem(2 * 16384);
    std::vector<double> D(128 * 128), hi(128 * 128);
    out.assign((size_t)rows * N, 0.0);
    for (long long rt = 0; rt < rows / 128; ++rt)
        for (int ct = 0; ct < N / 128; ++ct) {
            for (int q = 0; q < ng; ++q) {
                for (int k = gstart[q]; k < gstart[q + 1]; ++k) {
                    const int i = pi[k], j = pj[k];
                    if (i + j != gw[q]) ++failures;
                    for (int kb = 0; kb < KB; ++kb) {
                        memcpy(smem.data(), pa.data() + (size_t)i * rows * K + ((size_t)rt * KB + kb) * 8192, 16384);
                        memcpy(smem.data() + 16384, pb.data() + (size_t)j * N * K + ((size_t)ct * KB + kb) * 8192,
                               16384);
                        for (int c = 0; c < 4; ++c)
                            mma_emulate(smem.data(), smem_desc(256u * c), smem_desc(16384u + 256u * c), D,
                                        k != gstart[q] || (kb | c) != 0);
                    }
                }
                for (int t = 0; t < 128 * 128; ++t) {
                    if (std::fabs(D[t]) > 16777216.0) ++failures;  // float32 accumulation must stay exact
                    const double w = ldexp(D[t], -7 * (gw[q] + 2));
                    hi[t] = q == 0 ? w : hi[t] + w;
                }
            }
            for (int m = 0; m < 128; ++m)
                for (int n = 0; n < 128; ++n) {
                    const long long row = rt * 128 + m, col = (long long)ct * 128 + n;
                    const long long sl = row / R, rin = row % R;
                    out[(size_t)(sl * R * N + col * R + rin)] = ldexp(hi[m * 128 + n], ea[row] + eB);
                }
        }
}

// The packed digit slices of S's folded halves (h = n/2 rows of h values,
// digit slices digit_rows(h) * h apart, S_e's then S_o's) for every size the
// tensor-core DST takes: no element written twice, every B tile the MMA
// kernel reads (128- or 64-row tiles, per 64-K step) lies on written elements
// of its own digit and half, and all of it within the n * n * nsl elements
// allocated per axis.
static void test_tc_s_layout() {
    for (int n = 128; n <= 1024; n += 128)
        for (int nsl = 3; nsl <= 7; ++nsl) {
            const long long h = n / 2, K = h, KB = K / 64, sl = digit_rows(h) * h;
            const long long total = (long long)nsl * n * n;
            std::vector<int> owner((size_t)total / 8, -1);  // 8-element groups: (half, digit) + 1
            bool ok = 2 * nsl * sl <= total;
            for (int half = 0; half < 2 && ok; ++half)
                for (int d = 0; d < nsl && ok; ++d)
                    for (long long r = 0; r < h && ok; ++r)
                        for (long long k = 0; k < K; k += 8) {
                            const long long e = half * nsl * sl + d * sl + packed_offset(r, (int)k, (int)KB);
                            if (e + 8 > total || owner[(size_t)(e / 8)] != -1) {
                                ok = false;
                                break;
                            }
                            owner[(size_t)(e / 8)] = half * 8 + d;
                        }
            const int BN = h % 128 ? 64 : 128;
            for (int half = 0; half < 2 && ok; ++half)
                for (int d = 0; d < nsl && ok; ++d)
                    for (long long ct = 0; ct < h / BN && ok; ++ct)
                        for (long long kb = 0; kb < KB && ok; ++kb) {
                            const long long boff = (ct * BN / 128) * KB * 8192 + ((ct * BN) % 128) * 64;
                            const long long start = half * nsl * sl + d * sl + boff + kb * 8192;
                            for (long long e = start; e < start + BN * 64; e += 8)
                                if (e + 8 > total || owner[(size_t)(e / 8)] != half * 8 + d) {
                                    ok = false;
                                    break;
                                }
                        }
            if (!ok) {
                ++failures;
                printf("FAIL tensor-core DST operand layout n %d nsl %d\n", n, nsl);
            }
        }
}

// every digit pair once, most significant weight first, each group of one
// weight and its worst-case float32 sum within 2^24
static void test_tc_groups() {
    for (int nsl = 1; nsl <= 7; ++nsl)
        for (int K = 64; K <= 1024; K += 64) {
            int np = 0, ng = 0;
            unsigned char pi[32], pj[32], gstart[33], gw[32];
            tc_groups(nsl, K, &np, &ng, pi, pj, gstart, gw);
            int seen[8][8] = {{0}};
            if (np != nsl * (nsl + 1) / 2 || ng < nsl || ng > np || gstart[0] != 0 || gstart[ng] != np) ++failures;
            for (int q = 0; q < ng; ++q) {
                long long sum = 0;
                if (gstart[q + 1] <= gstart[q] || (q > 0 && gw[q] < gw[q - 1])) ++failures;
                for (int k = gstart[q]; k < gstart[q + 1]; ++k) {
                    if (pi[k] + pj[k] != gw[q]) ++failures;
                    ++seen[pi[k]][pj[k]];
                    sum += (long long)K * (pi[k] ? 64 : 128) * (pj[k] ? 64 : 128);
                }
                if (sum > (1LL << 24)) ++failures;
            }
            for (int i = 0; i < nsl; ++i)
                for (int j = 0; j < nsl; ++j)
                    if (seen[i][j] != (i + j < nsl ? 1 : 0)) ++failures;
            if (K == 1024 && nsl == 6 && ng != 10) ++failures;  // 21 pairs in 10 groups at the 1024^2 workload
        }
}

static void test_tc_dst(std::mt19937_64& rng) {
    const int NY = 256, NX = 128, ns = 2, nsl = 5;
    auto dst = [](int n) {
        std::vector<double> S((size_t)n * n);
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k) S[(size_t)j * n + k] = sqrt(2.0 / (n + 1)) * sin(M_PI * (j + 1.0) * (k + 1.0) / (n + 1));
        return S;
    };
    const std::vector<double> Sx = dst(NX), Sy = dst(NY);
    std::normal_distribution<double> N01;
    std::vector<double> X((size_t)ns * NY * NX);
    for (size_t t = 0; t < X.size(); ++t) X[t] = N01(rng) * ((t % 7) == 0 ? 1e3 : 1.0);  // uneven row scales
    std::vector<double> T, Y;
    auto ebound = [](int n) {  // the exponent the library gives the DST digits
        int e;
        frexp(sqrt(2.0 / (n + 1)), &e);
        return e;
    };
    tc_pass_host(X, (long long)ns * NY, NY, Sx, NX, NX, nsl, ebound(NX), T);   // T[s] = (X[s] S_x)^T
    tc_pass_host(T, (long long)ns * NX, NX, Sy, NY, NY, nsl, ebound(NY), Y);   // Y[s] = (T[s] S_y)^T = S_y X[s] S_x
    double e2 = 0, r2 = 0;
    for (int s = 0; s < ns; ++s)
        for (int y = 0; y < NY; ++y)
            for (int x = 0; x < NX; ++x) {
                double ref = 0;
                for (int a = 0; a < NY; ++a) {
                    double t = 0;
                    for (int b = 0; b < NX; ++b) t += X[((size_t)s * NY + a) * NX + b] * Sx[(size_t)b * NX + x];
                    ref += Sy[(size_t)y * NY + a] * t;
                }
                const double d = Y[((size_t)s * NY + y) * NX + x] - ref;
                e2 += d * d;
                r2 += ref * ref;
            }
    check("tensor-core DST (digits, packing, descriptors)", sqrt(e2 / r2), 1e-9, NY, NX);
}

int main() {
    std::mt19937_64 rng(1234);
    test_conversions(rng);
    test_dd_complex(rng);
    test_tc_groups();
    test_tc_s_layout();
    test_tc_dst(rng);
    for (int l = 1; l <= 12; ++l)
        for (int sign = -1; sign <= 1; sign += 2) {
            test_fft<double, double2>(l, sign, 1e-13, rng);
            test_fft<float, float2>(l, sign, 2e-5, rng);
        }
    test_reg_fft_all<double, double2, 2>(1e-14, rng);
    test_reg_fft_all<double, double2, 4>(1e-14, rng);
    test_reg_fft_all<double, double2, 8>(1e-14, rng);
    test_reg_fft_all<double, double2, 16>(1e-14, rng);
    test_reg_fft_all<double, double2, 32>(1e-14, rng);
    test_reg_fft_all<float, float2, 4>(1e-6, rng);
    test_reg_fft_all<float, float2, 16>(2e-6, rng);
    test_reg_fft_all<float, float2, 32>(2e-6, rng);
    const int sizes[] = {2, 3, 4, 5, 7, 8, 11, 15, 16, 27, 31, 32, 59, 63, 64, 123, 127, 128, 251, 255, 256, 1000};
    const int orders[] = {1, 2, 3, 6};
    const double Es[] = {1.0, 0.7, 0.0};
    for (int Ns : sizes)
        for (int order : orders) {
            if (Ns < order + 1) continue;
            for (double E : Es) {
                test_column<double, double2>(Ns, order, E, 1e-3, 1e-11, rng);
                test_column<double, double2>(Ns, order, E, 0.3, 1e-12, rng);
                test_column<float, float2>(Ns, order, E, 0.3, 1e-4 * std::max(1.0, Ns / 256.0), rng);
                test_column<float, float2>(Ns, order, E, 1e-3, 3e-3, rng);
            }
        }
    if (failures) {
        printf("%d failures\n", failures);
        return 1;
    }
    printf("OK\n");
    return 0;
}
