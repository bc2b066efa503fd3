// Double-float ("dd") arithmetic: a value is the unevaluated sum hi + lo of two
// floats with |lo| <= ulp(hi)/2, giving a 48-bit significand (unit roundoff
// 2^-48 ~ 3.6e-15) computed entirely on the float32 pipes.  GB300 executes
// float64 at 1/58 of its float32 rate, so a dd butterfly (~100 float32
// operations) costs about a fifth of a float64 one.
//
// Building blocks are the error-free transformations: Knuth's two-sum (exact
// a + b = s + e for any floats), the fast two-sum for |a| >= |b| (Dekker), and
// the FMA two-product (exact a * b = p + e).  Addition here is the "sloppy"
// variant (one two-sum of the high parts, low parts added then renormalised):
// its error is bounded by 2^-46 (|x| + |y|), which is what the normwise error
// analysis of an FFT butterfly needs.
#pragma once

#include <string.h>

#include "common.cuh"

// ---- float64 -> float32 / double-float by integer operations -------------
// GB300 runs float64 arithmetic and float64 conversions on a pipe 1/58 the
// rate of float32, so converting a large float64 array is ALU-bound.  These
// split the binary64 encoding with integer operations instead: sign, the
// 11-bit exponent e and the 52 fraction bits.
EXPD_HD unsigned long long f64_bits(double v) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(v);
#else
    unsigned long long b;
    memcpy(&b, &v, 8);
    return b;
#endif
}
EXPD_HD float f32_from_bits(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

// The ordinary (float64-pipe) conversions of the rare operands -- subnormal
// results, values beyond float's range, infinities, NaN -- are out of line:
// inlined, the compiler evaluates them for every element and selects, which
// puts one float64-pipe instruction on every conversion.
#ifdef __CUDA_ARCH__
static __device__ __noinline__ float f32_of_f64_rare(double v) { return (float)v; }
static __device__ __noinline__ double f64_of_f32_rare(float f) { return (double)f; }
#else
inline float f32_of_f64_rare(double v) { return (float)v; }
inline double f64_of_f32_rare(float f) { return (double)f; }
#endif

// Round to nearest even, as the hardware conversion; values whose float is
// subnormal, zero, infinite or NaN take the ordinary conversion.
EXPD_HD float f32_rn_from_f64(double v) {
    const unsigned long long b = f64_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if ((b << 1) == 0ull) return f32_from_bits((unsigned)(b >> 63) << 31);  // signed zero
    if (e < 897 || e > 1150) return f32_of_f64_rare(v);  // outside float's normal range
    const unsigned long long m = b & 0xfffffffffffffULL;
    unsigned u = ((unsigned)(b >> 63) << 31) | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29);
    const unsigned long long tail = m & 0x1fffffffULL;  // the 29 dropped bits
    if (tail > 0x10000000ULL || (tail == 0x10000000ULL && (u & 1u))) ++u;  // carries into the exponent
    return f32_from_bits(u);
}

// Exact float -> double by integer operations (every float is a double):
// normal values rebias the exponent and widen the fraction, subnormals are
// normalised by their leading-zero count, zeros keep their sign; infinities
// and NaN take the ordinary conversion.
EXPD_HD double f64_from_f32(float f) {
#ifdef __CUDA_ARCH__
    const unsigned u = __float_as_uint(f);
#else
    unsigned u;
    memcpy(&u, &f, 4);
#endif
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    unsigned long long b;
    if (e == 0u) {
        if (m == 0u) {
            b = (unsigned long long)(u >> 31) << 63;  // signed zero
        } else {
            // subnormal: m 2^-149 = 1.f 2^(22 - z - 149), z leading zeros of m in 23 bits
#ifdef __CUDA_ARCH__
            const int z = __clz(m) - 9;
#else
            const int z = __builtin_clz(m) - 9;
#endif
            b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(896 - z) << 52) |
                ((unsigned long long)((m << (z + 1)) & 0x7fffffu) << 29);
        }
    } else if (e == 0xffu) {
        return f64_of_f32_rare(f);  // infinity, NaN
    } else {
        b = ((unsigned long long)(u >> 31) << 63) | ((unsigned long long)(e + 896u) << 52) |
            ((unsigned long long)m << 29);
    }
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, 8);
    return d;
#endif
}

// The same with magnitudes below float's normal range (|v| < 2^-126) flushed
// to signed zero, all by integer operations: the input conversion of the
// float32 preconditioner, whose float32 transforms hold values relative to
// the largest one, far above 2^-126 (finite values above float's range take the
// hardware conversion, to infinity).
EXPD_HD float f32_ftz_from_f64(double v) {
    const unsigned long long b = f64_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e < 897) return f32_from_bits((unsigned)(b >> 63) << 31);
    if (e > 1150) return f32_of_f64_rare(v);
    const unsigned long long m = b & 0xfffffffffffffULL;
    unsigned u = ((unsigned)(b >> 63) << 31) | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29);
    const unsigned long long tail = m & 0x1fffffffULL;
    if (tail > 0x10000000ULL || (tail == 0x10000000ULL && (u & 1u))) ++u;
    return f32_from_bits(u);
}

struct dd;
EXPD_HD dd dd_from_f64(double v);

struct dd {
    float hi, lo;
    dd() = default;
    EXPD_HD explicit dd(double v);
    EXPD_HD explicit dd(float v) : hi(v), lo(0.0f) {}
    EXPD_HD explicit dd(int v) : hi((float)v), lo(0.0f) {}
    EXPD_HD dd(float h, float l) : hi(h), lo(l) {}
    EXPD_HD explicit operator double() const { return (double)hi + (double)lo; }
    EXPD_HD explicit operator float() const { return hi + lo; }
};

struct dd2 {
    dd x, y;
};

template <>
struct cplx<dd> {
    typedef dd2 t;
};

EXPD_HD dd dd_fast_two_sum(float a, float b) {
    const float s = a + b;
    return dd(s, b - (s - a));
}

// hi = the leading 24 significand bits (truncated), lo = the next 29 bits
// rounded to a float, renormalised: hi + lo equals v to 2^-48 relative.
// |v| < 2^-74 keeps hi only (lo would be subnormal), |v| < 2^-126 gives 0,
// |v| >= 2^128, infinities and NaN take the float64 path (NaN propagates).
EXPD_HD dd dd_from_f64(double v) {
    const unsigned long long b = f64_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned sgn = (unsigned)(b >> 63) << 31;
    if (e > 1150) {
        const float h = (float)v;
        return dd(h, 0.0f);
    }
    if (e < 897) return dd(f32_from_bits(sgn), 0.0f);
    const unsigned long long m = b & 0xfffffffffffffULL;
    const float hi = f32_from_bits(sgn | ((unsigned)(e - 896) << 23) | (unsigned)(m >> 29));
    if (e < 949) return dd(hi, 0.0f);
    // (m mod 2^29) * 2^(e - 1075); 2^(e - 1075) is a normal float for e >= 949
    float lo = (float)(unsigned)(m & 0x1fffffffULL) * f32_from_bits((unsigned)(e - 948) << 23);
    if (sgn) lo = -lo;
    return dd_fast_two_sum(hi, lo);
}

EXPD_HD dd::dd(double v) { *this = dd_from_f64(v); }

EXPD_HD dd dd_two_sum(float a, float b) {
    const float s = a + b;
    const float v = s - a;
    return dd(s, (a - (s - v)) + (b - v));
}

EXPD_HD dd operator+(dd a, dd b) {
    const dd s = dd_two_sum(a.hi, b.hi);
    return dd_fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
EXPD_HD dd operator-(dd a) { return dd(-a.hi, -a.lo); }
EXPD_HD dd operator-(dd a, dd b) { return a + (-b); }
EXPD_HD dd operator*(dd a, dd b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return dd_fast_two_sum(p, e);
}
EXPD_HD dd operator*(dd a, float b) {
    const float p = a.hi * b;
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return dd_fast_two_sum(p, e);
}
EXPD_HD dd fma(dd a, dd b, dd c) { return a * b + c; }
EXPD_HD dd& operator+=(dd& a, dd b) {
    a = a + b;
    return a;
}

// ---- complex dd, with the same names as the double2/float2 helpers ----
EXPD_HD dd2 c2(dd x, dd y) {
    dd2 r;
    r.x = x;
    r.y = y;
    return r;
}
EXPD_HD dd2 cadd(dd2 a, dd2 b) { return c2(a.x + b.x, a.y + b.y); }
EXPD_HD dd2 csub(dd2 a, dd2 b) { return c2(a.x - b.x, a.y - b.y); }
// a b + s c d (s = +-1) with one renormalisation: the two leading products
// and their exact errors (fma), an exact two-sum of the leading products, and
// the cross terms accumulated in float (a.lo b.lo, of relative size 2^-48, is
// dropped as in operator*)
EXPD_HD dd dd_dot2(dd a, dd b, float sg, dd c, dd d) {
    const float p1 = a.hi * b.hi;
    const float e1 = fmaf(a.hi, b.hi, -p1);
    const float p2 = sg * (c.hi * d.hi);
    const float e2 = fmaf(sg * c.hi, d.hi, -p2);
    const dd s = dd_two_sum(p1, p2);
    float lo = s.lo + (e1 + e2);
    lo = fmaf(a.hi, b.lo, lo);
    lo = fmaf(a.lo, b.hi, lo);
    lo = fmaf(sg * c.hi, d.lo, lo);
    lo = fmaf(sg * c.lo, d.hi, lo);
    return dd_fast_two_sum(s.hi, lo);
}
EXPD_HD dd2 cmul(dd2 a, dd2 b) { return c2(dd_dot2(a.x, b.x, -1.0f, a.y, b.y), dd_dot2(a.x, b.y, 1.0f, a.y, b.x)); }
EXPD_HD dd2 cconj(dd2 a) { return c2(a.x, -a.y); }
EXPD_HD dd2 cscale(dd2 a, dd s) { return c2(a.x * s, a.y * s); }
EXPD_HD dd2 cmulc(dd2 a, dd2 b) { return c2(dd_dot2(a.x, b.x, 1.0f, a.y, b.y), dd_dot2(a.y, b.x, -1.0f, a.x, b.y)); }
EXPD_HD dd2 cmuli(dd2 a) { return c2(-a.y, a.x); }

// conversions between the complex storage types
EXPD_HD dd2 to_dd2(double2 v) { return c2(dd(v.x), dd(v.y)); }
EXPD_HD dd2 to_dd2(float2 v) { return c2(dd(v.x), dd(v.y)); }
EXPD_HD dd2 to_dd2(dd2 v) { return v; }
EXPD_HD double2 dd2_to_c64(dd2 v) { return make_double2((double)v.x, (double)v.y); }
EXPD_HD float2 dd2_to_c32(dd2 v) { return make_float2((float)v.x, (float)v.y); }

// cvt2<T2>(v): complex conversion between double2, float2 and dd2 storage
template <typename T2>
EXPD_HD T2 cvt2(double2 v);
template <typename T2>
EXPD_HD T2 cvt2(float2 v);
template <typename T2>
EXPD_HD T2 cvt2(dd2 v);
template <>
EXPD_HD double2 cvt2<double2>(double2 v) { return v; }
template <>
EXPD_HD float2 cvt2<float2>(double2 v) { return make_float2(f32_rn_from_f64(v.x), f32_rn_from_f64(v.y)); }
template <>
EXPD_HD dd2 cvt2<dd2>(double2 v) { return to_dd2(v); }
template <>
EXPD_HD double2 cvt2<double2>(float2 v) { return make_double2((double)v.x, (double)v.y); }
template <>
EXPD_HD float2 cvt2<float2>(float2 v) { return v; }
template <>
EXPD_HD dd2 cvt2<dd2>(float2 v) { return to_dd2(v); }
template <>
EXPD_HD double2 cvt2<double2>(dd2 v) { return dd2_to_c64(v); }
template <>
EXPD_HD float2 cvt2<float2>(dd2 v) { return dd2_to_c32(v); }
template <>
EXPD_HD dd2 cvt2<dd2>(dd2 v) { return v; }

// coefficient helpers (see common.cuh) for double-float storage
EXPD_HD dd2 acc_add(dd2 a, dd c) { return c2(a.x + c, a.y); }
EXPD_HD dd2 acc_add(dd2 a, dd2 c) { return cadd(a, c); }
EXPD_HD dd2 sub_cx(dd2 r, dd c, dd2 x) { return c2(r.x - c * x.x, r.y - c * x.y); }
EXPD_HD dd2 sub_cx(dd2 r, dd2 c, dd2 x) { return csub(r, cmul(c, x)); }
template <>
EXPD_HD dd coef_zero<dd>() { return dd(0.0f, 0.0f); }
template <>
EXPD_HD dd2 coef_zero<dd2>() { return c2(dd(0.0f, 0.0f), dd(0.0f, 0.0f)); }
