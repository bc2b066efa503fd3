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

#include "common.cuh"

struct dd {
    float hi, lo;
    dd() = default;
    EXPD_HD explicit dd(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
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
EXPD_HD dd2 cmul(dd2 a, dd2 b) { return c2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
EXPD_HD dd2 cconj(dd2 a) { return c2(a.x, -a.y); }
EXPD_HD dd2 cscale(dd2 a, dd s) { return c2(a.x * s, a.y * s); }
EXPD_HD dd2 cmulc(dd2 a, dd2 b) { return c2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }
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
EXPD_HD float2 cvt2<float2>(double2 v) { return make_float2((float)v.x, (float)v.y); }
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
