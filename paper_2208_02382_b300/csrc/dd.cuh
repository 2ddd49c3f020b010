// Double-double ("dd") arithmetic for the integrated Green's function.
//
// A dd value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits.
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum
// and the FMA form of TwoProduct (Dekker 1971); add/mul/div/sqrt follow the
// double-double algorithms of Hida, Li and Bailey (QD library, 2001).
// Elementary functions are built here from their series and one Newton step
// started from the FP64 result of the CUDA math library:
//   exp : argument reduction by k ln2 and 2^-10, Taylor series of expm1,
//         ten squarings of (1 + s)
//   log : y1 = y0 + a exp(-y0) - 1 with y0 = log(a.hi)
//   atan: z1 = z0 + cos z0 (a cos z0 - sin z0) with z0 = atan(a.hi), sin and
//         cos by Taylor series at z0/8 and three double-angle steps;
//         |a| > 1 uses atan(a) = pi/2 - atan(1/a)
// Constants ln 2 and pi/2 are given as hi + lo pairs (60-digit values split
// to two doubles).
#pragma once

namespace bt {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_make(double a) { return {a, 0.0}; }

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b|
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_add_d(dd a, double b) {
    dd s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_scale(dd a, double pow2) { return {a.hi * pow2, a.lo * pow2}; }

__device__ __forceinline__ dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

__device__ __forceinline__ dd dd_div_d(dd a, double b) {
    double q1 = a.hi / b;
    dd p = two_prod(q1, b);
    dd r = dd_sub(a, p);
    double q2 = r.hi / b;
    r = dd_sub(r, two_prod(q2, b));
    double q3 = r.hi / b;
    dd q = fast_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

__device__ __forceinline__ dd dd_sqrt(dd a) {  // a > 0
    double x = sqrt(a.hi);
    dd r = dd_sub(a, two_prod(x, x));
    double c = r.hi / (2.0 * x);
    return fast_two_sum(x, c);
}

constexpr double DD_LN2_HI = 0.6931471805599453;
constexpr double DD_LN2_LO = 2.3190468138462996e-17;
constexpr double DD_PI2_HI = 1.5707963267948966;
constexpr double DD_PI2_LO = 6.123233995736766e-17;

// exp(a), |a| < 700.
__device__ __noinline__ dd dd_exp(dd a) {
    double k = rint(a.hi / DD_LN2_HI);
    dd ln2 = {DD_LN2_HI, DD_LN2_LO};
    dd r = dd_sub(a, dd_mul_d(ln2, k));
    r = dd_scale(r, 1.0 / 1024.0);  // |r| <= 3.4e-4
    // expm1(r) = sum_{j>=1} r^j / j!, nine terms (next term < 1e-37)
    dd term = r;
    dd s = r;
    for (int j = 2; j <= 9; ++j) {
        term = dd_div_d(dd_mul(term, r), (double)j);
        s = dd_add(s, term);
    }
    // (1 + s)^2 - 1 = s (2 + s), ten times
    for (int j = 0; j < 10; ++j) s = dd_mul(s, dd_add_d(s, 2.0));
    dd e = dd_add_d(s, 1.0);
    double p = ldexp(1.0, (int)k);
    return dd_scale(e, p);
}

// log(a), a > 0.
__device__ __noinline__ dd dd_log(dd a) {
    double y0 = log(a.hi);
    dd e = dd_exp(dd_make(-y0));
    dd t = dd_add_d(dd_mul(a, e), -1.0);
    return dd_add_d(t, y0);
}

// sin and cos of a double z with |z| <= pi/4.
__device__ __noinline__ void dd_sincos_small(double z, dd *s_out, dd *c_out) {
    dd r = dd_make(z * 0.125);  // exact
    dd r2 = dd_mul(r, r);
    // sin r = r - r^3/3! + ..., cos r = 1 - r^2/2! + ..., |r| <= 0.1, ten terms each
    dd ts = r, s = r;
    dd tc = dd_make(1.0), c = dd_make(1.0);
    for (int j = 1; j <= 10; ++j) {
        ts = dd_neg(dd_div_d(dd_mul(ts, r2), (double)((2 * j) * (2 * j + 1))));
        s = dd_add(s, ts);
        tc = dd_neg(dd_div_d(dd_mul(tc, r2), (double)((2 * j - 1) * (2 * j))));
        c = dd_add(c, tc);
    }
    for (int j = 0; j < 3; ++j) {  // double angle: sin 2a = 2 s c, cos 2a = (c - s)(c + s)
        dd s2 = dd_scale(dd_mul(s, c), 2.0);
        dd c2 = dd_mul(dd_sub(c, s), dd_add(c, s));
        s = s2;
        c = c2;
    }
    *s_out = s;
    *c_out = c;
}

// atan(a) for 0 <= a <= 1.
__device__ __noinline__ dd dd_atan_unit(dd a) {
    double z0 = atan(a.hi);
    dd s, c;
    dd_sincos_small(z0, &s, &c);
    dd d = dd_sub(dd_mul(a, c), s);
    return dd_add(dd_make(z0), dd_mul(c, d));
}

__device__ __forceinline__ dd dd_atan(dd a) {
    bool neg = a.hi < 0.0;
    if (neg) a = dd_neg(a);
    dd r;
    if (a.hi > 1.0) {
        dd inv = dd_div(dd_make(1.0), a);
        r = dd_sub(dd{DD_PI2_HI, DD_PI2_LO}, dd_atan_unit(inv));
    } else {
        r = dd_atan_unit(a);
    }
    return neg ? dd_neg(r) : r;
}

}  // namespace bt
