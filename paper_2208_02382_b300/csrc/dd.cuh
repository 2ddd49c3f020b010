// Double-double ("dd") arithmetic for the integrated Green's function.
//
// A dd value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits.
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum
// and the FMA form of TwoProduct (Dekker 1971); add/mul/div/sqrt follow the
// double-double algorithms of Hida, Li and Bailey (QD library, 2001).
// Elementary functions are built here from their series and one Newton step
// started from the FP64 result of the CUDA math library:
//   exp : argument reduction by k ln2 and 2^-8, Taylor polynomial of expm1
//         in Horner form, eight squarings of (1 + s)
//   log : y1 = y0 + a exp(-y0) - 1 with y0 = log(a.hi)
//   atan: z1 = z0 + cos z0 (a cos z0 - sin z0) with z0 = atan(a.hi), sin and
//         cos by Taylor polynomials at z0/4 and two double-angle steps;
//         |a| > 1 uses atan(a) = pi/2 - atan(1/a)
// Accuracy targets ~1e-28: far beyond the ~1e-21 relative accuracy of the
// antiderivative that a 1e-12 Green's function needs after the worst 8-corner
// cancellation (~1e9).
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

// 1/k! for k = 0..20 as double-double (the exact rationals rounded to hi,
// then the remainder rounded to lo).
__constant__ double DD_INVFACT_HI[21] = {
    1.0, 1.0, 0.5, 0.16666666666666666, 0.041666666666666664, 0.008333333333333333,
    0.001388888888888889, 0.0001984126984126984, 2.48015873015873e-05, 2.7557319223985893e-06,
    2.755731922398589e-07, 2.505210838544172e-08, 2.08767569878681e-09, 1.6059043836821613e-10,
    1.1470745597729725e-11, 7.647163731819816e-13, 4.779477332387385e-14,
    2.8114572543455206e-15, 1.5619206968586225e-16, 8.22063524662433e-18,
    4.110317623312165e-19};
__constant__ double DD_INVFACT_LO[21] = {
    0.0, 0.0, 0.0, 9.25185853854297e-18, 2.3129646346357427e-18, 1.1564823173178714e-19,
    -5.300543954373577e-20, 1.7209558293420705e-22, 2.1511947866775882e-23,
    -1.858393274046472e-22, 2.3767714622250297e-23, -1.448814070935912e-24,
    -1.20734505911326e-25, 1.2585294588752098e-26, 2.0655512752830745e-28,
    7.03872877733453e-30, 4.399205485834081e-31, 1.6508842730861433e-31,
    1.1910679660273754e-32, 2.2141894119604265e-34, 1.4412973378659527e-36};

// a + b with one TwoSum (relative error ~2^-104 unless a and b nearly cancel;
// used in Horner steps whose terms shrink fast).
__device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd invfact(int k, bool neg) {
    return neg ? dd{-DD_INVFACT_HI[k], -DD_INVFACT_LO[k]} : dd{DD_INVFACT_HI[k], DD_INVFACT_LO[k]};
}

// exp(a), |a| < 700: a = k ln2 + 2^8 r, |r| <= 1.4e-3; expm1(r) by its Taylor
// polynomial through r^8/8! (next term below 4e-32) in Horner form with the
// double-double 1/j!; eight squarings (1 + s)^2 - 1 = s (2 + s).  Relative
// error about 1e-29.
__device__ __noinline__ dd dd_exp(dd a) {
    const double k = rint(a.hi * 1.4426950408889634);
    dd r = dd_sub(a, dd_mul_d(dd{DD_LN2_HI, DD_LN2_LO}, k));
    r = dd_scale(r, 1.0 / 256.0);
    dd p = invfact(8, false);
#pragma unroll
    for (int j = 7; j >= 1; --j) p = dd_add_fast(dd_mul(p, r), invfact(j, false));
    dd s = dd_mul(p, r);
#pragma unroll
    for (int j = 0; j < 8; ++j) s = dd_mul(s, dd_add_d(s, 2.0));
    return dd_scale(dd_add_d(s, 1.0), ldexp(1.0, (int)k));
}

// log(a), a > 0: one Newton step y1 = y0 + a exp(-y0) - 1 from y0 = log(a.hi).
__device__ __noinline__ dd dd_log(dd a) {
    const double y0 = log(a.hi);
    const dd e = dd_exp(dd_make(-y0));
    const dd t = dd_add_d(dd_mul(a, e), -1.0);
    return dd_add_d(t, y0);
}

// sin and cos of a double z, |z| <= pi/4: Taylor series at r = z/4 (|r| <=
// 0.197) through r^17/17! and r^16/16! (next terms below 1e-30) in Horner form
// in r^2, then two double-angle steps.
__device__ __noinline__ void dd_sincos_small(double z, dd *s_out, dd *c_out) {
    const dd r = dd_make(z * 0.25);  // exact
    const dd x = dd_mul(r, r);
    dd ps = invfact(17, false), pc = invfact(16, false);
#pragma unroll
    for (int k = 7; k >= 0; --k) {
        ps = dd_add_fast(dd_mul(ps, x), invfact(2 * k + 1, (k & 1) != 0));
        pc = dd_add_fast(dd_mul(pc, x), invfact(2 * k, (k & 1) != 0));
    }
    // ps was seeded with +1/17! (k = 8, even): sin r = r * ps(x), cos r = pc(x)
    dd s = dd_mul(ps, r), c = pc;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const dd s2 = dd_scale(dd_mul(s, c), 2.0);
        const dd c2 = dd_mul(dd_sub(c, s), dd_add(c, s));
        s = s2;
        c = c2;
    }
    *s_out = s;
    *c_out = c;
}

// atan(a) for 0 <= a <= 1: one Newton step z1 = z0 + cos z0 (a cos z0 - sin z0)
// from z0 = atan(a.hi).
__device__ __noinline__ dd dd_atan_unit(dd a) {
    const double z0 = atan(a.hi);
    dd s, c;
    dd_sincos_small(z0, &s, &c);
    const dd d = dd_sub(dd_mul(a, c), s);
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
