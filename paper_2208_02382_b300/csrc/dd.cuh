// Double-double ("dd") arithmetic for the integrated Green's function.
//
// A dd value is hi + lo with |lo| <= ulp(hi)/2, about 106 significant bits.
// Error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum
// and the FMA form of TwoProduct (Dekker 1971); add/mul/div/sqrt follow the
// double-double algorithms of Hida, Li and Bailey (QD library, 2001).
// Elementary functions are built here from tables and short series:
//   log : a = 2^e m, log m = log(1 + j/128) + 2 atanh((m - c)/(m + c))
//   atan: atan(n/d) = atan(j/64) + atan((n - c d)/(d + c n)) for n <= d;
//         n > d uses pi/2 - atan(d/n)
// with the tables of gen_dd_tables.py (50-digit values split to hi + lo).
// Accuracy targets ~1e-28: far beyond the ~1e-21 relative accuracy of the
// antiderivative that a 1e-12 Green's function needs after the worst 8-corner
// cancellation (~1e9).
// Constants ln 2 and pi/2 are given as hi + lo pairs (60-digit values split
// to two doubles).
#pragma once

#include "dd_tables.cuh"

namespace bt {

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_make(double a) { return {a, 0.0}; }

// The error-free transformations are written with round-to-nearest intrinsics,
// which the compiler never fuses into an FMA with a neighbouring operation
// (a contracted a*b + c would no longer match the separately rounded product
// that the error term describes).
__device__ __forceinline__ dd two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b|
    const double s = __dadd_rn(a, b);
    const double e = __dsub_rn(b, __dsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    const double e = fma(a, b, -p);
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

// a / b: three quotient digits from one IEEE reciprocal of b.hi, each
// remainder formed exactly in double-double, so the reciprocal's rounding only
// affects the next digit.
__device__ __forceinline__ dd dd_div(dd a, dd b) {
    const double rb = 1.0 / b.hi;
    double q1 = a.hi * rb;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi * rb;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi * rb;
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

__device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
    // a + b with one TwoSum (relative error ~2^-104 unless a and b nearly
    // cancel; used in Horner steps whose terms shrink fast)
    dd s = two_sum(a.hi, b.hi);
    s.lo += a.lo + b.lo;
    return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd invodd(int k, bool neg) {
    return neg ? dd{-DD_INVODD_HI[k], -DD_INVODD_LO[k]} : dd{DD_INVODD_HI[k], DD_INVODD_LO[k]};
}

// Table entry through the read-only data path (indices differ per thread).
__device__ __forceinline__ dd dd_tab(const double *hi, const double *lo, int j) {
    return dd{__ldg(hi + j), __ldg(lo + j)};
}

// log(a), a > 0: a = 2^e m with m in [1, 2); c = 1 + j/128 nearest to m;
// log m = log c + 2 atanh(s), s = (m - c)/(m + c), |s| <= 2e-3, the atanh
// series through s^11 (next term below 1e-31 relative).  a = 0 gives -Inf,
// a < 0 or NaN gives NaN, a = +Inf gives +Inf; the table index stays in
// range for every input.
static __device__ __noinline__ dd dd_log(dd a) {
    if (!(a.hi > 0.0)) return dd{a.hi == 0.0 ? -INFINITY : NAN, 0.0};
    if (isinf(a.hi)) return dd{INFINITY, 0.0};
    const int e = ilogb(a.hi);
    // 2^-e in two exact steps (one overflows for subnormal a)
    const double s1 = ldexp(1.0, -(e / 2)), s2 = ldexp(1.0, (e / 2) - e);
    const dd m = {a.hi * s1 * s2, a.lo * s1 * s2};
    const int j = min(max((int)((m.hi - 1.0) * 128.0 + 0.5), 0), 128);
    const double c = 1.0 + (double)j * (1.0 / 128.0);
    const dd s = dd_div(dd_add_d(m, -c), dd_add_d(m, c));
    const dd x = dd_mul(s, s);
    dd p = invodd(5, false);
#pragma unroll
    for (int k = 4; k >= 0; --k) p = dd_add_fast(dd_mul(p, x), invodd(k, false));
    const dd t = dd_scale(dd_mul(s, p), 2.0);
    const dd base = dd_add(dd_mul_d(dd{DD_LN2_HI, DD_LN2_LO}, (double)e),
                           dd_tab(DD_LOGTAB_HI, DD_LOGTAB_LO, j));
    return dd_add(base, t);
}

// atan(n/d) for 0 <= n <= d: c = j/64 nearest to n/d; atan(n/d) = atan c +
// atan u with u = (n - c d)/(d + c n) (one division), |u| <= 7.9e-3, the atan
// series through u^15 (next term below 1e-34 relative).
static __device__ __noinline__ dd dd_atan_ratio_unit(dd n, dd d) {
    const int j = min(max((int)(n.hi / d.hi * 64.0 + 0.5), 0), 64);  // NaN ratio: 0
    const double c = (double)j * (1.0 / 64.0);
    const dd u = dd_div(dd_sub(n, dd_mul_d(d, c)), dd_add(d, dd_mul_d(n, c)));
    const dd x = dd_mul(u, u);
    dd q = invodd(7, true);
#pragma unroll
    for (int k = 6; k >= 0; --k) q = dd_add_fast(dd_mul(q, x), invodd(k, (k & 1) != 0));
    return dd_add(dd_tab(DD_ATANTAB_HI, DD_ATANTAB_LO, j), dd_mul(u, q));
}

// atan(n/d) for any signs of n and d != 0 (the principal value of atan of
// the quotient): |n| > |d| uses atan(n/d) = pi/2 - atan(d/n).
__device__ __forceinline__ dd dd_atan_ratio(dd n, dd d) {
    const bool neg = (n.hi < 0.0) != (d.hi < 0.0);
    if (n.hi < 0.0) n = dd_neg(n);
    if (d.hi < 0.0) d = dd_neg(d);
    dd r;
    if (n.hi > d.hi) r = dd_sub(dd{DD_PI2_HI, DD_PI2_LO}, dd_atan_ratio_unit(d, n));
    else r = dd_atan_ratio_unit(n, d);
    return neg ? dd_neg(r) : r;
}

}  // namespace bt
