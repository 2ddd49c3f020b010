// Fixed-point helpers of the particle-grid kernels.  On this GPU the integer
// pipes issue tens of times more operations per clock than the FP64 pipe, so
// the CIC weights, the field interpolation and the charge accumulation run in
// 64-bit fixed point, exactly or to better than FP64 resolution.
#pragma once

namespace bt {

// u to unsigned fixed point with 52 fractional bits by exponent/mantissa
// arithmetic (integer operations only; on this GPU even an FP64 comparison
// takes an FP64-pipe slot): exact for 1 <= u < 2^11, truncated below 1;
// negative u gives 0, u >= 2^11 (and Inf/NaN) saturates to 2^63 - 1.
__device__ __forceinline__ unsigned long long to_fixed52(double u) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    if (b >> 63) return 0ull;
    const int e = (int)(b >> 52) - 1023;
    if (e < -60) return 0ull;
    if (e > 10) return 0x7FFFFFFFFFFFFFFFull;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return e >= 0 ? (mant << e) : (mant >> (-e));
}

// Bits of |u| (orders like the magnitude for non-NaN values).
__device__ __forceinline__ unsigned long long abs_bits(double u) {
    return (unsigned long long)__double_as_longlong(u) & 0x7FFFFFFFFFFFFFFFull;
}

// Inf or NaN, tested on the exponent bits.
__device__ __forceinline__ bool nonfinite_bits(double v) {
    return ((unsigned long long)__double_as_longlong(v) & 0x7FF0000000000000ull) ==
           0x7FF0000000000000ull;
}

// Products of 32-bit operands as 64-bit values, each one wide multiply (the
// compiler otherwise widens a signed-by-unsigned product of limbs to a full
// 64 x 64-bit multiply).
__device__ __forceinline__ long long mul_wide_s(int a, int b) {
    long long d;
    asm("mul.wide.s32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ unsigned long long mul_wide_u(unsigned a, unsigned b) {
    unsigned long long d;
    asm("mul.wide.u32 %0, %1, %2;" : "=l"(d) : "r"(a), "r"(b));
    return d;
}

// A 52-bit fraction split into two 26-bit limbs, so that products run on
// 32x32->64-bit multiplies: F = hi * 2^26 + lo.
struct Frac {
    unsigned hi, lo;
};
__device__ __forceinline__ Frac split26(unsigned long long F) {
    return Frac{(unsigned)(F >> 26), (unsigned)(F & 0x3FFFFFFull)};
}

// (a * b) >> 52 for fractions a, b <= 2^52, from three 26x26-bit partial
// products (the dropped low product and the truncated middle term leave an
// error below 2 units of 2^-52).
__device__ __forceinline__ unsigned long long mulshr52(Frac a, Frac b) {
    const unsigned long long hh = mul_wide_u(a.hi, b.hi);
    const unsigned long long mid = mul_wide_u(a.hi, b.lo) + mul_wide_u(a.lo, b.hi);
    return hh + (mid >> 26);
}

// a + (b - a) * F / 2^52 for |a|, |b| < 2^50 (so |b - a| < 2^51) and a
// fraction F <= 2^52: d = b - a split as dh * 2^26 + dl (dh signed, dl in
// [0, 2^26)), d * F / 2^52 = dh*Fh + (dh*Fl + dl*Fh) / 2^26 (+ dl*Fl/2^52,
// below one unit, dropped).  Error below 2 units of the last place.
__device__ __forceinline__ long long lerp52(long long a, long long b, Frac F) {
    const long long d = b - a;
    const int dh = (int)(d >> 26);
    const unsigned dl = (unsigned)(d & 0x3FFFFFFll);
    const long long hh = mul_wide_s(dh, (int)F.hi);
    const long long mid = mul_wide_s(dh, (int)F.lo) + (long long)mul_wide_u(dl, F.hi);
    return a + hh + (mid >> 26);
}

// v * 2^-e as a double for |v| < 2^53 (exact: no rounding needed), with
// integer operations only.  Results below the normal range flush to zero.
__device__ __forceinline__ double i64_scaled_to_double(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int msb = 63 - __clzll((long long)a);
    const long long ex = (long long)msb - e + 1023;
    if (ex <= 0) return __longlong_as_double((long long)sign);
    const unsigned long long mant = a << (52 - msb);
    return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace bt
