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

// (a * b) >> 52 for a, b <= 2^52 (the top bits of the 104-bit product).
__device__ __forceinline__ unsigned long long mulshr52(unsigned long long a, unsigned long long b) {
    unsigned long long lo = a * b, hi = __umul64hi(a, b);
    return (hi << 12) | (lo >> 52);
}

// a + (b - a) * F / 2^52 for |a|, |b| < 2^61 and 0 <= F <= 2^52 (truncated
// to 4 units of the last place).
__device__ __forceinline__ long long lerp52(long long a, long long b, unsigned long long F) {
    return a + (__mul64hi(b - a, (long long)(F << 10)) << 2);
}

// v * 2^-e rounded to nearest-even double, with integer operations only.
// Results below the normal range flush to zero.
__device__ __forceinline__ double i64_scaled_to_double(long long v, int e) {
    if (v == 0) return 0.0;
    const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
    const int msb = 63 - __clzll((long long)a);
    long long ex = (long long)msb - e + 1023;
    unsigned long long mant;
    if (msb <= 52) {
        mant = a << (52 - msb);
    } else {
        const int sh = msb - 52;
        mant = a >> sh;
        const unsigned long long rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) {
            mant += 1;
            if (mant >> 53) {
                mant >>= 1;
                ex += 1;
            }
        }
    }
    if (ex <= 0) return __longlong_as_double((long long)sign);
    if (ex >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
    return __longlong_as_double((long long)(sign | ((unsigned long long)ex << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
}

}  // namespace bt
