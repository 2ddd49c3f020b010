// Per-particle arithmetic shared by the forward particle kernels and their
// adjoints, so that both see bit-identical cells, fractions and maps.
#pragma once

#include "common.cuh"
#include "fixed.cuh"

namespace bt {

template <int MK>
__device__ __forceinline__ void apply_map_k(const MapCoef &m, double &x, double &px, double &y,
                                            double &py, double &t, double pt) {
    if constexpr (MK == MAP_DRIFT) {
        x = fma(m.m01, px, x);
        y = fma(m.m23, py, y);
        t = fma(m.m45, pt, t);
    } else if constexpr (MK == MAP_QUAD) {
        double nx = m.m00 * x + m.m01 * px;
        double npx = m.m10 * x + m.m11 * px;
        double ny = m.m22 * y + m.m23 * py;
        double npy = m.m32 * y + m.m33 * py;
        t = fma(m.m45, pt, t);
        x = nx;
        px = npx;
        y = ny;
        py = npy;
    } else if constexpr (MK == MAP_BEND) {
        double nx = m.m00 * x + m.m01 * px + m.m05 * pt;
        double npx = m.m10 * x + m.m11 * px + m.m15 * pt;
        double nt = t + m.m40 * x + m.m41 * px + m.m45 * pt;
        y = fma(m.m23, py, y);
        x = nx;
        px = npx;
        t = nt;
    } else if constexpr (MK == MAP_GENERAL) {
        double nx = m.m00 * x + m.m01 * px + m.m05 * pt;
        double npx = m.m10 * x + m.m11 * px + m.m15 * pt;
        double ny = m.m22 * y + m.m23 * py;
        double npy = m.m32 * y + m.m33 * py;
        double nt = t + m.m40 * x + m.m41 * px + m.m45 * pt;
        x = nx;
        px = npx;
        y = ny;
        py = npy;
        t = nt;
    }
}

// Thin multipole kick of a SplitRec: P(x + i y) by Horner's rule in complex
// FP64, then px -= Re P, py += Im P.
__device__ __forceinline__ void thin_multipole_kick(const SplitRec &r, double x, double &px,
                                                    double y, double &py) {
    const int nc = (int)r.nc;
    double pr = 0.0, pi = 0.0;
    for (int j = nc - 1; j >= 0; --j) {  // P = P z + c_j
        const double nr = fma(pr, x, fma(-pi, y, r.cr[j]));
        pi = fma(pr, y, fma(pi, x, r.ci[j]));
        pr = nr;
    }
    px -= pr;
    py += pi;
}

__device__ __forceinline__ void apply_split(const SplitRec &r, double &x, double &px, double &y,
                                            double &py, double &t, double pt) {
    apply_map_k<MAP_GENERAL>(r.before, x, px, y, py, t, pt);
    thin_multipole_kick(r, x, px, y, py);
    apply_map_k<MAP_GENERAL>(r.after, x, px, y, py, t, pt);
}

// The SplitRec of table entry `row` (kind MAP_SPLIT).
__device__ __forceinline__ const SplitRec *split_rec(const MapCoef *row) {
    return reinterpret_cast<const SplitRec *>(row + (long long)row->aux);
}

// MAP_TABLE: the map (and its class in `kind`) comes from the per-call
// device table entry `row` (a copy of it in `m`); the class branch is
// uniform across the grid.
__device__ __forceinline__ void apply_map_table(const MapCoef &m, const MapCoef *row, double &x,
                                                double &px, double &y, double &py, double &t,
                                                double pt) {
    const int k = (int)m.kind;
    if (k == MAP_DRIFT) apply_map_k<MAP_DRIFT>(m, x, px, y, py, t, pt);
    else if (k == MAP_QUAD) apply_map_k<MAP_QUAD>(m, x, px, y, py, t, pt);
    else if (k == MAP_BEND) apply_map_k<MAP_BEND>(m, x, px, y, py, t, pt);
    else if (k == MAP_SPLIT) apply_split(*split_rec(row), x, px, y, py, t, pt);
    else apply_map_k<MAP_GENERAL>(m, x, px, y, py, t, pt);
}

// A node's field record (x, y, z and the pad word; records are 32-byte
// aligned) in one 32-byte read-only load: half the load instructions of a
// 16-byte and an 8-byte load, which the gathers' random node accesses are
// bound by.
__device__ __forceinline__ void ld_efix(const EFix *q, long long &x, long long &y, long long &z) {
    [[maybe_unused]] long long pad;
    asm("ld.global.nc.v4.b64 {%0, %1, %2, %3}, [%4];"
        : "=l"(x), "=l"(y), "=l"(z), "=l"(pad)
        : "l"(q));
}

// All six finite: the largest exponent field (from the 32-bit high words,
// combined with integer max so the test stays on the integer pipes) is below
// the all-ones exponent of Inf/NaN.
__device__ __forceinline__ bool finite6(double a, double b, double c, double d, double e, double f) {
    const unsigned m = 0x7FF00000u;
    const unsigned hm = max(max(max((unsigned)__double2hiint(a) & m, (unsigned)__double2hiint(b) & m),
                                max((unsigned)__double2hiint(c) & m, (unsigned)__double2hiint(d) & m)),
                            max((unsigned)__double2hiint(e) & m, (unsigned)__double2hiint(f) & m));
    return hm != m;
}

// A box far from the origin relative to its cell size needs the unfused u.
__host__ __device__ __forceinline__ bool box_far_offset(const Box &b) {
    for (int d = 0; d < 3; ++d)
        if (fabs(b.lo[d] * b.inv_h[d]) > 4096.0 || fabs(b.hi[d] * b.inv_h[d]) > 4096.0) return true;
    return false;
}

// Cell index and 52-bit fraction per dimension from u, with integer
// operations only.  u below -1e-9 or above n-1+1e-6 (beyond the rounding of
// u for a particle inside [lo, hi)) sets `outside`.
constexpr unsigned long long NEG_TOL_BITS = 0x3E112E0BE826D695ull;  // bits of 1e-9
__device__ __forceinline__ void cell_frac(double u, int nn, int &cell, unsigned long long &F,
                                          bool &outside) {
    const unsigned long long umax = (unsigned long long)(nn - 1) << 52;
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    unsigned long long U = to_fixed52(u);
    outside |= ((b >> 63) && abs_bits(u) > NEG_TOL_BITS) || U > umax + 4503599627ull;
    if (U > umax) U = umax;
    unsigned long long i = U >> 52;
    if (i > (unsigned long long)(nn - 2)) i = nn - 2;
    F = U - (i << 52);
    cell = (int)i;
}

// u = (X - lo)/h per dimension of a particle at (x, y, t) (rest frame:
// Z = -beta gamma t): one FMA with the box's constants, X * (1/h) - lo/h, or,
// for a box far from the origin relative to its cell size (EX), the
// subtraction first.
template <bool EX>
__device__ __forceinline__ void box_u(const Box &b, double nbg, double x, double y, double t,
                                      double &u0, double &u1, double &u2) {
    u0 = EX ? (x - b.lo[0]) * b.inv_h[0] : fma(x, b.inv_h[0], b.off[0]);
    u1 = EX ? (y - b.lo[1]) * b.inv_h[1] : fma(y, b.inv_h[1], b.off[1]);
    u2 = EX ? (__dmul_rn(nbg, t) - b.lo[2]) * b.inv_h[2] : fma(t, b.tz, b.off[2]);
}

// floor(a b / 2^51) for a, b <= 2^51, exact (full 64 x 64 -> 128-bit product;
// measured faster here than the same floor from 26-bit limb products).
__device__ __forceinline__ unsigned long long mulfloor51(unsigned long long a, unsigned long long b) {
    return (__umul64hi(a, b) << 13) | ((a * b) >> 51);
}

// CIC weights of a particle in its cell as unsigned fixed point with
// DEP_FRAC_BITS = 51 fractional bits, from the cell fractions F_d (52 bits;
// the lowest is dropped: u itself carries at most 46 fractional bits on grids
// of 128 nodes).  With X, Y, Z the fractions and 1 = 2^51: P = floor(X Y),
// the four x-y weights (1-X)(1-Y) = 1 - X - Y + P, X(1-Y) = X - P,
// (1-X)Y = Y - P, XY = P, then each times Z: q = floor(W Z) to the node at
// z+1 and W - q to the node at z.  Five exact floor products; every weight is
// non-negative (each is its exact value minus the dropped fractions of at most
// its own products, and an integer) and the eight sum to exactly 1, so the
// deposit conserves charge exactly.  w[(dz*2 + dy)*2 + dx] is node
// (c0 + dx, c1 + dy, c2 + dz).
__device__ __forceinline__ void cic_weights(unsigned long long F0, unsigned long long F1,
                                            unsigned long long F2, unsigned long long w[8]) {
    const unsigned long long one = 1ull << DEP_FRAC_BITS;
    const unsigned long long X = F0 >> 1, Y = F1 >> 1, Z = F2 >> 1;
    const unsigned long long P = mulfloor51(X, Y);
    const unsigned long long wxy[4] = {one - X - Y + P, X - P, Y - P, P};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const unsigned long long q = mulfloor51(wxy[k], Z);
        w[k] = wxy[k] - q;
        w[4 + k] = q;
    }
}

}  // namespace bt
