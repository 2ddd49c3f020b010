// Integrated Green's function table in double-double precision.
//
// Reading of the paper's rest-frame Poisson solve (arXiv:2208.02382, Model
// Assumptions; ABLASTR Poisson solver): the cell-integrated Green's function
// of Qiang et al., PRSTAB 9, 044204 (2006),
//   G(a,b,c) = 1/(4 pi eps0) * box integral of 1/r over the cell centred at
//              (a hx, b hy, c hz),
// as the alternating 8-corner sum of the antiderivative
//   F = -z^2/2 atan(xy/(zr)) - y^2/2 atan(xz/(yr)) - x^2/2 atan(yz/(xr))
//       + yz ln(x+r) + xz ln(y+r) + xy ln(z+r).
// The corner sum cancels up to ~9 digits at far cells, so F and the sum run in
// double-double and G is rounded to double once.  Corner coordinates are
// (i - 1/2) h, never zero; ln(u + r) for u < 0 is ln((r^2 - u^2)/(r - u)).
//
// Far cells (corner radius |h|/2 at most 1/8 of the distance R) take the
// cell-integrated Taylor series instead (igf_far.cuh, written by
// gen_igf_far.py): G = V/(4 pi eps0 R) (1 + sum_{n=1..L} Q_n(U,V,W)/R^2n), U =
// (x/R)^2 etc., with Q_n's coefficients formed once per block from h; the
// truncation error is below 5.6e-17 of G and the series terms are at most
// 1/60 of the leading V/R, which is formed in double-double.  Only the near
// region (a box of about 8|h|/h_d cells per dimension around the origin)
// needs corner values.
//
// Two kernels: one thread per corner of the near region evaluates F once;
// one thread per octant cell (n+1)^3 forms the corner sum (near) or the series
// (far).
#include <algorithm>

#include "common.cuh"
#include "dd.cuh"
#include "igf_far.cuh"

namespace bt {

// 1/(4 pi eps0) with eps0 = 8.8541878128e-12 F/m (CODATA 2018), as hi + lo.
constexpr double KE_HI = 8987551792.261171;
constexpr double KE_LO = 8.180103421400543e-07;

__device__ dd ln_u_plus_r(dd u, dd r, dd rest2) {
    if (u.hi >= 0.0) return dd_log(dd_add(u, r));
    return dd_log(dd_div(rest2, dd_sub(r, u)));
}

// The antiderivative F at corner (x, y, z), split over three lanes: lane j
// (0, 1, 2) forms the j-th atan term (z^2, y^2, x^2 times atan(xy/(zr)),
// atan(xz/(yr)), atan(yz/(xr)), halved) and the j-th log term (yz ln(x+r),
// xz ln(y+r), xy ln(z+r)); all three lanes take the same path.  The caller
// sums the six terms in a fixed order.
__device__ void igf_terms(dd x, dd y, dd z, int j, dd &at, dd &lg) {
    const dd x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    const dd r = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    // lane j's operands (selects, no divergence)
    const dd an = j == 0 ? dd_mul(x, y) : (j == 1 ? dd_mul(x, z) : dd_mul(y, z));
    const dd ad = j == 0 ? dd_mul(z, r) : (j == 1 ? dd_mul(y, r) : dd_mul(x, r));
    const dd ap = j == 0 ? z2 : (j == 1 ? y2 : x2);
    at = dd_scale(dd_mul(ap, dd_atan_ratio(an, ad)), 0.5);
    const dd lu = j == 0 ? x : (j == 1 ? y : z);
    const dd lr = j == 0 ? dd_add(y2, z2) : (j == 1 ? dd_add(x2, z2) : dd_add(x2, y2));
    const dd lp = j == 0 ? dd_mul(y, z) : (j == 1 ? dd_mul(x, z) : dd_mul(x, y));
    lg = dd_mul(lp, ln_u_plus_r(lu, r, lr));
}

// A cell at distance R (squared R2) is far when R2 >= 16 (hx^2 + hy^2 + hz^2),
// i.e. |h|/2 <= R/8.
__device__ __forceinline__ bool igf_is_far(double R2, double hsum2) { return R2 >= 16.0 * hsum2; }

// The far test of cell (a, b, c), rounded step by step (no contraction) so
// that the corner kernel (which skips corners no near cell reads) and the sum
// kernel (which reads the corners of near cells) always agree.
__device__ __forceinline__ bool igf_cell_is_far(int a, int b, int c, double hx, double hy, double hz,
                                                double hsum2) {
    const double xa = __dmul_rn((double)a, hx), yb = __dmul_rn((double)b, hy),
                 zc = __dmul_rn((double)c, hz);
    const double R2 = __dadd_rn(__dadd_rn(__dmul_rn(xa, xa), __dmul_rn(yb, yb)), __dmul_rn(zc, zc));
    return igf_is_far(R2, hsum2);
}

// Near cells have index below 4|h|/h_d + 1 in dimension d (rounding slack).
__device__ __forceinline__ int igf_near_extent(int n, double hd, double hsum2) {
    const double e = 4.0 * sqrt(hsum2) / hd;
    return e >= (double)n ? n : min(n, (int)e + 1);
}

// With a tracking state `gate`, the cell size is the state's box h and the
// kernel does nothing unless the Green's function is stale.  Four lanes per
// corner (three used), eight corners per warp.
__global__ void k_igf_corner(int n, double hx, double hy, double hz, double2 *__restrict__ fc,
                             const TrackState *gate) {
    if (gate) {
        if (!gate->green_stale || gate->halt) return;
        hx = gate->box.h[0];
        hy = gate->box.h[1];
        hz = gate->box.h[2];
    }
    const int m = n + 2;
    const double hsum2 = hx * hx + hy * hy + hz * hz;
    // corners 0..A+1 per dimension serve the near cells 0..A
    const int ci = igf_near_extent(n, hx, hsum2) + 2, cj = igf_near_extent(n, hy, hsum2) + 2,
              ck = igf_near_extent(n, hz, hsum2) + 2;
    const long long total = (long long)ci * cj * ck;
    const int lane = threadIdx.x & 3, j = lane < 3 ? lane : 2;
    const long long stride = (long long)gridDim.x * blockDim.x / 4;
    // every lane of a group runs the same iterations (the shuffles need all 32)
    for (long long base = (blockIdx.x * (long long)blockDim.x) / 4; base < total; base += stride) {
        const long long idx = base + threadIdx.x / 4;
        const bool live = idx < total;
        const long long id = live ? idx : 0;
        const int i = (int)(id % ci);
        const int jj = (int)((id / ci) % cj);
        const int k = (int)(id / ((long long)ci * cj));
        // corner (i, jj, k) serves cells i-1..i, jj-1..jj, k-1..k; when the one
        // nearest the origin is far, all are, and no near cell reads the corner
        const bool need = live && !igf_cell_is_far(max(i - 1, 0), max(jj - 1, 0), max(k - 1, 0),
                                                   hx, hy, hz, hsum2);
        dd at = {0.0, 0.0}, lg = {0.0, 0.0};
        if (need)
            igf_terms(two_prod(i - 0.5, hx), two_prod(jj - 0.5, hy), two_prod(k - 0.5, hz), j, at, lg);
        // lane 0 of the group gathers the other lanes' terms
        const int g0 = threadIdx.x & ~3;
        const double a1h = __shfl_sync(0xffffffffu, at.hi, g0 + 1), a1l = __shfl_sync(0xffffffffu, at.lo, g0 + 1);
        const double a2h = __shfl_sync(0xffffffffu, at.hi, g0 + 2), a2l = __shfl_sync(0xffffffffu, at.lo, g0 + 2);
        const double l1h = __shfl_sync(0xffffffffu, lg.hi, g0 + 1), l1l = __shfl_sync(0xffffffffu, lg.lo, g0 + 1);
        const double l2h = __shfl_sync(0xffffffffu, lg.hi, g0 + 2), l2l = __shfl_sync(0xffffffffu, lg.lo, g0 + 2);
        if (lane == 0 && need) {
            // F = -z^2/2 atan(..) - y^2/2 atan(..) - x^2/2 atan(..) + yz ln + xz ln + xy ln
            dd f = dd_neg(at);
            f = dd_sub(f, dd{a1h, a1l});
            f = dd_sub(f, dd{a2h, a2l});
            f = dd_add(f, lg);
            f = dd_add(f, dd{l1h, l1l});
            f = dd_add(f, dd{l2h, l2l});
            fc[((long long)k * m + jj) * m + i] = make_double2(f.hi, f.lo);
        }
    }
}

constexpr int IGF_FAR_NC = 164;  // sum over n = 1..8 of (n+1)(n+2)/2 monomials

// Coefficients of Q_n (n = 1..8) over U^i V^j W^k for half-sides a = h/2:
// sum over (p,q,t) of a_x^2p a_y^2q a_z^2t times the tabulated coefficient.
// Six one-warp blocks per build (the work of one SM's FP64 pipe spread over
// six); the sum kernel's blocks read the result.
__global__ void k_igf_coef(double hx, double hy, double hz, const TrackState *gate, double *c) {
    if (gate) {
        if (!gate->green_stale || gate->halt) return;
        hx = gate->box.h[0];
        hy = gate->box.h[1];
        hz = gate->box.h[2];
    }
    const double ax2 = 0.25 * hx * hx, ay2 = 0.25 * hy * hy, az2 = 0.25 * hz * hz;
    // powers a^2p, p <= 8, per dimension
    double P[9], Q[9], T[9];
    P[0] = Q[0] = T[0] = 1.0;
    for (int e = 1; e <= 8; ++e) {
        P[e] = P[e - 1] * ax2;
        Q[e] = Q[e - 1] * ay2;
        T[e] = T[e - 1] * az2;
    }
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < IGF_FAR_NC; k += gridDim.x * blockDim.x) {
        int n = 1, base = 0;
        while (k >= base + (n + 1) * (n + 2) / 2) {
            base += (n + 1) * (n + 2) / 2;
            ++n;
        }
        const int nt = (n + 1) * (n + 2) / 2, mono = k - base;
        double acc = 0.0;
        int ti = 0;
        for (int p = n; p >= 0; --p)
            for (int q = n - p; q >= 0; --q, ++ti)
                acc = fma(P[p] * Q[q] * T[n - p - q],
                          __ldg(&IGF_FAR_P[IGF_FAR_OFF[n - 1] + ti * nt + mono]), acc);
        c[k] = acc;
    }
}

// sum_{n <= L} Q_n(U, V, W) iR2^n = sum over 1 <= i+j+k <= L of
// c_ijk a^i b^j w^k with a = U iR2, b = V iR2, w = W iR2, by nested Horner
// schemes in w, b, a (one FMA per coefficient plus one per (i, j) and per i:
// 164 + 44 at L = 8, against two products and an FMA per monomial).  c holds
// order n's coefficients from offset sum_{m < n} (m+1)(m+2)/2, the monomial
// U^i V^j W^(n-i-j) at (n-i)(n-i+1)/2 + (n-i-j) within its order.
template <int L>
__device__ __forceinline__ double igf_far_series(double a, double b, double w, const double *c) {
    double sa = 0.0;
#pragma unroll
    for (int i = L; i >= 0; --i) {
        double sb = 0.0;
#pragma unroll
        for (int j = L - i; j >= 0; --j) {
            double sw = 0.0;
#pragma unroll
            for (int k = L - i - j; k >= 0; --k) {
                const int n = i + j + k;
                const int base = n * (n + 1) * (n + 2) / 6 - 1;   // sum_{m=1}^{n-1} (m+1)(m+2)/2
                const double cv = n == 0 ? 0.0 : c[base + (n - i) * (n - i + 1) / 2 + (n - i - j)];
                sw = fma(sw, w, cv);
            }
            sb = fma(sb, b, sw);
        }
        sa = fma(sa, a, sb);
    }
    return sa;
}

// G of a far cell at (x, y, z) = (a hx, b hy, c hz), with the coefficients c
// and q = V/(4 pi eps0) in double-double.  The series stops at the order L
// whose remainder rho^(2L+2) is small (rho^2 = |h|^2/(4 R^2)): L = 8 for
// rho <= 1/8 (5.6e-17), 6 for rho <= 1/16, 5 for rho <= 1/32, 4 for
// rho <= 1/64, 3 for rho <= 1/256 (each below 1.4e-17).
// 1/R comes from rsqrt and one Newton step with a double-double residual.
__device__ double igf_far_cell(int a, int b, int cc, double hx, double hy, double hz,
                               double hsum2, const double *c, dd q) {
    const dd x = two_prod((double)a, hx), y = two_prod((double)b, hy), z = two_prod((double)cc, hz);
    const dd R2 = dd_add(dd_add(dd_mul(x, x), dd_mul(y, y)), dd_mul(z, z));
    // 1/R^2 for the corrections from the same rsqrt as 1/R below (a few ulps:
    // the corrections are at most 1/60 of G)
    const double y0 = rsqrt(R2.hi);
    const double iR2 = y0 * y0;
    const double rho2 = 0.25 * hsum2 * iR2;
    const double i4 = iR2 * iR2;
    const double sa = x.hi * x.hi * i4, sb = y.hi * y.hi * i4, sw = z.hi * z.hi * i4;
    // series order from rho^2 > 0, compared as bit patterns (integer pipes)
    const long long rb = __double_as_longlong(rho2);
    double corr;
    if (rb > 0x3F70000000000000ll) corr = igf_far_series<8>(sa, sb, sw, c);        // 2^-8
    else if (rb > 0x3F50000000000000ll) corr = igf_far_series<6>(sa, sb, sw, c);   // 2^-10
    else if (rb > 0x3F30000000000000ll) corr = igf_far_series<5>(sa, sb, sw, c);   // 2^-12
    else if (rb > 0x3EF0000000000000ll) corr = igf_far_series<4>(sa, sb, sw, c);   // 2^-16
    else corr = igf_far_series<3>(sa, sb, sw, c);
    // 1/R: y0 = rsqrt(R2), y1 = y0 + y0 (1 - R2 y0^2)/2 with the residual in dd
    const dd t = dd_mul(R2, two_prod(y0, y0));
    const double e = __dsub_rn(1.0, t.hi) - t.lo;
    const dd iR = fast_two_sum(y0, 0.5 * y0 * e);
    const dd lead = dd_mul(q, iR);
    return lead.hi + fma(lead.hi, corr, lead.lo);
}

__global__ void k_igf_sum(int n, double hx, double hy, double hz, const double2 *__restrict__ fc,
                          const double *__restrict__ coef, double *__restrict__ g,
                          const TrackState *gate) {
    if (gate) {
        if (!gate->green_stale || gate->halt) return;
        hx = gate->box.h[0];
        hy = gate->box.h[1];
        hz = gate->box.h[2];
    }
    __shared__ double sc[IGF_FAR_NC];
    for (int k = threadIdx.x; k < IGF_FAR_NC; k += blockDim.x) sc[k] = coef[k];
    __syncthreads();
    const int m = n + 2, q = n + 1;
    const long long total = (long long)q * q * q;
    const dd ke = {KE_HI, KE_LO};
    const double hsum2 = hx * hx + hy * hy + hz * hz;
    const dd qv = dd_mul(ke, dd_mul_d(two_prod(hx, hy), hz));
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int a = (int)(idx % q);
        int b = (int)((idx / q) % q);
        int c = (int)(idx / ((long long)q * q));
        if (igf_cell_is_far(a, b, c, hx, hy, hz, hsum2)) {
            g[idx] = igf_far_cell(a, b, c, hx, hy, hz, hsum2, sc, qv);
            continue;
        }
        dd s = dd_make(0.0);
        for (int dk = 0; dk < 2; ++dk)
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    double2 v = fc[((long long)(c + dk) * m + (b + dj)) * m + (a + di)];
                    dd f = {v.x, v.y};
                    // +1 when the number of lower corners is even
                    s = ((di + dj + dk) & 1) ? dd_add(s, f) : dd_sub(s, f);
                }
        s = dd_mul(s, ke);
        g[idx] = s.hi;
    }
}

cudaError_t launch_igf_table(int n, const double h[3], double *fcorner, double *gtable,
                             cudaStream_t s, const TrackState *gate) {
    const int q = n + 1, m = n + 2;
    const long long ts = (long long)q * q * q;
    // series coefficients after the corner table (igf_scratch_doubles)
    double *coef = fcorner + 2LL * m * m * m;
    // the near region's size is known on the device only (h may come from the
    // state): one-warp blocks, a few per SM, grid-stride.  A corner is a long
    // chain of FP64 double-double work; three lanes share it and one-warp
    // blocks spread the ~1e3 corners of a typical near region over all SMs
    // instead of a few.
    const int bc = 148 * 4;
    const int bs = (int)std::min<long long>((ts + 255) / 256, 148 * 16);
    const double h0 = h ? h[0] : 0.0, h1 = h ? h[1] : 0.0, h2 = h ? h[2] : 0.0;
    BT_LAUNCH(K_IGF_CORNER, s, k_igf_coef<<<6, 32, 0, s>>>(h0, h1, h2, gate, coef));
    BT_LAUNCH(K_IGF_CORNER, s, k_igf_corner<<<bc, 32, 0, s>>>(n, h0, h1, h2, (double2 *)fcorner, gate));
    BT_LAUNCH(K_IGF_SUM, s, k_igf_sum<<<bs, 256, 0, s>>>(n, h0, h1, h2, (const double2 *)fcorner,
                                                         coef, gtable, gate));
    return cudaGetLastError();
}

// After a gated rebuild: the spectrum now belongs to the box's h.
__global__ void k_green_commit(TrackState *st) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && st->green_stale && !st->halt) {
        for (int d = 0; d < 3; ++d) st->green_h[d] = st->box.h[d];
        st->green_stale = 0;
    }
}

cudaError_t launch_green_commit(TrackState *st, cudaStream_t s) {
    BT_LAUNCH(K_BOX, s, k_green_commit<<<1, 32, 0, s>>>(st));
    return cudaGetLastError();
}

}  // namespace bt
