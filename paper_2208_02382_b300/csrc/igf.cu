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
// Two kernels: one thread per corner of the (n+2)^3 corner lattice evaluates
// F once; one thread per octant cell (n+1)^3 forms the corner sum.
#include "common.cuh"
#include "dd.cuh"

namespace bt {

// 1/(4 pi eps0) with eps0 = 8.8541878128e-12 F/m (CODATA 2018), as hi + lo.
constexpr double KE_HI = 8987551792.261171;
constexpr double KE_LO = 8.180103421400543e-07;

__device__ dd ln_u_plus_r(dd u, dd r, dd rest2) {
    if (u.hi >= 0.0) return dd_log(dd_add(u, r));
    return dd_log(dd_div(rest2, dd_sub(r, u)));
}

__device__ dd igf_antiderivative(dd x, dd y, dd z) {
    dd x2 = dd_mul(x, x), y2 = dd_mul(y, y), z2 = dd_mul(z, z);
    dd r = dd_sqrt(dd_add(dd_add(x2, y2), z2));
    dd a1 = dd_atan_ratio(dd_mul(x, y), dd_mul(z, r));
    dd a2 = dd_atan_ratio(dd_mul(x, z), dd_mul(y, r));
    dd a3 = dd_atan_ratio(dd_mul(y, z), dd_mul(x, r));
    dd lx = ln_u_plus_r(x, r, dd_add(y2, z2));
    dd ly = ln_u_plus_r(y, r, dd_add(x2, z2));
    dd lz = ln_u_plus_r(z, r, dd_add(x2, y2));
    dd f = dd_scale(dd_mul(z2, a1), -0.5);
    f = dd_sub(f, dd_scale(dd_mul(y2, a2), 0.5));
    f = dd_sub(f, dd_scale(dd_mul(x2, a3), 0.5));
    f = dd_add(f, dd_mul(dd_mul(y, z), lx));
    f = dd_add(f, dd_mul(dd_mul(x, z), ly));
    f = dd_add(f, dd_mul(dd_mul(x, y), lz));
    return f;
}

// With a tracking state `gate`, the cell size is the state's box h and the
// kernel does nothing unless the Green's function is stale.
__global__ void k_igf_corner(int n, double hx, double hy, double hz, double2 *__restrict__ fc,
                             const TrackState *gate) {
    if (gate) {
        if (!gate->green_stale || gate->halt) return;
        hx = gate->box.h[0];
        hy = gate->box.h[1];
        hz = gate->box.h[2];
    }
    const int m = n + 2;
    const long long total = (long long)m * m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx % m);
        int j = (int)((idx / m) % m);
        int k = (int)(idx / ((long long)m * m));
        dd x = two_prod(i - 0.5, hx);
        dd y = two_prod(j - 0.5, hy);
        dd z = two_prod(k - 0.5, hz);
        dd f = igf_antiderivative(x, y, z);
        fc[idx] = make_double2(f.hi, f.lo);
    }
}

__global__ void k_igf_sum(int n, const double2 *__restrict__ fc, double *__restrict__ g,
                          const TrackState *gate) {
    if (gate && (!gate->green_stale || gate->halt)) return;
    const int m = n + 2, q = n + 1;
    const long long total = (long long)q * q * q;
    const dd ke = {KE_HI, KE_LO};
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int a = (int)(idx % q);
        int b = (int)((idx / q) % q);
        int c = (int)(idx / ((long long)q * q));
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
    const int m = n + 2, q = n + 1;
    long long tc = (long long)m * m * m, ts = (long long)q * q * q;
    int bc = (int)((tc + 127) / 128), bs = (int)((ts + 255) / 256);
    const double h0 = h ? h[0] : 0.0, h1 = h ? h[1] : 0.0, h2 = h ? h[2] : 0.0;
    BT_LAUNCH(K_IGF_CORNER, s, k_igf_corner<<<bc, 128, 0, s>>>(n, h0, h1, h2, (double2 *)fcorner, gate));
    BT_LAUNCH(K_IGF_SUM, s, k_igf_sum<<<bs, 256, 0, s>>>(n, (const double2 *)fcorner, gtable, gate));
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
