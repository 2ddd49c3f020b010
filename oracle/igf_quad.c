/*
 * Integrated Green's function (IGF) of the free-space Poisson equation,
 * evaluated in __float128.  Oracle: test infrastructure only (the product CUDA
 * path never links this file).
 *
 * Paper anchor: arXiv:2208.02382 §Model Assumptions (Poisson equation solved in
 * the bunch rest frame) and the reused ABLASTR Poisson solver.  The paper gives
 * no Green's function; the reading is the cell-integrated Green's function of
 * Qiang et al., PRSTAB 9, 044204 (2006):
 *
 *   G(a,b,c) = 1/(4 pi eps0) * integral over the box centred at
 *              (a hx, b hy, c hz) with sides (hx, hy, hz) of d^3r / |r|
 *
 * evaluated as the alternating 8-corner sum of an antiderivative F with
 * d^3F/dx dy dz = 1/r:
 *
 *   F = -z^2/2 atan(xy/(zr)) - y^2/2 atan(xz/(yr)) - x^2/2 atan(yz/(xr))
 *       + yz ln(x+r) + xz ln(y+r) + xy ln(z+r),     r = |(x,y,z)|
 *
 * Box corners sit at half-integer multiples of the cell size, so no corner
 * coordinate is ever zero.  For a negative coordinate, ln(x+r) is taken as
 * ln((y^2+z^2)/(r-x)) to avoid cancellation.  The 8-corner sum cancels up to
 * ~9 decimal digits at far cells, which is why the whole evaluation runs in
 * 113-bit precision and is rounded to double once at the end.
 */
#include <quadmath.h>
#include <stdlib.h>

typedef __float128 q128;

static const q128 EPS0_Q = 8.8541878128e-12Q; /* CODATA 2018, F/m */

static q128 ln_u_plus_r(q128 u, q128 r, q128 rest2)
{
    if (u >= 0) return logq(u + r);
    return logq(rest2 / (r - u));
}

static q128 igf_antiderivative(q128 x, q128 y, q128 z)
{
    q128 x2 = x * x, y2 = y * y, z2 = z * z;
    q128 r = sqrtq(x2 + y2 + z2);
    return -0.5Q * z2 * atanq(x * y / (z * r))
           - 0.5Q * y2 * atanq(x * z / (y * r))
           - 0.5Q * x2 * atanq(y * z / (x * r))
           + y * z * ln_u_plus_r(x, r, y2 + z2)
           + x * z * ln_u_plus_r(y, r, x2 + z2)
           + x * y * ln_u_plus_r(z, r, x2 + y2);
}

/* Box integral of 1/r over [x0,x1]x[y0,y1]x[z0,z1] (no 1/(4 pi eps0)). */
static q128 box_integral(q128 x0, q128 x1, q128 y0, q128 y1, q128 z0, q128 z1)
{
    q128 s = 0;
    s += igf_antiderivative(x1, y1, z1);
    s -= igf_antiderivative(x0, y1, z1);
    s -= igf_antiderivative(x1, y0, z1);
    s -= igf_antiderivative(x1, y1, z0);
    s += igf_antiderivative(x0, y0, z1);
    s += igf_antiderivative(x0, y1, z0);
    s += igf_antiderivative(x1, y0, z0);
    s -= igf_antiderivative(x0, y0, z0);
    return s;
}

/* G at one (possibly non-integer or negative) offset, in units of the cell. */
double oracle_igf_point(double a, double b, double c, double hx, double hy, double hz)
{
    q128 x = (q128)a * hx, y = (q128)b * hy, z = (q128)c * hz;
    q128 s = box_integral(x - 0.5Q * hx, x + 0.5Q * hx, y - 0.5Q * hy, y + 0.5Q * hy,
                          z - 0.5Q * hz, z + 0.5Q * hz);
    return (double)(s / (4 * M_PIq * EPS0_Q));
}

/* Plain-double evaluation of the same 8-corner sum (used only by the tests to
 * show why extended precision is needed). */
double oracle_igf_point_double(double a, double b, double c, double hx, double hy, double hz);

/*
 * Octant table: out[(cc*(n+1) + bb)*(n+1) + aa] = G(aa, bb, cc), aa,bb,cc = 0..n.
 * F is evaluated once per corner of the (n+2)^3 corner lattice
 * x_i = (i - 1/2) hx, i = 0..n+1 (likewise y, z); G(a,b,c) is the alternating
 * sum over corners i in {a, a+1}, j in {b, b+1}, k in {c, c+1}.
 * Returns 0 on success, -1 on allocation failure.
 */
int oracle_igf_octant(int n, double hx, double hy, double hz, double *out)
{
    int m = n + 2;
    q128 *ft = (q128 *)malloc(sizeof(q128) * (size_t)m * m * m);
    if (!ft) return -1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < m; k++)
        for (int j = 0; j < m; j++)
            for (int i = 0; i < m; i++)
                ft[((size_t)k * m + j) * m + i] =
                    igf_antiderivative((i - 0.5Q) * hx, (j - 0.5Q) * hy, (k - 0.5Q) * hz);
    q128 norm = 4 * M_PIq * EPS0_Q;
#pragma omp parallel for collapse(2) schedule(static)
    for (int c = 0; c <= n; c++)
        for (int b = 0; b <= n; b++)
            for (int a = 0; a <= n; a++) {
                q128 s = 0;
                for (int dk = 0; dk < 2; dk++)
                    for (int dj = 0; dj < 2; dj++)
                        for (int di = 0; di < 2; di++) {
                            /* +1 when an even number of lower corners */
                            int sign = ((di + dj + dk) % 2 == 1) ? 1 : -1;
                            q128 v = ft[((size_t)(c + dk) * m + (b + dj)) * m + (a + di)];
                            s += sign > 0 ? v : -v;
                        }
                out[((size_t)c * (n + 1) + b) * (n + 1) + a] = (double)(s / norm);
            }
    free(ft);
    return 0;
}

static double f_double(double x, double y, double z)
{
    double x2 = x * x, y2 = y * y, z2 = z * z;
    double r = __builtin_sqrt(x2 + y2 + z2);
#define LNUR(u, rest2) ((u) >= 0 ? __builtin_log((u) + r) : __builtin_log((rest2) / (r - (u))))
    return -0.5 * z2 * __builtin_atan(x * y / (z * r)) - 0.5 * y2 * __builtin_atan(x * z / (y * r))
           - 0.5 * x2 * __builtin_atan(y * z / (x * r)) + y * z * LNUR(x, y2 + z2)
           + x * z * LNUR(y, x2 + z2) + x * y * LNUR(z, x2 + y2);
#undef LNUR
}

double oracle_igf_point_double(double a, double b, double c, double hx, double hy, double hz)
{
    double x0 = (a - 0.5) * hx, x1 = (a + 0.5) * hx, y0 = (b - 0.5) * hy, y1 = (b + 0.5) * hy;
    double z0 = (c - 0.5) * hz, z1 = (c + 0.5) * hz;
    double s = f_double(x1, y1, z1) - f_double(x0, y1, z1) - f_double(x1, y0, z1)
               - f_double(x1, y1, z0) + f_double(x0, y0, z1) + f_double(x0, y1, z0)
               + f_double(x1, y0, z0) - f_double(x0, y0, z0);
    return s / (4 * 3.14159265358979323846 * 8.8541878128e-12);
}
