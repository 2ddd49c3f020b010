// Reverse (adjoint) kernels of the tracking step: the transpose of the
// Jacobian of each forward kernel, per kick in reverse order.
//
// Paper anchor (arXiv:2208.02382): the Introduction and Outlook motivate
// coupling the code to machine-learning workflows; the paper gives no
// adjoint.  Forward step (Model Assumptions, Listing 1): map(ds/2) -> kick
// over ds from the rest-frame field of the CIC-deposited charge -> map(ds/2).
// With P_k the state before kick k (after the merged map M_k), the kick
// Q_k = P_k + dP(X(P_k)) and P_{k+1} = M_{k+1} Q_k.  Reverse of kick k, given
// Pbar_{k+1}:
//   B1  Qbar = M_{k+1}^T Pbar_{k+1};  Mbar_{k+1} = sum_p Pbar_{k+1} Q_k^T;
//       Kbar_d(node) = sum_p w_p(node) Qbar_{p_d}   (scatter, fixed point);
//       Xbar += Qbar_p . d(dP)/dX                  (gather-weight term)
//   grid  phibar = -D^T (c Kbar);  rhobar = G (*) phibar  (G even)
//   B2  Xbar += (q/V) sum_nodes rhobar(node) dw_p(node)/dX  (deposit term)
// with X = x, Y = y, Z = -beta gamma t.  The box of a kick is held fixed
// (piecewise constant in the coordinates; its derivative is taken as zero).
//
// Arithmetic follows the forward kernels: the cells and 52-bit fractions are
// the forward's (shared code), the field derivative is the derivative of its
// fixed-point trilinear interpolation formed from the same integer lerps, and
// the scatter accumulates in int64 fixed point (order-independent integer
// atomics, so the reverse pass is bitwise reproducible).  Block sums run in a
// fixed order.
#include <algorithm>
#include <climits>

#include "common.cuh"
#include "fixed.cuh"
#include "particle_math.cuh"

namespace bt {

constexpr int ATPB = 256;
constexpr int ADJ_PPT = 4;

int adj_blocks(int64_t n) {
    int64_t b = (n + ATPB * ADJ_PPT - 1) / (ATPB * ADJ_PPT);
    if (b > 148 * 8) b = 148 * 8;
    return (int)(b < 1 ? 1 : b);
}

// Sum of K values over the block in a fixed order (warp butterflies, then the
// warps in index order); thread k < K writes out[k].
template <int K>
__device__ __forceinline__ void block_sum_fixed(double (&v)[K], double *out) {
    __shared__ double sm[K][ATPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double a = v[k];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) sm[k][w] = a;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += ATPB) {
        double s = 0.0;
        for (int i = 0; i < ATPB / 32; ++i) s += sm[k][i];
        out[k] = s;
    }
}

// Block maximum of |v| per component as bits, folded in with integer atomics.
template <int K>
__device__ __forceinline__ void block_max_commit(unsigned long long (&v)[K],
                                                 unsigned long long *const dst[K]) {
    __shared__ unsigned long long sm[K][ATPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        unsigned long long a = v[k];
        for (int o = 16; o > 0; o >>= 1) a = max(a, __shfl_xor_sync(0xffffffffu, a, o));
        if (lane == 0) sm[k][w] = a;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        unsigned long long a = 0;
        for (int i = 0; i < ATPB / 32; ++i) a = max(a, sm[threadIdx.x][i]);
        atomicMax(dst[threadIdx.x], a);
    }
}

__device__ __forceinline__ void particle_range(int64_t n, int64_t &b0, int64_t &b1) {
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    b0 = (int64_t)blockIdx.x * chunk;
    b1 = min(n, b0 + chunk);
}

// Cells and fractions of a position exactly as the forward kernels form them.
struct CellU {
    double ih0, ih1, ih2, o0, o1, o2, tz, lo0, lo1, lo2, nbg;
    bool exact;
    __device__ void init(const Box &b, double nbg_) {
        nbg = nbg_;
        ih0 = b.inv_h[0];
        ih1 = b.inv_h[1];
        ih2 = b.inv_h[2];
        o0 = b.off[0];
        o1 = b.off[1];
        o2 = b.off[2];
        tz = b.tz;
        lo0 = b.lo[0];
        lo1 = b.lo[1];
        lo2 = b.lo[2];
        exact = box_far_offset(b);
    }
    __device__ __forceinline__ void cells(double x, double y, double t, int nn, int &c0, int &c1,
                                          int &c2, unsigned long long &F0, unsigned long long &F1,
                                          unsigned long long &F2) const {
        bool out = false;
        if (exact) {
            cell_frac((x - lo0) * ih0, nn, c0, F0, out);
            cell_frac((y - lo1) * ih1, nn, c1, F1, out);
            cell_frac((__dmul_rn(nbg, t) - lo2) * ih2, nn, c2, F2, out);
        } else {
            cell_frac(fma(x, ih0, o0), nn, c0, F0, out);
            cell_frac(fma(y, ih1, o1), nn, c1, F1, out);
            cell_frac(fma(t, tz, o2), nn, c2, F2, out);
        }
    }
};

// --------------------------------------------------------------- seeding

// dL/dz of L = w0 eps_x + w1 eps_y + w2 sigma_x + w3 sigma_y at the final
// bunch, from its means and centred second moments (1/n normalisation; the
// mean terms cancel):
//   d sigma_u/du = du/(n sigma_u)
//   d eps_u/du = (C_pp du - C_up dpu)/(n eps_u), d eps_u/dpu = (C_uu dpu - C_up du)/(n eps_u)
__global__ void k_adj_seed(P6 c, int64_t n, const double *__restrict__ mom,
                           double w0, double w1, double w2, double w3, P6 A,
                           unsigned long long *amax) {
    // moment layout: means[6], then the upper triangle (00, 01, .., 05, 11, ..)
    const double mx = mom[0], mpx = mom[1], my = mom[2], mpy = mom[3];
    const double cxx = mom[6 + 0], cxp = mom[6 + 1], cpp = mom[6 + 6];
    const double cyy = mom[6 + 11], cyp = mom[6 + 12], cqq = mom[6 + 15];
    const double inv_n = 1.0 / (double)n;
    const double ex = sqrt(cxx * cpp - cxp * cxp), ey = sqrt(cyy * cqq - cyp * cyp);
    const double ax = ex > 0.0 ? w0 * inv_n / ex : 0.0, ay = ey > 0.0 ? w1 * inv_n / ey : 0.0;
    const double sx = cxx > 0.0 ? w2 * inv_n / sqrt(cxx) : 0.0;
    const double sy = cyy > 0.0 ? w3 * inv_n / sqrt(cyy) : 0.0;
    unsigned long long mv[6] = {0, 0, 0, 0, 0, 0};
    int64_t b0, b1;
    particle_range(n, b0, b1);
    for (int64_t p = b0 + threadIdx.x; p < b1; p += ATPB) {
        const double dx = c.p[0][p] - mx, dpx = c.p[1][p] - mpx, dy = c.p[2][p] - my, dpy = c.p[3][p] - mpy;
        const double v[6] = {ax * (cpp * dx - cxp * dpx) + sx * dx, ax * (cxx * dpx - cxp * dx),
                             ay * (cqq * dy - cyp * dpy) + sy * dy, ay * (cyy * dpy - cyp * dy),
                             0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            A.p[k][p] = v[k];
            mv[k] = max(mv[k], abs_bits(v[k]));
        }
    }
    unsigned long long *dst[6] = {amax, amax + 1, amax + 2, amax + 3, amax + 4, amax + 5};
    block_max_commit<6>(mv, dst);
}

// ------------------------------------------------------------------ B1

struct Adj1Args {
    P6 P;                          // state before the kick
    P6 A;                          // adjoint: Pbar_{k+1} in, Pbar_k momenta + gather term out
    const EFix *ef;                // the kick's field (fixed point) and exponents
    const int *escale;
    const Box *box;                // the kick's box
    const MapCoef *map;            // table entry 1 + k: M_{k+1} and the kick factors
    double nbg;                    // -beta gamma
    int nn;
    int lg;                        // ceil(log2 n) + 1
    int64_t n;
    const unsigned long long *amax_in;   // max |Pbar_{k+1}| per component (bits)
    unsigned long long *amax_out;        // max |Pbar_k| momenta (bits)
    unsigned long long *kbar;            // 3 nn^3 two's-complement accumulators
    int *sexp;                           // scatter exponents (out, block 0)
    double *part;                        // per-block partial sums of Mbar (13)
};

// Largest exponent S with bound * 2^S below 2^(59 - lg): each scattered
// value then stays below 2^(59-lg) units and a node sum of n of them below 2^59.
__device__ __forceinline__ int scatter_exponent(double bound, int lg) {
    if (!(bound > 0.0) || !isfinite(bound)) return 0;
    return 58 - lg - ilogb(bound);
}

__global__ void __launch_bounds__(ATPB) k_adj_kick1(Adj1Args a) {
    const MapCoef m = *a.map;
    double amx[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) amx[k] = __longlong_as_double((long long)a.amax_in[k]);
    // |Qbar_p| <= sum_i |M_{k+1}[i][p]| max|Pbar_{k+1,i}|
    const double bpx = fabs(m.m01) * amx[0] + fabs(m.m11) * amx[1] + fabs(m.m41) * amx[4];
    const double bpy = fabs(m.m23) * amx[2] + fabs(m.m33) * amx[3];
    const double bpt = fabs(m.m05) * amx[0] + fabs(m.m15) * amx[1] + fabs(m.m45) * amx[4] + amx[5];
    const int S0 = scatter_exponent(bpx, a.lg), S1 = scatter_exponent(bpy, a.lg),
              S2 = scatter_exponent(bpt, a.lg);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.sexp[0] = S0;
        a.sexp[1] = S1;
        a.sexp[2] = S2;
    }
    const double sc0 = ldexp(1.0, S0), sc1 = ldexp(1.0, S1), sc2 = ldexp(1.0, S2);
    const int e0 = a.escale[0], e1 = a.escale[1], e2 = a.escale[2];
    const double ie0 = ldexp(1.0, -e0), ie1 = ldexp(1.0, -e1), ie2 = ldexp(1.0, -e2);
    CellU cu;
    cu.init(*a.box, a.nbg);
    const int nn = a.nn;
    const long long n3 = (long long)nn * nn * nn;
    const unsigned long long one = 1ull << 52;
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) acc[k] = 0.0;
    unsigned long long mv[3] = {0, 0, 0};
    int64_t b0, b1;
    particle_range(a.n, b0, b1);
    for (int64_t p = b0 + threadIdx.x; p < b1; p += ATPB) {
        const double x = a.P.p[0][p], px = a.P.p[1][p], y = a.P.p[2][p], py = a.P.p[3][p], t = a.P.p[4][p],
                     pt = a.P.p[5][p];
        const double bx = a.A.p[0][p], bpxv = a.A.p[1][p], by = a.A.p[2][p], bpyv = a.A.p[3][p],
                     bt = a.A.p[4][p], bptv = a.A.p[5][p];
        int c0, c1, c2;
        unsigned long long F0u, F1u, F2u;
        cu.cells(x, y, t, nn, c0, c1, c2, F0u, F1u, F2u);
        const Frac F0 = split26(F0u), F1 = split26(F1u), F2 = split26(F2u);
        // the forward's interpolation, and the derivatives of the same
        // trilinear form in u (differences of the integer lerps)
        const EFix *e = &a.ef[((long long)c2 * nn + c1) * nn + c0];
        long long val[3], du[3][3];
        // the four x edges of the cell (y, z) = (0,0), (1,0), (0,1), (1,1): each
        // node's record in one 32-byte load, per component the edge's lerp in x
        // and its difference
        long long g[3][4], dx[3][4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const EFix *q = e + (j & 1) * nn + (j >> 1) * (long long)nn * nn;
            long long v0[3], v1[3];
            ld_efix(q, v0[0], v0[1], v0[2]);
            ld_efix(q + 1, v1[0], v1[1], v1[2]);
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                g[cc][j] = lerp52(v0[cc], v1[cc], F0);
                dx[cc][j] = v1[cc] - v0[cc];
            }
        }
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const long long gy0 = lerp52(g[cc][0], g[cc][1], F1), gy1 = lerp52(g[cc][2], g[cc][3], F1);
            val[cc] = lerp52(gy0, gy1, F2);
            du[cc][2] = gy1 - gy0;
            du[cc][1] = lerp52(g[cc][1] - g[cc][0], g[cc][3] - g[cc][2], F2);
            du[cc][0] = lerp52(lerp52(dx[cc][0], dx[cc][1], F1), lerp52(dx[cc][2], dx[cc][3], F1), F2);
        }
        // post-kick state (bitwise the forward's)
        const double qx = x, qpx = px + i64_scaled_to_double(val[0], e0);
        const double qy = y, qpy = py + i64_scaled_to_double(val[1], e1);
        const double qpt = pt + i64_scaled_to_double(val[2], e2);
        // Qbar = M^T Pbar
        const double gx = m.m00 * bx + m.m10 * bpxv + m.m40 * bt;
        const double gpx = m.m01 * bx + m.m11 * bpxv + m.m41 * bt;
        const double gy = m.m22 * by + m.m32 * bpyv;
        const double gpy = m.m23 * by + m.m33 * bpyv;
        const double gt = bt;
        const double gpt = m.m05 * bx + m.m15 * bpxv + m.m45 * bt + bptv;
        // Mbar partials on the map's 13 free entries
        acc[0] = fma(bx, qx, acc[0]);
        acc[1] = fma(bx, qpx, acc[1]);
        acc[2] = fma(bx, qpt, acc[2]);
        acc[3] = fma(bpxv, qx, acc[3]);
        acc[4] = fma(bpxv, qpx, acc[4]);
        acc[5] = fma(bpxv, qpt, acc[5]);
        acc[6] = fma(by, qy, acc[6]);
        acc[7] = fma(by, qpy, acc[7]);
        acc[8] = fma(bpyv, qy, acc[8]);
        acc[9] = fma(bpyv, qpy, acc[9]);
        acc[10] = fma(bt, qx, acc[10]);
        acc[11] = fma(bt, qpx, acc[11]);
        acc[12] = fma(bt, qpt, acc[12]);
        // gather-weight term: d(dP_c)/du_e = du[c][e] 2^-e_c
        const double s0 = gpx * ie0, s1 = gpy * ie1, s2 = gpt * ie2;
        const double gu0 = s0 * (double)du[0][0] + s1 * (double)du[1][0] + s2 * (double)du[2][0];
        const double gu1 = s0 * (double)du[0][1] + s1 * (double)du[1][1] + s2 * (double)du[2][1];
        const double gu2 = s0 * (double)du[0][2] + s1 * (double)du[1][2] + s2 * (double)du[2][2];
        a.A.p[0][p] = fma(gu0, cu.ih0, gx);
        a.A.p[1][p] = gpx;
        a.A.p[2][p] = fma(gu1, cu.ih1, gy);
        a.A.p[3][p] = gpy;
        a.A.p[4][p] = fma(gu2, cu.tz, gt);
        a.A.p[5][p] = gpt;
        mv[0] = max(mv[0], abs_bits(gpx));
        mv[1] = max(mv[1], abs_bits(gpy));
        mv[2] = max(mv[2], abs_bits(gpt));
        // scatter of the momentum adjoint with the CIC weights (51-bit)
        const long long V[3] = {__double2ll_rn(gpx * sc0), __double2ll_rn(gpy * sc1),
                                __double2ll_rn(gpt * sc2)};
        const Frac wx[2] = {split26(one - F0u), split26(F0u)};
        const Frac wy[2] = {split26(one - F1u), split26(F1u)};
        const Frac wz[2] = {split26(one - F2u), split26(F2u)};
        const long long cell = ((long long)c2 * nn + c1) * nn + c0;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const Frac wyz = split26(mulshr52(wy[dy], wz[dz]));
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const unsigned long long W = (mulshr52(wx[dx], wyz) >> 1) << 13;
                    const long long node = cell + ((long long)dz * nn + dy) * nn + dx;
#pragma unroll
                    for (int cc = 0; cc < 3; ++cc) {
                        const long long v = V[cc];
                        const unsigned long long mag =
                            __umul64hi(v < 0 ? (unsigned long long)(-v) : (unsigned long long)v, W);
                        const unsigned long long add = v < 0 ? (0ull - mag) : mag;
                        if (mag) atomicAdd(&a.kbar[cc * n3 + node], add);
                    }
                }
            }
    }
    block_sum_fixed<13>(acc, a.part + (size_t)blockIdx.x * 13);
    unsigned long long *dst[3] = {a.amax_out + 1, a.amax_out + 3, a.amax_out + 5};
    block_max_commit<3>(mv, dst);
}

// ------------------------------------------------------------- grid part

// phibar(m) = sum_d c_d/(2 h_d) 2^-S_d (Kbar_d(m + e_d) - Kbar_d(m - e_d)) on
// nodes m = -1..n (index m + 1), Kbar = 0 outside nodes 0..n-1: the transpose
// of K_d = -c_d (phi(+e_d) - phi(-e_d))/(2 h_d).
__global__ void k_adj_phibar(const long long *__restrict__ kbar, int nn, const int *sexp,
                             const Box *box, const MapCoef *map, double *__restrict__ phibar) {
    const int q = nn + 2;
    const long long n3 = (long long)nn * nn * nn, q3 = (long long)q * q * q;
    // the forward field's k/(2h), formed the same way (from 1/h)
    const double c0 = ldexp(map->kick_t * (0.5 * box->inv_h[0]), -sexp[0]);
    const double c1 = ldexp(map->kick_t * (0.5 * box->inv_h[1]), -sexp[1]);
    const double c2 = ldexp(map->kick_z * (0.5 * box->inv_h[2]), -sexp[2]);
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < q3;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx % q) - 1, j = (int)((idx / q) % q) - 1, l = (int)(idx / ((long long)q * q)) - 1;
        auto K = [&](int d, int ii, int jj, int ll) -> long long {
            if (ii < 0 || jj < 0 || ll < 0 || ii >= nn || jj >= nn || ll >= nn) return 0;
            return kbar[d * n3 + ((long long)ll * nn + jj) * nn + ii];
        };
        const long long dx = K(0, i + 1, j, l) - K(0, i - 1, j, l);
        const long long dy = K(1, i, j + 1, l) - K(1, i, j - 1, l);
        const long long dz = K(2, i, j, l + 1) - K(2, i, j, l - 1);
        phibar[idx] = c0 * (double)dx + c1 * (double)dy + c2 * (double)dz;
    }
}

// ------------------------------------------------------------------ B2

struct Adj2Args {
    P6 P;
    P6 A;
    const Box *box;
    double nbg;
    int nn;
    int64_t n;
    const double *rb;              // solve_adjoint_shifted output: rhobar(j) = rb[j + 2]
    double q_macro;
    unsigned long long *amax_out;  // max |Pbar_k| positions (bits)
};

__global__ void __launch_bounds__(ATPB) k_adj_kick2(Adj2Args a) {
    CellU cu;
    cu.init(*a.box, a.nbg);
    const int nn = a.nn, q = nn + 2;
    const double qv = a.q_macro / (a.box->h[0] * a.box->h[1] * a.box->h[2]);
    const double kx = qv * cu.ih0, ky = qv * cu.ih1, kz = qv * cu.tz;
    unsigned long long mv[3] = {0, 0, 0};
    int64_t b0, b1;
    particle_range(a.n, b0, b1);
    for (int64_t p = b0 + threadIdx.x; p < b1; p += ATPB) {
        int c0, c1, c2;
        unsigned long long F0u, F1u, F2u;
        cu.cells(a.P.p[0][p], a.P.p[2][p], a.P.p[4][p], nn, c0, c1, c2, F0u, F1u, F2u);
        const double f0 = (double)F0u * 0x1p-52, f1 = (double)F1u * 0x1p-52, f2 = (double)F2u * 0x1p-52;
        const double *r = a.rb + ((long long)(c2 + 2) * q + (c1 + 2)) * q + (c0 + 2);
        const long long sy = q, sz = (long long)q * q;
        const double r000 = r[0], r001 = r[1], r010 = r[sy], r011 = r[sy + 1];
        const double r100 = r[sz], r101 = r[sz + 1], r110 = r[sz + sy], r111 = r[sz + sy + 1];
        // x-differences and x-interpolants per (y, z) edge
        const double d00 = r001 - r000, d01 = r011 - r010, d10 = r101 - r100, d11 = r111 - r110;
        const double a00 = fma(f0, d00, r000), a01 = fma(f0, d01, r010);
        const double a10 = fma(f0, d10, r100), a11 = fma(f0, d11, r110);
        const double ddx = fma(f2, fma(f1, d11 - d10, d10) - fma(f1, d01 - d00, d00),
                               fma(f1, d01 - d00, d00));
        const double ey0 = a01 - a00, ey1 = a11 - a10;
        const double ddy = fma(f2, ey1 - ey0, ey0);
        const double z0 = fma(f1, a01 - a00, a00), z1 = fma(f1, a11 - a10, a10);
        const double ddz = z1 - z0;
        const double vx = fma(kx, ddx, a.A.p[0][p]);
        const double vy = fma(ky, ddy, a.A.p[2][p]);
        const double vt = fma(kz, ddz, a.A.p[4][p]);
        a.A.p[0][p] = vx;
        a.A.p[2][p] = vy;
        a.A.p[4][p] = vt;
        mv[0] = max(mv[0], abs_bits(vx));
        mv[1] = max(mv[1], abs_bits(vy));
        mv[2] = max(mv[2], abs_bits(vt));
    }
    unsigned long long *dst[3] = {a.amax_out + 0, a.amax_out + 2, a.amax_out + 4};
    block_max_commit<3>(mv, dst);
}

// ------------------------------------------------------------ initial map

// zbar0 = M_0^T Pbar_0 (written to out), and per block the sums of
// Pbar_0 z0^T on the map's 13 entries and of zbar0 z0^T (36, row-major).
__global__ void __launch_bounds__(ATPB) k_adj_initial(P6 A, P6 z0, int64_t n,
                                                      const MapCoef *map0, P6 out, double *part) {
    const MapCoef m = *map0;
    double acc[49];
#pragma unroll
    for (int k = 0; k < 49; ++k) acc[k] = 0.0;
    int64_t b0, b1;
    particle_range(n, b0, b1);
    for (int64_t p = b0 + threadIdx.x; p < b1; p += ATPB) {
        const double bx = A.p[0][p], bpx = A.p[1][p], by = A.p[2][p], bpy = A.p[3][p],
                     bt = A.p[4][p], bpt = A.p[5][p];
        const double z[6] = {z0.p[0][p], z0.p[1][p], z0.p[2][p], z0.p[3][p], z0.p[4][p], z0.p[5][p]};
        const double g[6] = {m.m00 * bx + m.m10 * bpx + m.m40 * bt,
                             m.m01 * bx + m.m11 * bpx + m.m41 * bt,
                             m.m22 * by + m.m32 * bpy,
                             m.m23 * by + m.m33 * bpy,
                             bt,
                             m.m05 * bx + m.m15 * bpx + m.m45 * bt + bpt};
        acc[0] = fma(bx, z[0], acc[0]);
        acc[1] = fma(bx, z[1], acc[1]);
        acc[2] = fma(bx, z[5], acc[2]);
        acc[3] = fma(bpx, z[0], acc[3]);
        acc[4] = fma(bpx, z[1], acc[4]);
        acc[5] = fma(bpx, z[5], acc[5]);
        acc[6] = fma(by, z[2], acc[6]);
        acc[7] = fma(by, z[3], acc[7]);
        acc[8] = fma(bpy, z[2], acc[8]);
        acc[9] = fma(bpy, z[3], acc[9]);
        acc[10] = fma(bt, z[0], acc[10]);
        acc[11] = fma(bt, z[1], acc[11]);
        acc[12] = fma(bt, z[5], acc[12]);
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j) acc[13 + 6 * i + j] = fma(g[i], z[j], acc[13 + 6 * i + j]);
#pragma unroll
        for (int i = 0; i < 6; ++i) out.p[i][p] = g[i];
    }
    block_sum_fixed<49>(acc, part + (size_t)blockIdx.x * 49);
}

// out[k] = sum over blocks b (in order) of part[b*K + k].
__global__ void k_adj_reduce(const double *__restrict__ part, int nblocks, int K,
                             double *__restrict__ out) {
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(size_t)b * K + k];
        out[k] = s;
    }
}

// --------------------------------------------------- Green's function store

// dir 0: after a gated build, store[green_builds - 1] = ghat;
// dir 1: instead of a build, ghat = store[green_builds - 1].
__global__ void k_ghat_store(const TrackState *st, double *__restrict__ store,
                             double *__restrict__ ghat, long long count, int cap, int dir,
                             int32_t *status) {
    if (!st->green_stale || st->halt) return;
    const int slot = st->green_builds - 1;
    if (slot < 0 || slot >= cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(status, ST_OUTSIDE);
        return;
    }
    double *s = store + (long long)slot * count;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        if (dir == 0) s[i] = ghat[i];
        else ghat[i] = s[i];
    }
}

// ghat = store[slot_hist[k]] (the Green's function in use at kick k).
__global__ void k_ghat_fetch(const int32_t *slot_hist, long long k, const double *__restrict__ store,
                             double *__restrict__ ghat, long long count, int cap) {
    const int slot = slot_hist[k];
    if (slot < 0 || slot >= cap) return;
    const double *s = store + (long long)slot * count;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x)
        ghat[i] = s[i];
}

__global__ void k_set_deposit_gate(TrackState *st) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !st->halt) st->deposit_gate = 1;
}

// ------------------------------------------------------------- Twiss bunch

// u = sqrt(eps beta) xi_u, pu = sqrt(eps/beta) (xi_pu - alpha xi_u) per
// transverse plane; t = sigma_t xi_t, pt = sigma_pt xi_pt.
__global__ void k_twiss_beam(P6 xi, int64_t n, double sx, double spx, double ax, double sy,
                             double spy, double ay, double st, double spt, P6 out) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double x0 = xi.p[0][p], x1 = xi.p[1][p], y0 = xi.p[2][p], y1 = xi.p[3][p];
        out.p[0][p] = sx * x0;
        out.p[1][p] = spx * (x1 - ax * x0);
        out.p[2][p] = sy * y0;
        out.p[3][p] = spy * (y1 - ay * y0);
        out.p[4][p] = st * xi.p[4][p];
        out.p[5][p] = spt * xi.p[5][p];
    }
}

// Listing-1 parametrisation (see bx_distribution_beam): c[3 plane + 0] =
// sigmaU/sqrt(1-mu^2), c[3 plane + 1] = sigmaPu, c[3 plane + 2] = mu/sqrt(1-mu^2).
__global__ void k_distribution(int kind, P6 z, const double *__restrict__ uni, int64_t n,
                               Coef9 c9, P6 out) {
    const double *c = c9.c;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = z.p[k][p];
        if (kind == 1) {
            double r2 = 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) r2 += a[k] * a[k];
            const double s = sqrt(8.0) * pow(uni[p], 1.0 / 6.0) / sqrt(r2);
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] *= s;
        }
#pragma unroll
        for (int pl = 0; pl < 3; ++pl) {
            const double u = a[2 * pl], pu = a[2 * pl + 1];
            out.p[2 * pl][p] = c[3 * pl] * u;
            out.p[2 * pl + 1][p] = c[3 * pl + 1] * (pu - c[3 * pl + 2] * u);
        }
    }
}

// ---------------------------------------------------------------- launchers

static int grid_lin(long long n) {
    long long b = (n + 255) / 256;
    if (b > 148 * 16) b = 148 * 16;
    return (int)(b < 1 ? 1 : b);
}

cudaError_t launch_adj_seed(P6 c_dev, int64_t n, const double *mom, const double w[4], P6 A_dev,
                            unsigned long long *amax, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(amax, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    BT_LAUNCH(K_ADJ_PART, s, k_adj_seed<<<adj_blocks(n), ATPB, 0, s>>>(c_dev, n, mom, w[0], w[1],
                                                                       w[2], w[3], A_dev, amax));
    return cudaGetLastError();
}

cudaError_t launch_adj_kick(const AdjKick &k, cudaStream_t s) {
    const long long n3 = (long long)k.nn * k.nn * k.nn;
    const long long q = k.nn + 2, q3 = q * q * q;
    const int nb = adj_blocks(k.n);
    cudaError_t e = cudaMemsetAsync(k.kbar, 0, 3 * n3 * sizeof(long long), s);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(k.amax_out, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int lg = 1;
    while (((int64_t)1 << lg) < k.n) ++lg;
    lg += 1;
    Adj1Args a1{k.P, k.A, k.ef, k.escale, k.box, k.map, -k.betagamma, k.nn, lg, k.n, k.amax_in,
                k.amax_out, (unsigned long long *)k.kbar, k.sexp, k.part};
    BT_LAUNCH(K_ADJ_PART, s, k_adj_kick1<<<nb, ATPB, 0, s>>>(a1));
    BT_LAUNCH(K_ADJ_GRID, s, k_adj_reduce<<<1, 32, 0, s>>>(k.part, nb, 13, k.mbar));
    BT_LAUNCH(K_ADJ_GRID, s, k_adj_phibar<<<grid_lin(q3), 256, 0, s>>>(k.kbar, k.nn, k.sexp, k.box,
                                                                      k.map, k.phibar));
    BT_LAUNCH(K_ADJ_GRID, s, k_ghat_fetch<<<grid_lin(k.ghat_count), 256, 0, s>>>(
                                 k.slot_hist, k.kick, k.ghat_store, k.plan->ghat, k.ghat_count,
                                 k.ghat_cap));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = green_quantize(k.plan, s);
    if (e != cudaSuccess) return e;
    e = solve_adjoint_shifted_fixed(k.plan, k.phibar, k.rb, s);
    if (e != cudaSuccess) return e;
    Adj2Args a2{k.P, k.A, k.box, -k.betagamma, k.nn, k.n, k.rb, k.q_macro, k.amax_out};
    BT_LAUNCH(K_ADJ_PART, s, k_adj_kick2<<<nb, ATPB, 0, s>>>(a2));
    return cudaGetLastError();
}

cudaError_t launch_adj_initial(P6 A_dev, P6 z0_dev, int64_t n, const MapCoef *map0, P6 out_dev,
                               double *part, double *sums, cudaStream_t s) {
    const int nb = adj_blocks(n);
    BT_LAUNCH(K_ADJ_PART, s, k_adj_initial<<<nb, ATPB, 0, s>>>(A_dev, z0_dev, n, map0, out_dev, part));
    BT_LAUNCH(K_ADJ_GRID, s, k_adj_reduce<<<1, 64, 0, s>>>(part, nb, 49, sums));
    return cudaGetLastError();
}

cudaError_t launch_ghat_store(const TrackState *st, double *store, double *ghat, long long count,
                              int cap, int dir, int32_t *status, cudaStream_t s) {
    BT_LAUNCH(K_ADJ_GRID, s, k_ghat_store<<<grid_lin(count), 256, 0, s>>>(st, store, ghat, count,
                                                                         cap, dir, status));
    return cudaGetLastError();
}

cudaError_t launch_ghat_fetch(const int32_t *slot_hist, long long k, const double *store,
                              double *ghat, long long count, int cap, cudaStream_t s) {
    BT_LAUNCH(K_ADJ_GRID, s, k_ghat_fetch<<<grid_lin(count), 256, 0, s>>>(slot_hist, k, store, ghat,
                                                                         count, cap));
    return cudaGetLastError();
}

cudaError_t launch_set_deposit_gate(TrackState *st, cudaStream_t s) {
    BT_LAUNCH(K_BOX, s, k_set_deposit_gate<<<1, 32, 0, s>>>(st));
    return cudaGetLastError();
}

cudaError_t launch_distribution(int kind, P6 z, const double *uni, int64_t n, Coef9 c, P6 out,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_ADJ_PART, s, k_distribution<<<grid_lin(n), 256, 0, s>>>(kind, z, uni, n, c, out));
    return cudaGetLastError();
}

cudaError_t launch_twiss_beam(P6 xi_dev, int64_t n, const double c[8], P6 out_dev,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_ADJ_PART, s, k_twiss_beam<<<grid_lin(n), 256, 0, s>>>(
                                 xi_dev, n, c[0], c[1], c[2], c[3], c[4], c[5], c[6], c[7],
                                 out_dev));
    return cudaGetLastError();
}

__global__ void k_permute6(P6 in, const int *__restrict__ dest, int64_t n, P6 out, int gather) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = dest[p];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            if (gather) out.p[c][p] = in.p[c][d];
            else out.p[c][d] = in.p[c][p];
        }
    }
}

cudaError_t launch_permute6(P6 in, const int *dest, int64_t n, P6 out, bool gather,
                            cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int b = (int)std::min<int64_t>((n + 255) / 256, 148 * 16);
    BT_LAUNCH(K_ADJ_PART, s, k_permute6<<<b, 256, 0, s>>>(in, dest, n, out, gather ? 1 : 0));
    return cudaGetLastError();
}

}  // namespace bt
