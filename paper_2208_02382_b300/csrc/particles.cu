// Particle-side kernels of the tracking step: element push, exact min/max of
// the rest-frame positions, the grid-box rule, CIC charge deposition in fixed
// point, the rest-frame field and the fused gather + kick + push.
//
// Paper anchors (arXiv:2208.02382): Model Assumptions (linear symplectic maps
// in s; electrostatic rest-frame field; map-based split-operator step) and
// Listing 1 (particle shape, init_grids, elements with nslice).
#include "common.cuh"

namespace bt {

constexpr int TPB = 256;

__device__ __forceinline__ void apply_map(const MapCoef &m, double &x, double &px, double &y,
                                          double &py, double &t, double pt) {
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

static inline int grid_for(int64_t n) {
    int64_t b = (n + TPB - 1) / TPB;
    if (b > 148 * 16) b = 148 * 16;
    return (int)(b < 1 ? 1 : b);
}

// ---------------------------------------------------------------- push only

__global__ void k_push_maps(double *__restrict__ x, double *__restrict__ px,
                            double *__restrict__ y, double *__restrict__ py,
                            double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                            const MapCoef *__restrict__ maps, int nmaps) {
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a = x[p], b = px[p], c = y[p], d = py[p], e = t[p], f = pt[p];
        for (int k = 0; k < nmaps; ++k) apply_map(maps[k], a, b, c, d, e, f);
        x[p] = a;
        px[p] = b;
        y[p] = c;
        py[p] = d;
        t[p] = e;
    }
}

cudaError_t launch_push_maps(double *const c[6], int64_t n, const MapCoef *maps, int nmaps,
                             cudaStream_t s) {
    if (n <= 0 || nmaps <= 0) return cudaSuccess;
    BT_LAUNCH(K_PUSH, s, k_push_maps<<<grid_for(n), TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, maps, nmaps));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ min/max

// Block-level min/max of the rest-frame positions, folded into the state with
// integer atomics on order-preserving keys (exact and order-free).
__device__ __forceinline__ void block_minmax_commit(double lo[3], double hi[3], TrackState *st) {
    __shared__ double s_lo[3][TPB / 32], s_hi[3][TPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        double a = lo[d], b = hi[d];
        for (int o = 16; o > 0; o >>= 1) {
            a = fmin(a, __shfl_xor_sync(0xffffffffu, a, o));
            b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
        }
        if (lane == 0) {
            s_lo[d][w] = a;
            s_hi[d][w] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            double a = s_lo[d][0], b = s_hi[d][0];
            for (int k = 1; k < TPB / 32; ++k) {
                a = fmin(a, s_lo[d][k]);
                b = fmax(b, s_hi[d][k]);
            }
            atomicMin(&st->mm[d], dkey(a));
            atomicMax(&st->mm[3 + d], dkey(b));
        }
    }
}

__global__ void k_minmax(const double *__restrict__ x, const double *__restrict__ px,
                         const double *__restrict__ y, const double *__restrict__ py,
                         const double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                         double nbg, TrackState *st, int32_t *status) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a = x[p], b = y[p], c = t[p];
        bad |= !(isfinite(a) && isfinite(px[p]) && isfinite(b) && isfinite(py[p]) &&
                 isfinite(c) && isfinite(pt[p]));
        double z = nbg * c;
        lo[0] = fmin(lo[0], a);
        hi[0] = fmax(hi[0], a);
        lo[1] = fmin(lo[1], b);
        hi[1] = fmax(hi[1], b);
        lo[2] = fmin(lo[2], z);
        hi[2] = fmax(hi[2], z);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    block_minmax_commit(lo, hi, st);
}

cudaError_t launch_minmax(double *const c[6], int64_t n, double betagamma, TrackState *st,
                          int32_t *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_MINMAX, s, k_minmax<<<grid_for(n), TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, -betagamma, st,
                                         status));
    return cudaGetLastError();
}

// ----------------------------------------------------------------- box rule

// Reading of Listing 1 init_grids (the paper states no rule): regrid when no
// box exists, a particle is outside [lo, hi), or an extent fell below half of
// the box; the new box is centred on (min+max)/2 with half-width 0.55*extent,
// extents floored at 1e-6 of the largest (1e-6 m if all are zero).  Explicit
// round-to-nearest intrinsics keep every operation as written (no FMA
// contraction), so the decision matches a plain IEEE evaluation.
__global__ void k_box_rule(TrackState *st, int nn, long long *log, int64_t cap) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mn[3], mx[3], ext[3];
    double big = 0.0;
    for (int d = 0; d < 3; ++d) {
        mn[d] = dkey_inv(st->mm[d]);
        mx[d] = dkey_inv(st->mm[3 + d]);
        ext[d] = __dsub_rn(mx[d], mn[d]);
        big = fmax(big, ext[d]);
    }
    double floor_ext = big > 0.0 ? __dmul_rn(1e-6, big) : 1e-6;
    bool need = st->has_box == 0;
    for (int d = 0; d < 3; ++d) {
        ext[d] = fmax(ext[d], floor_ext);
        if (!need) {
            const Box &b = st->box;
            if (mn[d] < b.lo[d] || mx[d] >= b.hi[d] ||
                ext[d] < __dmul_rn(0.5, __dsub_rn(b.hi[d], b.lo[d])))
                need = true;
        }
    }
    if (need) {
        for (int d = 0; d < 3; ++d) {
            double c = __dmul_rn(0.5, __dadd_rn(mn[d], mx[d]));
            double w = __dmul_rn(0.55, ext[d]);
            double lo = __dsub_rn(c, w), hi = __dadd_rn(c, w);
            double h = __ddiv_rn(__dsub_rn(hi, lo), (double)(nn - 1));
            st->box.lo[d] = lo;
            st->box.hi[d] = hi;
            st->box.h[d] = h;
            st->box.inv_h[d] = __drcp_rn(h);
        }
        st->has_box = 1;
        if (st->nlog < cap) log[st->nlog] = st->kick;
        st->nlog += 1;
    }
    st->regrid = need ? 1 : 0;
    st->green_stale = (st->box.h[0] != st->green_h[0] || st->box.h[1] != st->green_h[1] ||
                       st->box.h[2] != st->green_h[2])
                          ? 1
                          : 0;
    for (int d = 0; d < 3; ++d) {
        st->mm[d] = dkey(INFINITY);
        st->mm[3 + d] = dkey(-INFINITY);
    }
}

cudaError_t launch_box_rule(TrackState *st, int nn, int64_t n, long long *log, int64_t cap,
                            cudaStream_t s) {
    (void)n;
    BT_LAUNCH(K_BOX, s, k_box_rule<<<1, 32, 0, s>>>(st, nn, log, cap));
    return cudaGetLastError();
}

// ------------------------------------------------------------------ deposit

// u (>= 0, < 2^11) to unsigned fixed point with 52 fractional bits, by
// exponent/mantissa arithmetic: exact for u >= 1, truncated below 1.
__device__ __forceinline__ unsigned long long to_fixed52(double u) {
    unsigned long long b = (unsigned long long)__double_as_longlong(u);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -60 || u <= 0.0) return 0ull;
    unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return e >= 0 ? (mant << e) : (mant >> (-e));
}

// (a * b) >> 52 for a, b <= 2^52 (the top bits of the 104-bit product).
__device__ __forceinline__ unsigned long long mulshr52(unsigned long long a,
                                                      unsigned long long b) {
    unsigned long long lo = a * b, hi = __umul64hi(a, b);
    return (hi << 12) | (lo >> 52);
}

// Charge deposition (Listing 1 particle shape 1 = CIC; ABLASTR deposition):
// node weights (1-f, f) per dimension, products in unsigned fixed point
// (52-bit fractions, 51-bit result), accumulated by integer atomics so the
// result is independent of particle order.
__global__ void k_deposit(const double *__restrict__ x, const double *__restrict__ y,
                          const double *__restrict__ t, int64_t n, double nbg, const Box *box,
                          int nn, unsigned long long *__restrict__ acc_hi,
                          unsigned long long *__restrict__ acc_lo, int32_t *status) {
    const double lo0 = box->lo[0], lo1 = box->lo[1], lo2 = box->lo[2];
    const double ih0 = box->inv_h[0], ih1 = box->inv_h[1], ih2 = box->inv_h[2];
    const unsigned long long one = 1ull << 52;
    const unsigned long long umax = (unsigned long long)(nn - 1) << 52;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double u[3];
        u[0] = (x[p] - lo0) * ih0;
        u[1] = (y[p] - lo1) * ih1;
        u[2] = (__dmul_rn(nbg, t[p]) - lo2) * ih2;  // Z rounded as stored, then offset
        int cell[3];
        unsigned long long w[3][2];
        bool outside = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            // a box that contains the particle gives u in [0, n-1] up to rounding
            outside |= !(u[d] >= 0.0) || u[d] > (double)(nn - 1) + 1e-6;
            unsigned long long U = to_fixed52(u[d]);
            if (U > umax) U = umax;
            unsigned long long i = U >> 52;
            if (i > (unsigned long long)(nn - 2)) i = nn - 2;
            unsigned long long f = U - (i << 52);
            cell[d] = (int)i;
            w[d][0] = one - f;
            w[d][1] = f;
        }
        if (outside) {
            atomicOr(status, ST_OUTSIDE);
            continue;
        }
        const long long base = ((long long)cell[2] * nn + cell[1]) * nn + cell[0];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                unsigned long long wyz = mulshr52(w[1][dy], w[2][dz]);
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    unsigned long long v = mulshr52(w[0][dx], wyz) >> 1;  // 51-bit result
                    long long node = base + ((long long)dz * nn + dy) * nn + dx;
                    atomicAdd(&acc_hi[node], v >> DEP_SPLIT);
                    atomicAdd(&acc_lo[node], v & ((1ull << DEP_SPLIT) - 1));
                }
            }
    }
}

cudaError_t launch_deposit(double *const c[6], int64_t n, double betagamma, const Box *box,
                              int nn, unsigned long long *acc_hi, unsigned long long *acc_lo,
                              int32_t *status, cudaStream_t s) {
    size_t nodes = (size_t)nn * nn * nn;
    cudaError_t e = cudaMemsetAsync(acc_hi, 0, nodes * 8, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc_lo, 0, nodes * 8, s);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_DEPOSIT, s, k_deposit<<<grid_for(n), TPB, 0, s>>>(c[0], c[2], c[4], n, -betagamma, box, nn, acc_hi, acc_lo,
                                          status));
    return cudaGetLastError();
}

// rho[node] = q * W / (hx hy hz) with W = (hi * 2^31 + lo) * 2^-51 the summed weights.
__global__ void k_acc_to_rho(const unsigned long long *__restrict__ acc_hi,
                             const unsigned long long *__restrict__ acc_lo, long long nodes,
                             double q_macro, const Box *box, double *__restrict__ rho) {
    const double vol = box->h[0] * box->h[1] * box->h[2];
    const double scale = q_macro / vol;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        double w = ((double)acc_hi[i] * 2147483648.0 + (double)acc_lo[i]) * 0x1p-51;
        rho[i] = scale * w;
    }
}

cudaError_t launch_acc_to_rho(const unsigned long long *acc_hi, const unsigned long long *acc_lo,
                              int nn, double q_macro, const Box *box, double *rho,
                              cudaStream_t s) {
    long long nodes = (long long)nn * nn * nn;
    BT_LAUNCH(K_ACC_TO_RHO, s, k_acc_to_rho<<<(int)((nodes + TPB - 1) / TPB), TPB, 0, s>>>(acc_hi, acc_lo, nodes, q_macro,
                                                               box, rho));
    return cudaGetLastError();
}

// -------------------------------------------------------------------- field

// Rest-frame field by centred differences on nodes 0..n-1 from phi on nodes
// -1..n, pre-multiplied by the kick factor of the slice:
//   efield[node] = (c_x (phi(i+1) - phi(i-1)), c_y (...), c_z (...), 0)
// with c_d = -kick_d / (2 h_d), so the gathered value is the momentum change.
__global__ void k_field(const double *__restrict__ phi, int nn, const Box *box, double kx,
                        double ky, double kz, Field4 *__restrict__ ef) {
    const int q = nn + 2;
    const double cx = -kx / (2.0 * box->h[0]);
    const double cy = -ky / (2.0 * box->h[1]);
    const double cz = -kz / (2.0 * box->h[2]);
    const long long nodes = (long long)nn * nn * nn;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nodes;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx % nn), j = (int)((idx / nn) % nn), l = (int)(idx / ((long long)nn * nn));
        long long c = ((long long)(l + 1) * q + (j + 1)) * q + (i + 1);
        double ex = cx * (phi[c + 1] - phi[c - 1]);
        double ey = cy * (phi[c + q] - phi[c - q]);
        double ez = cz * (phi[c + (long long)q * q] - phi[c - (long long)q * q]);
        ef[idx] = Field4{ex, ey, ez, 0.0};
    }
}

cudaError_t launch_field(const double *phi, int nn, const Box *box, double kx, double ky,
                         double kz, double *efield, cudaStream_t s) {
    long long nodes = (long long)nn * nn * nn;
    BT_LAUNCH(K_FIELD, s, k_field<<<(int)((nodes + TPB - 1) / TPB), TPB, 0, s>>>(phi, nn, box, kx, ky, kz,
                                                          (Field4 *)efield));
    return cudaGetLastError();
}

// ------------------------------------------------- gather + kick (+ push)

// CIC gather of the pre-scaled field at the particle (same weights as the
// deposit), momentum kick, then (optionally) the merged half-slice map, and
// (optionally) the min/max of the new rest-frame positions for the next box.
__global__ void k_gather_kick_push(double *__restrict__ x, double *__restrict__ px,
                                   double *__restrict__ y, double *__restrict__ py,
                                   double *__restrict__ t, double *__restrict__ pt, int64_t n,
                                   double nbg, const Box *box, int nn,
                                   const Field4 *__restrict__ ef, const MapCoef *map,
                                   TrackState *st, int32_t *status) {
    const double lo0 = box->lo[0], lo1 = box->lo[1], lo2 = box->lo[2];
    const double ih0 = box->inv_h[0], ih1 = box->inv_h[1], ih2 = box->inv_h[2];
    MapCoef m;
    if (map) m = *map;
    double mlo[3] = {INFINITY, INFINITY, INFINITY}, mhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a = x[p], b = px[p], c = y[p], d = py[p], e = t[p], f = pt[p];
        double u[3] = {(a - lo0) * ih0, (c - lo1) * ih1, (__dmul_rn(nbg, e) - lo2) * ih2};
        int cell[3];
        double wt[3][2];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            double fl = fmin(fmax(floor(u[k]), 0.0), (double)(nn - 2));
            double fr = u[k] - fl;
            cell[k] = (int)fl;
            wt[k][0] = 1.0 - fr;
            wt[k][1] = fr;
        }
        const long long base = ((long long)cell[2] * nn + cell[1]) * nn + cell[0];
        double ex = 0.0, ey = 0.0, ez = 0.0;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                double wyz = wt[1][dy] * wt[2][dz];
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    double w = wt[0][dx] * wyz;
                    Field4 v = ef[base + ((long long)dz * nn + dy) * nn + dx];
                    ex += w * v.x;
                    ey += w * v.y;
                    ez += w * v.z;
                }
            }
        b += ex;
        d += ey;
        f += ez;
        if (map) apply_map(m, a, b, c, d, e, f);
        bad |= !(isfinite(a) && isfinite(b) && isfinite(c) && isfinite(d) && isfinite(e) &&
                 isfinite(f));
        x[p] = a;
        px[p] = b;
        y[p] = c;
        py[p] = d;
        t[p] = e;
        pt[p] = f;
        double z = nbg * e;
        mlo[0] = fmin(mlo[0], a);
        mhi[0] = fmax(mhi[0], a);
        mlo[1] = fmin(mlo[1], c);
        mhi[1] = fmax(mhi[1], c);
        mlo[2] = fmin(mlo[2], z);
        mhi[2] = fmax(mhi[2], z);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    if (st) block_minmax_commit(mlo, mhi, st);
}

cudaError_t launch_gather_kick_push(double *const c[6], int64_t n, double betagamma,
                                    const Box *box, int nn, const double *efield,
                                    const MapCoef *map, TrackState *st, int32_t *status,
                                    cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_GATHER, s, k_gather_kick_push<<<grid_for(n), TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n,
                                                   -betagamma, box, nn,
                                                   (const Field4 *)efield, map, st, status));
    return cudaGetLastError();
}

}  // namespace bt
