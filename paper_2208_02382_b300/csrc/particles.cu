// Particle-side kernels of the tracking step: element push, exact min/max of
// the rest-frame positions, the grid-box rule, the rest-frame field in fixed
// point, and the fused particle kernel (CIC gather + kick + merged half-slice
// map + the next kick's CIC deposit + min/max).
//
// Paper anchors (arXiv:2208.02382): Model Assumptions (linear symplectic maps
// in s; electrostatic rest-frame field; map-based split-operator step) and
// Listing 1 (particle shape 1 = CIC, init_grids, elements with nslice).
//
// FP64 is spent only where the phase-space state is updated: u = (X - lo)/h,
// the linear map, and adding the kick.  Cell indices, CIC fractions and
// weights, the field interpolation, the charge accumulation and the min/max
// run in 64-bit fixed point on the integer pipes.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "fixed.cuh"
#include "particle_math.cuh"

namespace bt {

constexpr int TPB = 256;

static inline int grid_for(int64_t n) {
    int64_t b = (n + TPB - 1) / TPB;
    if (b > 148 * 16) b = 148 * 16;
    return (int)(b < 1 ? 1 : b);
}


int map_kind(const MapCoef &m) {
    if (m.m05 == 0.0 && m.m15 == 0.0 && m.m40 == 0.0 && m.m41 == 0.0) {
        if (m.m00 == 1.0 && m.m10 == 0.0 && m.m11 == 1.0 && m.m22 == 1.0 && m.m32 == 0.0 &&
            m.m33 == 1.0)
            return MAP_DRIFT;
        return MAP_QUAD;
    }
    if (m.m22 == 1.0 && m.m32 == 0.0 && m.m33 == 1.0) return MAP_BEND;
    return MAP_GENERAL;
}

// --------------------------------------------------- min/max and push only

// Warp minimum / maximum of a signed 64-bit value from two 32-bit warp
// reductions (redux): the extreme high word, then the extreme low word among
// the lanes holding it (signed 64-bit order is that of (signed high, unsigned
// low)).  All 32 lanes must call them.
__device__ __forceinline__ long long warp_min_i64(long long v) {
    const int h = (int)(v >> 32);
    const int mh = __reduce_min_sync(0xffffffffu, h);
    const unsigned ml = __reduce_min_sync(0xffffffffu, h == mh ? (unsigned)v : 0xFFFFFFFFu);
    return (long long)(((unsigned long long)(unsigned)mh << 32) | ml);
}
__device__ __forceinline__ long long warp_max_i64(long long v) {
    const int h = (int)(v >> 32);
    const int mh = __reduce_max_sync(0xffffffffu, h);
    const unsigned ml = __reduce_max_sync(0xffffffffu, h == mh ? (unsigned)v : 0u);
    return (long long)(((unsigned long long)(unsigned)mh << 32) | ml);
}

// Block min/max of order-preserving keys, folded into the state with integer
// atomics (exact, order-free).  All threads of the block must call it.
__device__ __forceinline__ void block_keys_commit(long long lo[3], long long hi[3],
                                                  TrackState *st) {
    __shared__ long long s_lo[3][TPB / 32], s_hi[3][TPB / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const long long a = warp_min_i64(lo[d]), b = warp_max_i64(hi[d]);
        if (lane == 0) {
            s_lo[d][w] = a;
            s_hi[d][w] = b;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            long long a = s_lo[d][0], b = s_hi[d][0];
            for (int k = 1; k < TPB / 32; ++k) {
                a = min(a, s_lo[d][k]);
                b = max(b, s_hi[d][k]);
            }
            atomicMin(&st->mm[d], a);
            atomicMax(&st->mm[3 + d], b);
        }
    }
}


// Maps (each by its class, uniform per entry) applied to every particle; with
// `st`, also the min/max keys of the new rest-frame positions (the box rule's
// input), so a call's prologue reads the bunch once.
__global__ void k_push_maps(double *__restrict__ x, double *__restrict__ px,
                            double *__restrict__ y, double *__restrict__ py,
                            double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                            const MapCoef *__restrict__ maps, int nmaps, int32_t *status,
                            TrackState *st, double nbg) {
    bool bad = false;
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a = x[p], b = px[p], c = y[p], d = py[p], e = t[p], f = pt[p];
        for (int k = 0; k < nmaps; ++k) apply_map_table(maps[k], maps + k, a, b, c, d, e, f);
        bad |= !finite6(a, b, c, d, e, f);
        x[p] = a;
        px[p] = b;
        y[p] = c;
        py[p] = d;
        t[p] = e;
        if (st) {
            const long long k0 = dkey(a), k1 = dkey(c), k2 = dkey(__dmul_rn(nbg, e));
            lo[0] = min(lo[0], k0);
            hi[0] = max(hi[0], k0);
            lo[1] = min(lo[1], k1);
            hi[1] = max(hi[1], k1);
            lo[2] = min(lo[2], k2);
            hi[2] = max(hi[2], k2);
        }
    }
    if (bad && status) atomicOr(status, ST_NONFINITE);
    if (st) block_keys_commit(lo, hi, st);
}

cudaError_t launch_push_maps(double *const c[6], int64_t n, const MapCoef *maps, int nmaps,
                             cudaStream_t s, int32_t *status, TrackState *st, double betagamma) {
    if (n <= 0 || nmaps <= 0) return cudaSuccess;
    BT_LAUNCH(K_PUSH, s, k_push_maps<<<grid_for(n), TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4],
                                                                 c[5], n, maps, nmaps, status, st,
                                                                 -betagamma));
    return cudaGetLastError();
}

__global__ void k_minmax(const double *__restrict__ x, const double *__restrict__ px,
                         const double *__restrict__ y, const double *__restrict__ py,
                         const double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                         double nbg, TrackState *st, int32_t *status) {
    long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double a = x[p], b = y[p], c = t[p];
        bad |= !finite6(a, px[p], b, py[p], c, pt[p]);
        const long long k0 = dkey(a), k1 = dkey(b), k2 = dkey(__dmul_rn(nbg, c));
        lo[0] = min(lo[0], k0);
        hi[0] = max(hi[0], k0);
        lo[1] = min(lo[1], k1);
        hi[1] = max(hi[1], k1);
        lo[2] = min(lo[2], k2);
        hi[2] = max(hi[2], k2);
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    block_keys_commit(lo, hi, st);
}

cudaError_t launch_minmax(double *const c[6], int64_t n, double betagamma, TrackState *st,
                          int32_t *status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    BT_LAUNCH(K_MINMAX, s, k_minmax<<<grid_for(n), TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5],
                                                                n, -betagamma, st, status));
    return cudaGetLastError();
}

// ----------------------------------------------------------------- box rule

// Reading of Listing 1 init_grids (the paper states no rule): regrid when no
// box exists, a particle is outside [lo, hi), or an extent fell below half of
// the box; the new box is centred on (min+max)/2 with half-width 0.55*extent,
// extents floored at 1e-6 of the largest (1e-6 m if all are zero).  Explicit
// round-to-nearest intrinsics keep every operation as written (no FMA
// contraction), so the decision matches a plain IEEE evaluation.
// With a replay table (differentiation runs) the box of each kick is taken
// from the table instead, a regrid being a box that differs from the current.

// With `advance` (tracking), the kick index of the call advances, the global
// kick counter is logged and incremented, and the gates of this kick are set.
__device__ void box_rule_body(TrackState *st, int nn, long long *log, int64_t cap, int advance) {
    if (advance) st->k_in_call += 1;
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
    if (st->box_replay) {
        const Box &rb = st->box_replay[st->kick];
        need = st->has_box == 0;
        for (int d = 0; d < 3; ++d)
            need = need || rb.lo[d] != st->box.lo[d] || rb.hi[d] != st->box.hi[d] ||
                   rb.h[d] != st->box.h[d] || rb.inv_h[d] != st->box.inv_h[d];
        if (need) {
            st->box = rb;
            st->has_box = 1;
            if (st->nlog < cap) log[st->nlog] = st->kick;
            st->nlog += 1;
        }
    } else if (need) {
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
    box_finish(st->box, st->nbg);
    // a box that is not finite (a bunch with Inf/NaN coordinates, or extents
    // beyond the double range) halts the kick: no Green's function, deposit,
    // sort or next kick (the particle kernel flags the coordinates)
    bool finite = true;
    for (int d = 0; d < 3; ++d)
        finite = finite && isfinite(st->box.lo[d]) && isfinite(st->box.hi[d]) && st->box.h[d] > 0.0 &&
                 isfinite(st->box.h[d]) && isfinite(st->box.inv_h[d]);
    st->regrid = need ? 1 : 0;
    st->halt = finite ? 0 : 1;
    st->green_stale = (finite && (st->box.h[0] != st->green_h[0] || st->box.h[1] != st->green_h[1] ||
                                  st->box.h[2] != st->green_h[2]))
                          ? 1
                          : 0;
    if (advance) {
        const int k = st->k_in_call;
        if (st->green_stale) st->green_builds += 1;
        if (st->box_hist) st->box_hist[st->kick] = st->box;
        if (st->slot_hist) st->slot_hist[st->kick] = st->green_builds - 1;
        // deposit for this kick unless it is in the accumulators already: the
        // previous kick's B, or (first kick of a call) the fused prologue into
        // the box that the rule kept
        // re-binning on the global kick count (it carries over between calls,
        // so tracking one kick per call re-bins every sort_interval kicks too)
        st->sort_gate =
            (finite && st->sort_interval > 0 && st->kick % st->sort_interval == 0) ? 1 : 0;
        // after a re-binning the kick deposits again: the charge is the same
        // (integer sums), but the stored cells must follow the new order
        st->deposit_gate = (finite && (need || st->sort_gate || (k == 0 && !st->pro_dep))) ? 1 : 0;
        st->next_gate = (finite && k + 1 < st->nkicks_call) ? 1 : 0;
        st->exact_u = box_far_offset(st->box) ? 1 : 0;
        st->rho_scale = st->q_macro / (st->box.h[0] * st->box.h[1] * st->box.h[2]);
        st->kick += 1;
    }
    for (int d = 0; d < 3; ++d) {
        st->mm[d] = LLONG_MAX;
        st->mm[3 + d] = LLONG_MIN;
    }
}

__global__ void k_box_rule(TrackState *st, int nn, long long *log, int64_t cap, int advance) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    box_rule_body(st, nn, log, cap, advance);
}

// Graph form: the gates also set the conditions of the kick graph's IF nodes.
__global__ void k_box_rule_graph(TrackState *st, int nn, long long *log, int64_t cap,
                                 cudaGraphConditionalHandle h_green,
                                 cudaGraphConditionalHandle h_sort,
                                 cudaGraphConditionalHandle h_dep,
                                 cudaGraphConditionalHandle h_next,
                                 cudaGraphConditionalHandle h_loop, int has_loop) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    box_rule_body(st, nn, log, cap, 1);
    cudaGraphSetConditional(h_green, st->green_stale ? 1u : 0u);
    cudaGraphSetConditional(h_sort, st->sort_gate ? 1u : 0u);
    cudaGraphSetConditional(h_dep, st->deposit_gate ? 1u : 0u);
    cudaGraphSetConditional(h_next, st->next_gate ? 1u : 0u);
    if (has_loop) cudaGraphSetConditional(h_loop, st->next_gate ? 1u : 0u);
}

cudaError_t launch_box_rule_graph(TrackState *st, int nn, long long *log, int64_t cap,
                                  cudaGraphConditionalHandle hg, cudaGraphConditionalHandle hs,
                                  cudaGraphConditionalHandle hd, cudaGraphConditionalHandle hn,
                                  cudaStream_t s, cudaGraphConditionalHandle hl, bool has_loop) {
    BT_LAUNCH(K_BOX, s, k_box_rule_graph<<<1, 32, 0, s>>>(st, nn, log, cap, hg, hs, hd, hn, hl,
                                                           has_loop ? 1 : 0));
    return cudaGetLastError();
}

cudaError_t launch_box_rule(TrackState *st, int nn, int64_t n, long long *log, int64_t cap,
                            bool advance, cudaStream_t s) {
    (void)n;
    BT_LAUNCH(K_BOX, s, k_box_rule<<<1, 32, 0, s>>>(st, nn, log, cap, advance ? 1 : 0));
    return cudaGetLastError();
}

// Start of a device-driven bx_track call.
// A fresh tracking state (no box, no Green's function, counters 0) set up
// for a call of nkicks kicks (the device-side counterpart of bx_reset +
// the start of bx_track, for graphs that track from scratch at each launch).
__global__ void k_state_reset(TrackState *st, int nkicks, double q_macro, int sort_interval,
                              double nbg) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        TrackState z;
        memset(&z, 0, sizeof(z));
        for (int d = 0; d < 3; ++d) {
            z.mm[d] = LLONG_MAX;
            z.mm[3 + d] = LLONG_MIN;
        }
        z.k_in_call = -1;
        z.nkicks_call = nkicks;
        z.q_macro = q_macro;
        z.sort_interval = sort_interval;
        z.nbg = nbg;
        *st = z;
    }
}

cudaError_t launch_state_reset(TrackState *st, int nkicks, double q_macro, int sort_interval,
                               cudaStream_t s, double betagamma) {
    BT_LAUNCH(K_BOX, s, k_state_reset<<<1, 32, 0, s>>>(st, nkicks, q_macro, sort_interval,
                                                        -betagamma));
    return cudaGetLastError();
}

__global__ void k_call_init(TrackState *st, int nkicks, double q_macro, int sort_interval,
                            long long kick0, double nbg, int fused_prologue) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        // a fused prologue deposits into the box of the previous call when one
        // exists and was made for the same beta gamma (its u_z constant)
        st->pro_dep = fused_prologue && st->has_box && st->nbg == nbg ? 1 : 0;
        st->nbg = nbg;
        st->k_in_call = -1;
        st->nkicks_call = nkicks;
        st->q_macro = q_macro;
        st->sort_interval = sort_interval;
        st->kick = kick0;
        st->deposit_gate = st->sort_gate = st->next_gate = 0;
        st->box_hist = nullptr;
        st->box_replay = nullptr;
        st->slot_hist = nullptr;
    }
}

cudaError_t launch_call_init(TrackState *st, int nkicks, double q_macro, int sort_interval,
                             long long kick0, cudaStream_t s, double betagamma,
                             bool fused_prologue) {
    BT_LAUNCH(K_BOX, s, k_call_init<<<1, 32, 0, s>>>(st, nkicks, q_macro, sort_interval, kick0,
                                                      -betagamma, fused_prologue ? 1 : 0));
    return cudaGetLastError();
}

// Zero the deposit accumulators when `gate` is set (or unconditionally).
__global__ void k_zero_acc(unsigned long long *__restrict__ a, unsigned long long *__restrict__ b,
                           long long nodes, const int *gate) {
    if (gate && *gate == 0) return;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        a[i] = 0ull;
        b[i] = 0ull;
    }
}

cudaError_t launch_zero_acc(unsigned long long *a, unsigned long long *b, int nn, const int *gate,
                            cudaStream_t s) {
    const long long nodes = (long long)nn * nn * nn;
    const int blocks = (int)((nodes + TPB - 1) / TPB) < 148 * 8 ? (int)((nodes + TPB - 1) / TPB) : 148 * 8;
    BT_LAUNCH(K_ZERO, s, k_zero_acc<<<blocks, TPB, 0, s>>>(a, b, nodes, gate));
    return cudaGetLastError();
}

// -------------------------------------------------- rho from accumulators

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
    BT_LAUNCH(K_ACC_TO_RHO, s, k_acc_to_rho<<<(int)((nodes + TPB - 1) / TPB), TPB, 0, s>>>(
                                   acc_hi, acc_lo, nodes, q_macro, box, rho));
    return cudaGetLastError();
}

// -------------------------------------------------------------------- field

// Rest-frame field by centred differences on nodes 0..n-1 from phi on nodes
// -1..n, pre-multiplied by the kick factor of the slice:
//   E'_d = c_d (phi(+e_d) - phi(-e_d)),  c_d = -kick_d / (2 h_d),
// so the interpolated value is the momentum change; stored in int64 fixed
// point, E_fix = rint(E'_d 2^e_d) with max |E'_d| 2^e_d in [2^49, 2^50).  Two
// passes over phi (which stays in L2 between them): the per-component max
// |phi(+e_d) - phi(-e_d)| (max |E'_d| = |c_d| times it: rounding is monotone),
// then the conversion.  The FP64 pipe only forms the differences and one
// product per component (c_d 2^e_d in one constant when that is a normal
// double); maxima, rounding to integers and the indexing (n is a power of
// two) run on the integer pipes.
struct FieldCoef {
    double cx, cy, cz;
};

__device__ __forceinline__ FieldCoef field_coef(const Box *box, double kx, double ky, double kz,
                                                const TrackState *st, const MapCoef *maps) {
    if (maps) {  // tracking: kick factors of this kick from the per-call table
        const MapCoef &m = maps[1 + st->k_in_call];
        kx = ky = m.kick_t;
        kz = m.kick_z;
    }
    // -k/(2h) from the box's 1/h: products, not three FP64 divisions per thread
    return FieldCoef{-kx * (0.5 * box->inv_h[0]), -ky * (0.5 * box->inv_h[1]),
                     -kz * (0.5 * box->inv_h[2])};
}

// phi(+e_d) - phi(-e_d) at node idx (x fastest, lg = log2 n).
__device__ __forceinline__ void phi_diffs(const double *__restrict__ phi, int nn, int lg,
                                          long long idx, double &dx, double &dy, double &dz) {
    const int q = nn + 2;
    const int i = (int)(idx & (nn - 1)), j = (int)((idx >> lg) & (nn - 1)), l = (int)(idx >> (2 * lg));
    const long long qq = (long long)q * q;
    const long long c = (l + 1) * qq + (long long)(j + 1) * q + (i + 1);
    dx = __ldg(&phi[c + 1]) - __ldg(&phi[c - 1]);
    dy = __ldg(&phi[c + q]) - __ldg(&phi[c - q]);
    dz = __ldg(&phi[c + qq]) - __ldg(&phi[c - qq]);
}

// rint(v) (round half to even) from the bits, on the integer pipes: the
// FP64 conversion instruction's result for |v| < 2^62; larger values and
// infinities saturate to +-(2^63 - 1), NaN gives 0.
__device__ __forceinline__ long long rint_bits(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -1) return 0;
    if (e > 61) {
        if (e == 1024 && (b & 0xFFFFFFFFFFFFFull)) return 0;
        return (b >> 63) ? -LLONG_MAX : LLONG_MAX;
    }
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned long long r;
    if (e >= 52) {
        r = mant << (e - 52);
    } else {
        const int sh = 52 - e;                       // 1..53
        r = mant >> sh;
        const unsigned long long rem = mant & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        r += (rem > half || (rem == half && (r & 1ull))) ? 1ull : 0ull;
    }
    return (b >> 63) ? -(long long)r : (long long)r;
}

__global__ void k_field(const double *__restrict__ phi, int nn, int lg,
                        unsigned long long *__restrict__ emax) {
    const long long nodes = 1ll << (3 * lg);
    // max |difference| from the bit patterns shifted left by one (the sign
    // falls out; a mask would be compiled as an FP64 absolute value)
    unsigned long long b0 = 0, b1 = 0, b2 = 0;
    auto key = [](double v) { return (unsigned long long)__double_as_longlong(v) << 1; };
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nodes;
         idx += (long long)gridDim.x * blockDim.x) {
        double dx, dy, dz;
        phi_diffs(phi, nn, lg, idx, dx, dy, dz);
        b0 = max(b0, key(dx));
        b1 = max(b1, key(dy));
        b2 = max(b2, key(dz));
    }
    b0 >>= 1;
    b1 >>= 1;
    b2 >>= 1;
    // (NaN bit patterns sort above Inf: a NaN difference makes the max non-finite)
    for (int o = 16; o > 0; o >>= 1) {
        b0 = max(b0, __shfl_xor_sync(0xffffffffu, b0, o));
        b1 = max(b1, __shfl_xor_sync(0xffffffffu, b1, o));
        b2 = max(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    }
    __shared__ unsigned long long sm[3][TPB / 32];
    if ((threadIdx.x & 31) == 0) {
        sm[0][threadIdx.x >> 5] = b0;
        sm[1][threadIdx.x >> 5] = b1;
        sm[2][threadIdx.x >> 5] = b2;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        unsigned long long v = 0;
        for (int w = 0; w < TPB / 32; ++w) v = max(v, sm[threadIdx.x][w]);
        atomicMax(&emax[threadIdx.x], v);
    }
}

// Scale exponent e with max * 2^e in [2^49, 2^50): node values and their
// differences fit the 26-bit-limb interpolation, interpolated values convert
// to double exactly, and the resolution (2^-49 of the largest value) is that
// of a double.
__device__ __forceinline__ int field_exponent(double m) {
    if (!(m > 0.0) || !isfinite(m)) return 0;
    return 49 - ilogb(m);
}

// One component's conversion: c 2^e as one constant when it is a normal
// double (then diff * (c 2^e) = (c diff) 2^e exactly for every value that
// does not round to 0), else the product and a scaling.
struct FieldConv {
    double c, k;
    int e;
    bool fused;
};
__device__ __forceinline__ FieldConv field_conv(double c, unsigned long long maxdiff_bits) {
    FieldConv f;
    f.c = c;
    f.e = field_exponent(fabs(c) * __longlong_as_double((long long)maxdiff_bits));
    f.k = ldexp(c, f.e);
    const unsigned long long kb = abs_bits(f.k);
    f.fused = kb >= 0x0010000000000000ull && kb < 0x7FF0000000000000ull;
    return f;
}
__device__ __forceinline__ long long field_fix(const FieldConv &f, double diff) {
    return rint_bits(f.fused ? diff * f.k : ldexp(f.c * diff, f.e));
}
__device__ __forceinline__ long long field_fix_fused(const FieldConv &f, double diff) {
    return rint_bits(diff * f.k);
}

__global__ void k_efix(const double *__restrict__ phi, int nn, int lg, const Box *box, double kx,
                       double ky, double kz, const unsigned long long *__restrict__ emax,
                       EFix *__restrict__ out, int *__restrict__ escale, const TrackState *st,
                       const MapCoef *maps) {
    // the conversion constants once per block (their FP64 setup per thread
    // had cost as much as the conversions of a thread's nodes)
    __shared__ FieldConv sconv[3];
    if (threadIdx.x < 3) {
        const FieldCoef c = field_coef(box, kx, ky, kz, st, maps);
        const double cd = threadIdx.x == 0 ? c.cx : threadIdx.x == 1 ? c.cy : c.cz;
        sconv[threadIdx.x] = field_conv(cd, emax[threadIdx.x]);
        if (blockIdx.x == 0) escale[threadIdx.x] = sconv[threadIdx.x].e;
    }
    __syncthreads();
    const FieldConv f0 = sconv[0], f1 = sconv[1], f2 = sconv[2];
    const long long nodes = 1ll << (3 * lg);
    // the uniform choice outside the loop (a per-node select would also run
    // the scaling path on the FP64 pipe)
    if (f0.fused && f1.fused && f2.fused) {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
             i += (long long)gridDim.x * blockDim.x) {
            double dx, dy, dz;
            phi_diffs(phi, nn, lg, i, dx, dy, dz);
            out[i] = EFix{field_fix_fused(f0, dx), field_fix_fused(f1, dy), field_fix_fused(f2, dz), 0};
        }
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
             i += (long long)gridDim.x * blockDim.x) {
            double dx, dy, dz;
            phi_diffs(phi, nn, lg, i, dx, dy, dz);
            out[i] = EFix{field_fix(f0, dx), field_fix(f1, dy), field_fix(f2, dz), 0};
        }
    }
}

cudaError_t launch_field(const double *phi, int nn, const Box *box, double kx, double ky,
                         double kz, unsigned long long *emax, EFix *efix, int *escale,
                         cudaStream_t s, const TrackState *st, const MapCoef *maps) {
    const int lg = __builtin_ctz((unsigned)nn);
    const long long nodes = 1ll << (3 * lg);
    cudaError_t e = cudaMemsetAsync(emax, 0, 3 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)((nodes + TPB - 1) / TPB);
    const int fblocks = blocks < 148 * 8 ? blocks : 148 * 8;
    BT_LAUNCH(K_FIELD, s, k_field<<<fblocks, TPB, 0, s>>>(phi, nn, lg, emax));
    BT_LAUNCH(K_EFIX, s, k_efix<<<fblocks, TPB, 0, s>>>(phi, nn, lg, box, kx, ky, kz, emax, efix,
                                                        escale, st, maps));
    return cudaGetLastError();
}

// -------------------------------------------------- fused particle kernel

constexpr int PPT = 4;                 // particles per thread
constexpr int CHUNK = TPB * PPT;       // particles per block
constexpr int TILE_CAP = 3072;         // nodes of the shared-memory deposit tile

struct PartArgs {
    double *x, *px, *y, *py, *t, *pt;
    double *ox, *opx, *oy, *opy, *ot, *opt;   // GATHER output (= input unless out of place)
    int64_t n;
    double nbg;                        // -beta*gamma
    const Box *box;
    int nn;
    const EFix *ef;                    // field in fixed point (GATHER)
    const int *escale;
    MapCoef map;
    unsigned long long *acc_hi, *acc_lo;   // deposit accumulators (DEP)
    TrackState *st;                    // min/max (MM)
    int32_t *status;
    int exact_u;                       // u = (X - lo) * (1/h) instead of one FMA
    int flag_outside;                  // report deposit particles outside the box
    const int *gate;                   // if set and 0, the kernel does nothing
    const int *dep_if;                 // if set and 0, no deposit (the rest runs)
    const MapCoef *maps;               // MAP_TABLE: per-call map table (entry 1 + k)
    const MapCoef *row;                // MAP_TABLE: this kick's entry (set by the kernel)
    const TrackState *dst;             // device-driven: exact_u and k from here
    int shape;                         // particle shape: 1 CIC, 2 TSC
    // cells of the deposit's positions (3 arrays of n, cell_code): DEP
    // stores them when set, a UL gather loads them instead of recomputing
    unsigned long long *cell_out;
    const unsigned long long *cell_in;
};

// A particle's cell (CIC) or nearest node (TSC) and 53-bit offset in one
// dimension as the deposit computed them, with the particle's outside flag:
// outside << 63 | cell << 53 | F (F <= 2^52, cell < 1024).
__device__ __forceinline__ unsigned long long cell_code(int cell, unsigned long long F, bool outside) {
    return ((unsigned long long)outside << 63) | ((unsigned long long)cell << 53) | F;
}

// Node and offset for the TSC shape (particle shape 2): u limited to
// [1/2, n - 3/2], nearest node i = floor(u + 1/2) limited to [1, n-2], and
// G = (u - i + 1/2) 2^52 in [0, 2^52] (so f = u - i = G 2^-52 - 1/2), with
// integer operations only; `outside` as for CIC.
__device__ __forceinline__ void tsc_node(double u, int nn, int &node, unsigned long long &G,
                                         bool &outside) {
    const unsigned long long umax = (unsigned long long)(nn - 1) << 52;
    const unsigned long long b = (unsigned long long)__double_as_longlong(u);
    unsigned long long U = to_fixed52(u);
    outside |= ((b >> 63) && abs_bits(u) > NEG_TOL_BITS) || U > umax + 4503599627ull;
    const unsigned long long ulo = 1ull << 51, uhi = (unsigned long long)(2 * nn - 3) << 51;
    U = U < ulo ? ulo : (U > uhi ? uhi : U);
    const unsigned long long V = U + (1ull << 51);
    unsigned long long i = V >> 52;
    if (i > (unsigned long long)(nn - 2)) i = nn - 2;
    G = V - (i << 52);
    node = (int)i;
}

// TSC weights of nodes i-1, i, i+1 as 52-bit fractions: (1-g)^2/2, the rest,
// g^2/2 (their sum is exactly 2^52).
__device__ __forceinline__ void tsc_weights(unsigned long long G, Frac w[3]) {
    const unsigned long long one = 1ull << 52;
    const unsigned long long wp = mulshr52(split26(G), split26(G)) >> 1;
    const unsigned long long wm = mulshr52(split26(one - G), split26(one - G)) >> 1;
    w[0] = split26(wm);
    w[1] = split26(one - wm - wp);
    w[2] = split26(wp);
}

// (e * W) >> 52 for a signed e (|e| < 2^51) and a fraction W <= 2^52, from
// 26-bit limbs (error below 2 units of the last place).
__device__ __forceinline__ long long mulfrac52(long long e, Frac W) {
    const int eh = (int)(e >> 26);
    const unsigned el = (unsigned)(e & 0x3FFFFFFll);
    const long long hh = mul_wide_s(eh, (int)W.hi);
    const long long mid = mul_wide_s(eh, (int)W.lo) + (long long)mul_wide_u(el, W.hi);
    return hh + (mid >> 26);
}

// u = (X - lo)/h.  For a box whose offset is small against its cell size
// (|lo/h| <= 4096, every ordinary box) one FMA, X*(1/h) - lo/h, is within
// 1e-12 of a cell; a box far from the origin relative to its size (e.g. the
// floored box of a single particle) takes the subtraction first.
bool box_needs_exact_u(const Box &b) { return box_far_offset(b); }


// CIC interpolation of the fixed-point field at a particle in cell (c0, c1,
// c2) with 53-bit offsets G0..G2, in lerp form: along x on the four (y, z)
// edges of the cell, then y, then z; each node's record (x, y, z and a pad
// word) in one 32-byte load.
__device__ __forceinline__ void cic_field(const EFix *__restrict__ ef, int nn, int c0, int c1,
                                          int c2, unsigned long long G0, unsigned long long G1,
                                          unsigned long long G2, long long comp[3]) {
    const Frac F0 = split26(G0), F1 = split26(G1), F2 = split26(G2);
    const EFix *e = &ef[((long long)c2 * nn + c1) * nn + c0];
    const long long ny = nn, nz = (long long)nn * nn;
    long long gxy[2][4], gz[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const EFix *q = e + (k & 1) * ny + (k >> 1) * nz;
        long long x0, y0, z0, x1, y1, z1;
        ld_efix(q, x0, y0, z0);
        ld_efix(q + 1, x1, y1, z1);
        gxy[0][k] = lerp52(x0, x1, F0);
        gxy[1][k] = lerp52(y0, y1, F0);
        gz[k] = lerp52(z0, z1, F0);
    }
    comp[0] = lerp52(lerp52(gxy[0][0], gxy[0][1], F1), lerp52(gxy[0][2], gxy[0][3], F1), F2);
    comp[1] = lerp52(lerp52(gxy[1][0], gxy[1][1], F1), lerp52(gxy[1][2], gxy[1][3], F1), F2);
    comp[2] = lerp52(lerp52(gz[0], gz[1], F1), lerp52(gz[2], gz[3], F1), F2);
}

// A particle's cells and offsets from the deposit's three cell codes, the
// cells limited to the shape's range (as the deposit's are), so that a kick
// halted before any deposit still reads inside the field.
template <int SH>
__device__ __forceinline__ void decode_cells(unsigned long long k0, unsigned long long k1,
                                             unsigned long long k2, int nn, int &c0, int &c1,
                                             int &c2, unsigned long long &G0,
                                             unsigned long long &G1, unsigned long long &G2,
                                             bool &out) {
    constexpr unsigned long long FM = (1ull << 53) - 1;
    constexpr int CLO = SH == 2 ? 1 : 0;
    out = ((k0 | k1 | k2) >> 63) != 0;
    c0 = min(max((int)((k0 >> 53) & 1023), CLO), nn - 2);
    c1 = min(max((int)((k1 >> 53) & 1023), CLO), nn - 2);
    c2 = min(max((int)((k2 >> 53) & 1023), CLO), nn - 2);
    G0 = k0 & FM;
    G1 = k1 & FM;
    G2 = k2 & FM;
}

// GATHER: interpolation of the fixed-point field at the current position
//         (SH 1: CIC in lerp form; SH 2: TSC, separable sums of fixed-point
//         products), kick, then the map (MK) and the store.
// DEP:    deposit of the new position (same box, same shape) into the
//         accumulators, through a shared-memory tile covering the block's
//         nodes when they fit.
// MM:     min/max keys of the new rest-frame positions.
// Without GATHER, a map MK (MAP_TABLE: entry 0 at a call's start) is applied
// and stored before DEP/MM (a tracking call's fused prologue).
// CIC instances fit 64 registers and (with 52 KB of shared memory for DEP) run 4 blocks
// per SM; the CIC gather that loads the deposit's cells fits 48 and runs 5 (its
// field loads are latency-bound); TSC instances and the map-plus-deposit
// prologue with the map table's run-time dispatch keep 3 (they would spill at
// 64); the prologue compiled for one map class fits 64 and runs 4.
template <int MK, bool GATHER, bool DEP, bool MM, int SH, bool UL = false, bool SPREAD = false>
__global__ void __launch_bounds__(TPB, (UL && SH == 1) ? 5 : (SH == 1 && !(DEP && MK == MAP_TABLE)) ? 4 : 3)
    k_particles(PartArgs a) {
    if (a.gate && *a.gate == 0) return;
    if (a.dst) a.exact_u = a.dst->exact_u;
    if constexpr (MK == MAP_TABLE) {
        a.row = a.maps + 1 + a.dst->k_in_call;
        a.map = *a.row;
    }
    extern __shared__ unsigned long long dsm[];
    unsigned long long *sF = dsm;                                // [3][CHUNK] fractions
    int *scell = (int *)(dsm + 3 * CHUNK);                       // [CHUNK] packed cell or -1
    unsigned long long *tile = dsm + 3 * CHUNK + CHUNK / 2;      // [TILE_CAP]
    __shared__ int s_bb[6];
    const int nn = a.nn;
    // u = (X - lo)/h as one FMA per dimension: X * (1/h) - lo/h
    const double ih0 = a.box->inv_h[0], ih1 = a.box->inv_h[1], ih2 = a.box->inv_h[2];
    const double o0 = a.box->off[0], o1 = a.box->off[1], o2 = a.box->off[2];
    const double tz = a.box->tz;
    const double lo0 = a.box->lo[0], lo1 = a.box->lo[1], lo2 = a.box->lo[2];
    int e0 = 0, e1 = 0, e2 = 0;
    if constexpr (GATHER) {
        e0 = a.escale[0];
        e1 = a.escale[1];
        e2 = a.escale[2];
    }
    if (DEP && threadIdx.x < 6) s_bb[threadIdx.x] = threadIdx.x < 3 ? INT_MAX : INT_MIN;
    long long klo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, khi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
    int blo[3] = {INT_MAX, INT_MAX, INT_MAX}, bhi[3] = {INT_MIN, INT_MIN, INT_MIN};
    bool bad = false, outside = false;
    const int64_t base = (int64_t)blockIdx.x * CHUNK;
    {
        // the rows this block reads (its CHUNK particles) into L2 by bulk
        // prefetches, one per row, so that the loads of its later iterations
        // hit L2: the six coordinates where a map is applied or a gather runs
        // (x, y, t only for a deposit alone), and the cell codes a gather reads
        constexpr bool ALL6 = GATHER || MK != MAP_NONE;
        constexpr int NROW = (ALL6 ? 6 : 3) + (GATHER && UL ? 3 : 0);
        if ((DEP || (GATHER && UL)) && threadIdx.x < NROW && base < a.n) {
            const int k = threadIdx.x;
            const void *row;
            if (ALL6 && k < 6)
                row = k == 0 ? (const void *)a.x : k == 1 ? (const void *)a.px
                    : k == 2 ? (const void *)a.y : k == 3 ? (const void *)a.py
                    : k == 4 ? (const void *)a.t : (const void *)a.pt;
            else if (!ALL6)
                row = k == 0 ? (const void *)a.x : k == 1 ? (const void *)a.y : (const void *)a.t;
            else
                row = (const void *)(a.cell_in + (k - 6) * a.n);
            const char *src = (const char *)row + base * 8;
            const unsigned bytes = (unsigned)(min((int64_t)CHUNK, a.n - base) & ~1ll) * 8u;
            if (((uintptr_t)src & 15u) == 0 && bytes)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(src), "r"(bytes)
                             : "memory");
        }
    }
    if (DEP) __syncthreads();
    bool dep_on = DEP;                                  // uniform over the grid
    if constexpr (DEP) dep_on = !a.dep_if || *a.dep_if != 0;
    // u = (X - lo)/h: one FMA with the box's constants, or (far-offset box)
    // the subtraction first; a uniform branch selects one of two compiled
    // copies of the particle loop, so each copy does only its own arithmetic
    auto particle_loop = [&](auto exact_tag) {
        constexpr bool EX = decltype(exact_tag)::value;
        // the deposit alone (CIC) fully unrolled: 0.523 -> 0.507 ms at 2.5e7
        // particles, no spills at 64 registers; the others keep one
        // particle in flight per thread (register budget)
        constexpr int UNR = (DEP && !GATHER && MK == MAP_NONE && SH == 1) ? PPT : 1;
        // UL gather: the next particle's cell codes are loaded one iteration
        // ahead, so that its field loads need not wait for them
        unsigned long long nk0 = 0, nk1 = 0, nk2 = 0;
        if constexpr (GATHER && UL) {
            const int64_t p0 = base + threadIdx.x;
            if (p0 < a.n) {
                nk0 = a.cell_in[p0];
                nk1 = a.cell_in[a.n + p0];
                nk2 = a.cell_in[2 * a.n + p0];
            }
        }
    #pragma unroll UNR
        for (int it = 0; it < PPT; ++it) {
            const int slot = it * TPB + threadIdx.x;
            const int64_t p = base + slot;
            const unsigned long long ck0 = nk0, ck1 = nk1, ck2 = nk2;
            if constexpr (GATHER && UL) {
                const int64_t pn = p + TPB;
                if (it + 1 < PPT && pn < a.n) {
                    nk0 = a.cell_in[pn];
                    nk1 = a.cell_in[a.n + pn];
                    nk2 = a.cell_in[2 * a.n + pn];
                }
            }
            if (DEP) scell[slot] = -1;
            if (p >= a.n) continue;
            double x = a.x[p], y = a.y[p], t = a.t[p];
            if constexpr (GATHER) {
                double px = a.px[p], py = a.py[p], pt = a.pt[p];
                int c0, c1, c2;
                unsigned long long G0, G1, G2;
                bool out0 = false;
                if constexpr (UL) {
                    // the cells the deposit of these positions into this box computed
                    decode_cells<SH>(ck0, ck1, ck2, nn, c0, c1, c2, G0, G1, G2, out0);
                } else {
                    const double u0 = EX ? (x - lo0) * ih0 : fma(x, ih0, o0);
                    const double u1 = EX ? (y - lo1) * ih1 : fma(y, ih1, o1);
                    const double u2 = EX ? (__dmul_rn(a.nbg, t) - lo2) * ih2 : fma(t, tz, o2);
                    if constexpr (SH == 2) {
                        tsc_node(u0, nn, c0, G0, out0);
                        tsc_node(u1, nn, c1, G1, out0);
                        tsc_node(u2, nn, c2, G2, out0);
                    } else {
                        cell_frac(u0, nn, c0, G0, out0);
                        cell_frac(u1, nn, c1, G1, out0);
                        cell_frac(u2, nn, c2, G2, out0);
                    }
                }
                long long comp[3];
                if constexpr (SH == 2) {
                    outside |= out0;
                    Frac wx[3], wy[3], wz[3];
                    tsc_weights(G0, wx);
                    tsc_weights(G1, wy);
                    tsc_weights(G2, wz);
                    // separable: along x on the nine (y, z) lines, then y, then z;
                    // each node record (x, y, z, pad) in one 32-byte load
                    const EFix *e = &a.ef[((long long)(c2 - 1) * nn + (c1 - 1)) * nn + (c0 - 1)];
                    const long long ny = nn, nz = (long long)nn * nn;
                    long long gz[3] = {0, 0, 0};
    #pragma unroll
                    for (int dz = 0; dz < 3; ++dz) {
                        long long gy[3] = {0, 0, 0};
    #pragma unroll
                        for (int dy = 0; dy < 3; ++dy) {
                            const EFix *q = e + dz * nz + dy * ny;
                            long long x0, y0, z0, x1, y1, z1, x2, y2, z2;
                            ld_efix(q, x0, y0, z0);
                            ld_efix(q + 1, x1, y1, z1);
                            ld_efix(q + 2, x2, y2, z2);
                            const long long gxx = mulfrac52(x0, wx[0]) + mulfrac52(x1, wx[1]) +
                                                  mulfrac52(x2, wx[2]);
                            const long long gxy = mulfrac52(y0, wx[0]) + mulfrac52(y1, wx[1]) +
                                                  mulfrac52(y2, wx[2]);
                            const long long gxz = mulfrac52(z0, wx[0]) + mulfrac52(z1, wx[1]) +
                                                  mulfrac52(z2, wx[2]);
                            gy[0] += mulfrac52(gxx, wy[dy]);
                            gy[1] += mulfrac52(gxy, wy[dy]);
                            gy[2] += mulfrac52(gxz, wy[dy]);
                        }
    #pragma unroll
                        for (int cc = 0; cc < 3; ++cc) gz[cc] += mulfrac52(gy[cc], wz[dz]);
                    }
                    comp[0] = gz[0];
                    comp[1] = gz[1];
                    comp[2] = gz[2];
                } else {
                    outside |= out0;
                    cic_field(a.ef, nn, c0, c1, c2, G0, G1, G2, comp);
                }
                const long long ex = comp[0], ey = comp[1], ez = comp[2];
                px += i64_scaled_to_double(ex, e0);
                py += i64_scaled_to_double(ey, e1);
                pt += i64_scaled_to_double(ez, e2);
                if constexpr (MK == MAP_TABLE) apply_map_table(a.map, a.row, x, px, y, py, t, pt);
                else apply_map_k<MK>(a.map, x, px, y, py, t, pt);
                bad |= !finite6(x, px, y, py, t, pt);
                a.ox[p] = x;
                a.opx[p] = px;
                a.oy[p] = y;
                a.opy[p] = py;
                a.ot[p] = t;
                a.opt[p] = pt;
            } else if constexpr (MK != MAP_NONE) {
                double px = a.px[p], py = a.py[p];
                const double pt = a.pt[p];
                if constexpr (MK == MAP_TABLE) apply_map_table(a.map, a.row, x, px, y, py, t, pt);
                else apply_map_k<MK>(a.map, x, px, y, py, t, pt);
                bad |= !finite6(x, px, y, py, t, pt);
                a.ox[p] = x;
                a.opx[p] = px;
                a.oy[p] = y;
                a.opy[p] = py;
                a.ot[p] = t;
            }
            if constexpr (DEP || MM) {
                if constexpr (MM) {
                    const long long k0 = dkey(x), k1 = dkey(y), k2 = dkey(__dmul_rn(a.nbg, t));
                    klo[0] = min(klo[0], k0);
                    khi[0] = max(khi[0], k0);
                    klo[1] = min(klo[1], k1);
                    khi[1] = max(khi[1], k1);
                    klo[2] = min(klo[2], k2);
                    khi[2] = max(khi[2], k2);
                }
                if constexpr (DEP) if (dep_on) {
                    int c0, c1, c2;
                    unsigned long long F0, F1, F2;
                    bool out1 = false;
                    const double u0 = EX ? (x - lo0) * ih0 : fma(x, ih0, o0);
                    const double u1 = EX ? (y - lo1) * ih1 : fma(y, ih1, o1);
                    const double u2 = EX ? (__dmul_rn(a.nbg, t) - lo2) * ih2 : fma(t, tz, o2);
                    if constexpr (SH == 2) {  // nearest node and offset
                        tsc_node(u0, nn, c0, F0, out1);
                        tsc_node(u1, nn, c1, F1, out1);
                        tsc_node(u2, nn, c2, F2, out1);
                    } else {
                        cell_frac(u0, nn, c0, F0, out1);
                        cell_frac(u1, nn, c1, F1, out1);
                        cell_frac(u2, nn, c2, F2, out1);
                    }
                    if (a.cell_out) {
                        a.cell_out[p] = cell_code(c0, F0, out1);
                        a.cell_out[a.n + p] = cell_code(c1, F1, out1);
                        a.cell_out[2 * a.n + p] = cell_code(c2, F2, out1);
                    }
                    if (out1 && a.flag_outside) outside = true;  // box not containing the bunch
                    if (!out1) {  // particles outside are left out: the box rule then regrids
                        sF[slot] = F0;
                        sF[CHUNK + slot] = F1;
                        sF[2 * CHUNK + slot] = F2;
                        scell[slot] = c0 | (c1 << 10) | (c2 << 20);  // n <= 256
                        blo[0] = min(blo[0], c0);
                        bhi[0] = max(bhi[0], c0);
                        blo[1] = min(blo[1], c1);
                        bhi[1] = max(bhi[1], c1);
                        blo[2] = min(blo[2], c2);
                        bhi[2] = max(bhi[2], c2);
                    }
                }
            }
        }
    };
    if (a.exact_u) particle_loop(std::true_type{});
    else particle_loop(std::false_type{});
    if (bad) atomicOr(a.status, ST_NONFINITE);
    if (outside) atomicOr(a.status, ST_OUTSIDE);
    if constexpr (MM) block_keys_commit(klo, khi, a.st);
    if constexpr (DEP) {
        if (!dep_on) return;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int l = __reduce_min_sync(0xffffffffu, blo[d]);
            const int h = __reduce_max_sync(0xffffffffu, bhi[d]);
            if ((threadIdx.x & 31) == 0) {
                atomicMin(&s_bb[d], l);
                atomicMax(&s_bb[3 + d], h);
            }
        }
        __syncthreads();
        if (s_bb[0] == INT_MAX) return;  // nothing to deposit in this block
        // CIC: nodes c..c+1 of the cells c; TSC: nodes c-1..c+1 around the nodes c
        constexpr int LOW = SH == 2 ? 1 : 0, SPAN = SH == 2 ? 3 : 2;
        const int i0 = s_bb[0] - LOW, j0 = s_bb[1] - LOW, l0 = s_bb[2] - LOW;
        const int tx = s_bb[3] - s_bb[0] + SPAN, ty = s_bb[4] - s_bb[1] + SPAN,
                  tz = s_bb[5] - s_bb[2] + SPAN;
        const bool use_tile = (long long)tx * ty * tz <= TILE_CAP;
        const unsigned long long one = 1ull << 52;
        // the tile as two 32-bit words per node (low word, high word): native
        // 32-bit shared atomics, where a 64-bit add would be a compare-and-swap
        // loop that retries on every collision of sorted neighbours; a carry
        // out of the low word goes into the high word.  A block adds at most
        // CHUNK weights below 2^51 to a node, so the high word stays below 2^30.
        unsigned *tlo = (unsigned *)tile, *thi = tlo + TILE_CAP;
        if (use_tile) {
            for (int i = threadIdx.x; i < tx * ty * tz; i += TPB) tlo[i] = thi[i] = 0u;
            __syncthreads();
        }
#pragma unroll 1
        for (int it = 0; it < PPT; ++it) {
            // SPREAD (particles ordered by cell): consecutive lanes take slots
            // 37 apart (37 is odd: a permutation of the block's CHUNK slots), so
            // that a warp's atomics go to the nodes of many cells instead of
            // colliding on the few cells of 32 consecutive particles
            const int slot = SPREAD ? ((it * TPB + threadIdx.x) * 37) & (CHUNK - 1)
                                    : it * TPB + threadIdx.x;
            const int cell = scell[slot];
            if (cell < 0) continue;
            const unsigned long long F0 = sF[slot], F1 = sF[CHUNK + slot], F2 = sF[2 * CHUNK + slot];
            const int c0 = cell & 1023, c1 = (cell >> 10) & 1023, c2 = cell >> 20;
            // tile index of the particle's first node; the others are fixed offsets
            const int lb = ((c2 - LOW - l0) * ty + (c1 - LOW - j0)) * tx + (c0 - LOW - i0);
            Frac wx[SPAN], wy[SPAN], wz[SPAN];
            unsigned long long wc[8];
            if constexpr (SH == 2) {
                tsc_weights(F0, wx);
                tsc_weights(F1, wy);
                tsc_weights(F2, wz);
            } else {
                cic_weights(F0, F1, F2, wc);
            }
#pragma unroll
            for (int dz = 0; dz < SPAN; ++dz)
#pragma unroll
                for (int dy = 0; dy < SPAN; ++dy) {
                    Frac wyz{};
                    if constexpr (SH == 2) wyz = split26(mulshr52(wy[dy], wz[dz]));
#pragma unroll
                    for (int dx = 0; dx < SPAN; ++dx) {
                        // 51-bit weight
                        const unsigned long long v = SH == 2 ? mulshr52(wx[dx], wyz) >> 1
                                                             : wc[(dz * 2 + dy) * 2 + dx];
                        const int ni = c0 + dx - LOW, nj = c1 + dy - LOW, nl = c2 + dz - LOW;
                        if (use_tile) {
                            const int li = lb + (dz * ty + dy) * tx + dx;
                            const unsigned lo = (unsigned)v;
                            const unsigned old = atomicAdd(&tlo[li], lo);
                            atomicAdd(&thi[li], (unsigned)(v >> 32) + (old + lo < old ? 1u : 0u));
                        } else {
                            const long long node = ((long long)nl * nn + nj) * nn + ni;
                            atomicAdd(&a.acc_hi[node], v >> DEP_SPLIT);
                            atomicAdd(&a.acc_lo[node], v & ((1ull << DEP_SPLIT) - 1));
                        }
                    }
                }
        }
        if (use_tile) {
            __syncthreads();
            // tile index i = (ll ty + jj) tx + ii, stepped by TPB with carries
            // (three divisions per thread instead of three per node)
            const int sa = TPB % tx, sb = (TPB / tx) % ty, sc = TPB / (tx * ty);
            int ii = threadIdx.x % tx, jj = (threadIdx.x / tx) % ty, ll = threadIdx.x / (tx * ty);
            for (int i = threadIdx.x; i < tx * ty * tz; i += TPB) {
                const unsigned long long v = ((unsigned long long)thi[i] << 32) + tlo[i];
                if (v != 0ull) {
                    const long long node = ((long long)(l0 + ll) * nn + (j0 + jj)) * nn + (i0 + ii);
                    atomicAdd(&a.acc_hi[node], v >> DEP_SPLIT);
                    atomicAdd(&a.acc_lo[node], v & ((1ull << DEP_SPLIT) - 1));
                }
                ii += sa;
                int carry = ii >= tx;
                ii -= carry ? tx : 0;
                jj += sb + carry;
                carry = jj >= ty;
                jj -= carry ? ty : 0;
                ll += sc + carry;
            }
        }
    }
}

static size_t particles_smem(bool dep) {
    return dep ? (size_t)(3 * CHUNK + CHUNK / 2 + TILE_CAP) * sizeof(unsigned long long) : 0;
}

template <int MK, bool G, bool D, bool M, int SH, bool UL = false, bool SPREAD = false>
static cudaError_t launch_pk_sh(const PartArgs &a, cudaStream_t s, int kid) {
    const size_t sm = particles_smem(D);
    if (D)
        cudaFuncSetAttribute(k_particles<MK, G, D, M, SH, UL, SPREAD>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const unsigned blocks = (unsigned)((a.n + CHUNK - 1) / CHUNK);
    BT_LAUNCH(kid, s, k_particles<MK, G, D, M, SH, UL, SPREAD><<<blocks, TPB, sm, s>>>(a));
    return cudaGetLastError();
}

// The deposit of particles ordered by cell (CIC; with or without the min/max
// keys): the tile deposit with its atomics spread over the block's particles.
static cudaError_t launch_deposit_spread(const PartArgs &a, bool mm, cudaStream_t s, int kid) {
    return mm ? launch_pk_sh<MAP_NONE, false, true, true, 1, false, true>(a, s, kid)
              : launch_pk_sh<MAP_NONE, false, true, false, 1, false, true>(a, s, kid);
}

template <int MK, bool G, bool D, bool M, bool UL = false>
static cudaError_t launch_pk(const PartArgs &a, cudaStream_t s, int kid) {
    return a.shape == 2 ? launch_pk_sh<MK, G, D, M, 2, UL>(a, s, kid)
                        : launch_pk_sh<MK, G, D, M, 1, UL>(a, s, kid);
}

static PartArgs part_args(double *const c[6], int64_t n, double betagamma, const Box *box, int nn,
                          int shape) {
    PartArgs a{};
    a.shape = shape;
    a.x = c[0];
    a.px = c[1];
    a.y = c[2];
    a.py = c[3];
    a.t = c[4];
    a.pt = c[5];
    a.ox = c[0];
    a.opx = c[1];
    a.oy = c[2];
    a.opy = c[3];
    a.ot = c[4];
    a.opt = c[5];
    a.n = n;
    a.nbg = -betagamma;
    a.box = box;
    a.nn = nn;
    return a;
}

cudaError_t launch_kick_push_deposit(double *const c[6], int64_t n, double betagamma,
                                     const Box *box, const Box &box_host, int nn, const EFix *ef,
                                     const int *escale, const MapCoef *map_host, bool deposit,
                                     unsigned long long *acc_hi, unsigned long long *acc_lo,
                                     TrackState *st, int32_t *status, cudaStream_t s, int shape) {
    if (n <= 0) return cudaSuccess;
    PartArgs a = part_args(c, n, betagamma, box, nn, shape);
    a.exact_u = box_needs_exact_u(box_host) ? 1 : 0;
    a.ef = ef;
    a.escale = escale;
    a.acc_hi = acc_hi;
    a.acc_lo = acc_lo;
    a.st = st;
    a.status = status;
    const int mk = map_host ? map_kind(*map_host) : MAP_NONE;
    if (map_host) a.map = *map_host;
    // gather + kick + map (no shared memory, 3 blocks/SM) ...
    cudaError_t e;
    switch (mk) {
        case MAP_NONE: e = launch_pk<MAP_NONE, true, false, false>(a, s, K_GATHER); break;
        case MAP_DRIFT: e = launch_pk<MAP_DRIFT, true, false, false>(a, s, K_GATHER); break;
        case MAP_QUAD: e = launch_pk<MAP_QUAD, true, false, false>(a, s, K_GATHER); break;
        case MAP_BEND: e = launch_pk<MAP_BEND, true, false, false>(a, s, K_GATHER); break;
        default: e = launch_pk<MAP_GENERAL, true, false, false>(a, s, K_GATHER); break;
    }
    if (e != cudaSuccess || !deposit) return e;
    // ... then the next kick's deposit and the min/max from the new x, y, t
    return launch_pk<MAP_NONE, false, true, true>(a, s, K_DEPOSIT);
}

// Device-driven tracking kick: A with the map of this kick from the table
// (part & 1), then, if a next kick follows, the zeroing of the accumulators
// and B (part & 2).
cudaError_t launch_track_particles(double *const c[6], int64_t n, double betagamma,
                                   const Box *box, int nn, const EFix *ef, const int *escale,
                                   const MapCoef *maps, unsigned long long *acc_hi,
                                   unsigned long long *acc_lo, TrackState *st, int32_t *status,
                                   cudaStream_t s, int part, int shape, unsigned long long *cells,
                                   bool spread) {
    if (n <= 0) {
        // no particles (a rank of a sharded run): the next kick's accumulators
        // must still start from zero
        return (part & 2) ? launch_zero_acc(acc_hi, acc_lo, nn, &st->next_gate, s) : cudaSuccess;
    }
    PartArgs a = part_args(c, n, betagamma, box, nn, shape);
    a.ef = ef;
    a.escale = escale;
    a.acc_hi = acc_hi;
    a.acc_lo = acc_lo;
    a.st = st;
    a.status = status;
    a.maps = maps;
    a.dst = st;
    cudaError_t e = cudaSuccess;
    if (part & 1) {
        if (cells) {
            a.cell_in = cells;   // the cells this kick's deposit computed
            e = launch_pk<MAP_TABLE, true, false, false, true>(a, s, K_GATHER);
            a.cell_in = nullptr;
        } else {
            e = launch_pk<MAP_TABLE, true, false, false>(a, s, K_GATHER);
        }
    }
    if (e != cudaSuccess || !(part & 2)) return e;
    e = launch_zero_acc(acc_hi, acc_lo, nn, &st->next_gate, s);
    if (e != cudaSuccess) return e;
    a.gate = &st->next_gate;
    a.cell_out = cells;
    if (spread && shape == 1) return launch_deposit_spread(a, true, s, K_DEPOSIT);
    return launch_pk<MAP_NONE, false, true, true>(a, s, K_DEPOSIT);
}

// Out-of-place device-driven kick (differentiation recompute): A reads cin and
// writes cout, then (gated on the next kick) B deposits cout's positions.
cudaError_t launch_track_particles_oop(double *const cin[6], double *const cout[6], int64_t n,
                                       double betagamma, const Box *box, int nn, const EFix *ef,
                                       const int *escale, const MapCoef *maps,
                                       unsigned long long *acc_hi, unsigned long long *acc_lo,
                                       TrackState *st, int32_t *status, cudaStream_t s, int shape) {
    if (n <= 0) return cudaSuccess;
    PartArgs a = part_args(cin, n, betagamma, box, nn, shape);
    a.ox = cout[0];
    a.opx = cout[1];
    a.oy = cout[2];
    a.opy = cout[3];
    a.ot = cout[4];
    a.opt = cout[5];
    a.ef = ef;
    a.escale = escale;
    a.st = st;
    a.status = status;
    a.maps = maps;
    a.dst = st;
    cudaError_t e = launch_pk<MAP_TABLE, true, false, false>(a, s, K_GATHER);
    if (e != cudaSuccess) return e;
    e = launch_zero_acc(acc_hi, acc_lo, nn, &st->next_gate, s);
    if (e != cudaSuccess) return e;
    PartArgs b = part_args(cout, n, betagamma, box, nn, shape);
    b.acc_hi = acc_hi;
    b.acc_lo = acc_lo;
    b.st = st;
    b.status = status;
    b.dst = st;
    b.gate = &st->next_gate;
    return launch_pk<MAP_NONE, false, true, true>(b, s, K_DEPOSIT);
}

// A tracking call's prologue in one pass: table entry 0 (the first half map),
// the min/max keys of the new positions, and, when the state kept a box from
// the previous call (pro_dep, set by the call init), the first kick's deposit
// into that box; the box rule then deposits again only if it regrids.
cudaError_t launch_track_prologue(double *const c[6], int64_t n, double betagamma, const Box *box,
                                  int nn, const MapCoef *maps, unsigned long long *acc_hi,
                                  unsigned long long *acc_lo, TrackState *st, int32_t *status,
                                  cudaStream_t s, int shape, unsigned long long *cells,
                                  const MapCoef *map0) {
    cudaError_t e = launch_zero_acc(acc_hi, acc_lo, nn, &st->pro_dep, s);
    if (e != cudaSuccess || n <= 0) return e;
    PartArgs a = part_args(c, n, betagamma, box, nn, shape);
    a.maps = maps;
    a.dst = st;
    a.st = st;
    a.acc_hi = acc_hi;
    a.acc_lo = acc_lo;
    a.status = status;
    a.dep_if = &st->pro_dep;
    a.cell_out = cells;
    // with the host's copy of table entry 0, a kernel compiled for its map
    // class (by value, fewer registers than the table's run-time dispatch)
    const int k0 = map0 ? (int)map0->kind : -1;
    if (k0 == MAP_DRIFT || k0 == MAP_QUAD || k0 == MAP_GENERAL || k0 == MAP_BEND) a.map = *map0;
    switch (k0) {
        case MAP_DRIFT: return launch_pk<MAP_DRIFT, false, true, true>(a, s, K_PUSH);
        case MAP_QUAD: return launch_pk<MAP_QUAD, false, true, true>(a, s, K_PUSH);
        case MAP_GENERAL: return launch_pk<MAP_GENERAL, false, true, true>(a, s, K_PUSH);
        case MAP_BEND: return launch_pk<MAP_BEND, false, true, true>(a, s, K_PUSH);
        default: return launch_pk<MAP_TABLE, false, true, true>(a, s, K_PUSH);
    }
}

// Device-driven deposit of the current positions when the box rule asks for it.
cudaError_t launch_track_deposit(double *const c[6], int64_t n, double betagamma, const Box *box,
                                 int nn, unsigned long long *acc_hi, unsigned long long *acc_lo,
                                 TrackState *st, int32_t *status, cudaStream_t s, int shape,
                                 unsigned long long *cells, bool spread) {
    cudaError_t e = launch_zero_acc(acc_hi, acc_lo, nn, &st->deposit_gate, s);
    if (e != cudaSuccess || n <= 0) return e;
    PartArgs a = part_args(c, n, betagamma, box, nn, shape);
    a.acc_hi = acc_hi;
    a.acc_lo = acc_lo;
    a.status = status;
    a.gate = &st->deposit_gate;
    a.dst = st;
    a.flag_outside = 1;
    a.cell_out = cells;
    if (spread && shape == 1) return launch_deposit_spread(a, false, s, K_REDEPOSIT);
    return launch_pk<MAP_NONE, false, true, false>(a, s, K_REDEPOSIT);
}

// Charge deposition alone (Listing 1 particle shape 1 = CIC): node weights
// (1-f, f) per dimension as unsigned fixed-point products (52-bit fractions,
// 51-bit result), summed with integer atomics, so the result does not depend
// on particle order.  Particles outside the box are left out and flagged.
cudaError_t launch_deposit(double *const c[6], int64_t n, double betagamma, const Box *box,
                           const Box &box_host, int nn, unsigned long long *acc_hi,
                           unsigned long long *acc_lo, int32_t *status, cudaStream_t s, int shape) {
    size_t nodes = (size_t)nn * nn * nn;
    cudaError_t e = cudaMemsetAsync(acc_hi, 0, nodes * 8, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(acc_lo, 0, nodes * 8, s);
    if (e != cudaSuccess) return e;
    if (n <= 0) return cudaSuccess;
    PartArgs a = part_args(c, n, betagamma, box, nn, shape);
    a.acc_hi = acc_hi;
    a.acc_lo = acc_lo;
    a.status = status;
    a.exact_u = box_needs_exact_u(box_host) ? 1 : 0;
    a.flag_outside = 1;
    return launch_pk<MAP_NONE, false, true, false>(a, s, K_DEPOSIT);
}

}  // namespace bt
