// Open-boundary Poisson solve on the doubled (Hockney) grid with hand-written
// shared-memory FFTs.
//
// Paper anchor (arXiv:2208.02382, Model Assumptions): the Poisson equation is
// solved in the bunch rest frame with open boundaries.  Reading: phi = G (*) rho
// as an aperiodic convolution, computed as a circular one on the zero-padded
// (2n)^3 grid; the doubled Green's function holds offset k for k <= n and
// k - 2n above (G is even: entry k is G(min(k, 2n-k)); offset +-n carries the
// true value), so phi is exact on nodes -1..n.
//
// Design (two kinds of passes: FP64 for the Green's function spectrum and the
// explicit bx_solve, as few floating-point operations as the transform allows
// since FP64 issue is scarce on this GPU; block floating point on int64 for
// the tracking solve, on the integer pipes, where the passes are bound by
// latency rather than by any pipe):
//  * real-to-complex along x with two real rows packed into one complex line
//    (a + i b) and separated afterwards by Hermitian symmetry; only kx = 0..n
//    is kept from then on;
//  * pruning: the forward passes skip the all-zero rows and planes of the
//    padded rho (x: n^2 of 4n^2 rows; y: n of 2n planes) and read each line's
//    zero upper half as zeros; the inverse passes only produce the n+2 planes,
//    rows and points that hold nodes -1..n;
//  * the z pass is fused: forward transform, multiply by the real spectrum of
//    G (stored as its even octant), inverse transform, one load and one store;
//  * each line transform is a mixed-radix Stockham FFT: a team of T threads
//    holds the line in registers, applies radix-4/8/16 DFT codelets with
//    twiddles exp(-+2 pi i j/m) from a shared-memory table (built once with
//    sincospi), and exchanges values through its own shared-memory line buffer
//    between radix steps; a team of at most 32 threads (lines of up to 256
//    points) synchronises with a warp barrier only, so the block's lines run
//    independently; a team's reductions (the block-floating-point exponent
//    maximum and L1 norm of its line) are warp redux instructions for a team of
//    one warp and shuffle trees for smaller teams.
#include <algorithm>
#include <climits>

#include "common.cuh"

namespace bt {

// ----------------------------------------------------------------- complex

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 w) {
    return make_double2(fma(a.x, w.x, -a.y * w.y), fma(a.x, w.y, a.y * w.x));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ double2 rot90(double2 a) {
    return INV ? make_double2(-a.y, a.x) : make_double2(a.y, -a.x);
}

// int64 fixed-point complex values (the tracking solve): sums are exact, a
// product by a constant or twiddle f in [-1, 1] (Q63: f 2^63) is
// floor(a f / 2^63) from the high half of one 64x64-bit product (|a| < 2^62).
__device__ __forceinline__ long long mulq(long long a, long long f) {
    return __mul64hi((long long)((unsigned long long)a << 1), f);
}
__device__ __forceinline__ long long q63(double c) { return (long long)(c * 0x1p63); }  // |c| < 1
__device__ __forceinline__ longlong2 cadd(longlong2 a, longlong2 b) { return make_longlong2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ longlong2 csub(longlong2 a, longlong2 b) { return make_longlong2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ longlong2 cmul(longlong2 a, longlong2 w) {
    return make_longlong2(mulq(a.x, w.x) - mulq(a.y, w.y), mulq(a.x, w.y) + mulq(a.y, w.x));
}
template <bool INV>
__device__ __forceinline__ longlong2 rot90(longlong2 a) {
    return INV ? make_longlong2(-a.y, a.x) : make_longlong2(a.y, -a.x);
}

constexpr double RS2 = 0.70710678118654752440;   // sqrt(2)/2
constexpr double C16 = 0.92387953251128675613;   // cos(pi/8)
constexpr double T16 = 0.41421356237309504880;   // tan(pi/8) = sqrt(2) - 1

// ---------------------------------------------------------------- codelets
// In-place DFT of R values in registers, natural order in and out:
// y_q = sum_m x_m exp(-+ 2 pi i m q / R)  (radix-2 decimation in time).
// The last butterfly layer takes each twiddle w = f (a + i b) with one real
// factor f pulled out, so the twiddle and the butterfly e +- w o cost six
// FP64 instructions (two for the rotation, four FMAs) instead of eight.

// lo, hi = e +- f r
__device__ __forceinline__ void bfly_f(double2 e, double2 r, double f, double2 &lo, double2 &hi) {
    lo = make_double2(fma(r.x, f, e.x), fma(r.y, f, e.y));
    hi = make_double2(fma(-r.x, f, e.x), fma(-r.y, f, e.y));
}

// w = exp(-+ i pi/4) = (1 -+ i)/sqrt2: w o = RS2 (o.x +- o.y, o.y -+ o.x)
template <bool INV>
__device__ __forceinline__ void bfly_w8_1(double2 e, double2 o, double2 &lo, double2 &hi) {
    const double2 r = INV ? make_double2(o.x - o.y, o.x + o.y) : make_double2(o.x + o.y, o.y - o.x);
    bfly_f(e, r, RS2, lo, hi);
}
// w = exp(-+ 3 i pi/4) = (-1 -+ i)/sqrt2
template <bool INV>
__device__ __forceinline__ void bfly_w8_3(double2 e, double2 o, double2 &lo, double2 &hi) {
    const double2 r = INV ? make_double2(-(o.x + o.y), o.x - o.y) : make_double2(o.y - o.x, -(o.x + o.y));
    bfly_f(e, r, RS2, lo, hi);
}
// w = c (1 + i t): w o = c (o.x - t o.y, o.y + t o.x)
__device__ __forceinline__ void bfly_ct(double2 e, double2 o, double c, double t, double2 &lo, double2 &hi) {
    bfly_f(e, make_double2(fma(-o.y, t, o.x), fma(o.x, t, o.y)), c, lo, hi);
}
// w = s (t + i): w o = s (t o.x - o.y, o.x + t o.y)
__device__ __forceinline__ void bfly_st(double2 e, double2 o, double s, double t, double2 &lo, double2 &hi) {
    bfly_f(e, make_double2(fma(o.x, t, -o.y), fma(o.y, t, o.x)), s, lo, hi);
}

// The same butterflies on fixed-point values (the real factor f and t as
// Q63 constants, folded at compile time).
__device__ __forceinline__ void bfly_f(longlong2 e, longlong2 r, double f, longlong2 &lo, longlong2 &hi) {
    const long long fq = q63(f);
    const longlong2 fr = make_longlong2(mulq(r.x, fq), mulq(r.y, fq));
    lo = cadd(e, fr);
    hi = csub(e, fr);
}
template <bool INV>
__device__ __forceinline__ void bfly_w8_1(longlong2 e, longlong2 o, longlong2 &lo, longlong2 &hi) {
    const longlong2 r = INV ? make_longlong2(o.x - o.y, o.x + o.y) : make_longlong2(o.x + o.y, o.y - o.x);
    bfly_f(e, r, RS2, lo, hi);
}
template <bool INV>
__device__ __forceinline__ void bfly_w8_3(longlong2 e, longlong2 o, longlong2 &lo, longlong2 &hi) {
    const longlong2 r = INV ? make_longlong2(-(o.x + o.y), o.x - o.y) : make_longlong2(o.y - o.x, -(o.x + o.y));
    bfly_f(e, r, RS2, lo, hi);
}
__device__ __forceinline__ void bfly_ct(longlong2 e, longlong2 o, double c, double t, longlong2 &lo, longlong2 &hi) {
    const long long tq = q63(t);
    bfly_f(e, make_longlong2(o.x - mulq(o.y, tq), o.y + mulq(o.x, tq)), c, lo, hi);
}
__device__ __forceinline__ void bfly_st(longlong2 e, longlong2 o, double s, double t, longlong2 &lo, longlong2 &hi) {
    const long long tq = q63(t);
    bfly_f(e, make_longlong2(mulq(o.x, tq) - o.y, mulq(o.y, tq) + o.x), s, lo, hi);
}

// DFT-4 of (v0, v1, v2, v3); HALF: v2 = v3 = 0 (not read).
template <bool INV, bool HALF, class C>
__device__ __forceinline__ void dft4(C *v) {
    if constexpr (HALF) {
        const C a = v[0], b = v[1], rb = rot90<INV>(b);
        v[0] = cadd(a, b);
        v[1] = cadd(a, rb);
        v[2] = csub(a, b);
        v[3] = csub(a, rb);
    } else {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
}

// DFT-8; HALF: v4..v7 = 0 (not read).
template <bool INV, bool HALF, class C>
__device__ __forceinline__ void dft8(C *v) {
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV, HALF>(e);
    dft4<INV, HALF>(o);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    bfly_w8_1<INV>(e[1], o[1], v[1], v[5]);
    const C r2 = rot90<INV>(o[2]);
    v[2] = cadd(e[2], r2);
    v[6] = csub(e[2], r2);
    bfly_w8_3<INV>(e[3], o[3], v[3], v[7]);
}

// DFT-16; HALF: v8..v15 = 0 (not read).  The twiddles exp(-+ 2 pi i q/16)
// (sg = -1 forward, +1 inverse; S16 = sin(pi/8) = C16 T16) are written as
// C16 (1 + i t) or sg C16 (t + i) with t = +-T16, as RS2 (+-1 +- i), or +-i.
template <bool INV, bool HALF, class C>
__device__ __forceinline__ void dft16(C *v) {
    C e[8], o[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        e[m] = v[2 * m];
        o[m] = v[2 * m + 1];
    }
    dft8<INV, HALF>(e);
    dft8<INV, HALF>(o);
    const double sg = INV ? 1.0 : -1.0;
    v[0] = cadd(e[0], o[0]);
    v[8] = csub(e[0], o[0]);
    bfly_ct(e[1], o[1], C16, sg * T16, v[1], v[9]);            // (C16, sg S16)
    bfly_w8_1<INV>(e[2], o[2], v[2], v[10]);
    bfly_st(e[3], o[3], sg * C16, sg * T16, v[3], v[11]);      // (S16, sg C16)
    const C r4 = rot90<INV>(o[4]);
    v[4] = cadd(e[4], r4);
    v[12] = csub(e[4], r4);
    bfly_st(e[5], o[5], sg * C16, -sg * T16, v[5], v[13]);     // (-S16, sg C16)
    bfly_w8_3<INV>(e[6], o[6], v[6], v[14]);
    bfly_ct(e[7], o[7], -C16, -sg * T16, v[7], v[15]);         // (-C16, sg S16)
}

template <int R, bool INV, bool HALF = false, class C>
__device__ __forceinline__ void dft(C *v) {
    if constexpr (R == 4) dft4<INV, HALF>(v);
    else if constexpr (R == 8) dft8<INV, HALF>(v);
    else dft16<INV, HALF>(v);
}

// ------------------------------------------------------------- line shapes
// Radix sequence (R0, R1[, R2]) and team size T (threads per line) for line
// length M; every step gives each thread M/T values.
template <int M> struct Shape;
template <> struct Shape<16> { static constexpr int S = 2, R0 = 4, R1 = 4, R2 = 1, T = 4; };
template <> struct Shape<32> { static constexpr int S = 2, R0 = 8, R1 = 4, R2 = 1, T = 4; };
template <> struct Shape<64> { static constexpr int S = 2, R0 = 8, R1 = 8, R2 = 1, T = 8; };
template <> struct Shape<128> { static constexpr int S = 3, R0 = 8, R1 = 4, R2 = 4, T = 16; };
template <> struct Shape<256> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 4, T = 32; };
template <> struct Shape<512> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 8, T = 64; };

constexpr int FFT_TPB = 256;

// Line buffers in shared memory hold one 16-byte pad slot per 16 elements:
// the first radix step stores element R0 t + q from thread t (R0 = 8 or 16), a
// stride that without the pads would put most lanes of a warp on the same banks.
__device__ __forceinline__ int sp(int i) { return i + (i >> 4); }
template <int M>
constexpr int kLineStride = M + M / 16;   // elements per padded line buffer

// One Stockham radix step on values held in registers.  Thread t of the team
// holds units u = t + j*T (j < U = (M/R)/T); unit u's inputs are the line
// elements u + m*(M/R), in v[j*R + m].  Twiddles W_{L R}^{k m} (k = u mod L)
// are applied before the radix-R DFT; output q of unit u belongs at line
// position (u-k)*R + q*L + k.
template <int M, int R, int L, bool INV, bool HALF = false, class C>
__device__ __forceinline__ void step_regs(C *v, int t, const C *__restrict__ tw) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j) {
        C *x = v + j * R;
        if constexpr (L > 1) {
            const int u = t + j * T, k = u % L;
#pragma unroll
            for (int m = 1; m < R; ++m) {
                C w = tw[(k * m) * (M / (L * R))];
                if (INV) w.y = -w.y;
                x[m] = cmul(x[m], w);
            }
        }
        dft<R, INV, HALF>(x);
    }
}

template <int M, int R, int L, class C>
__device__ __forceinline__ void store_step(const C *v, C *s, int t) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const int u = t + j * T, k = u % L;
#pragma unroll
        for (int q = 0; q < R; ++q) s[sp((u - k) * R + q * L + k)] = v[j * R + q];
    }
}

template <int M, int R, class C>
__device__ __forceinline__ void load_step(C *v, const C *s, int t) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j)
#pragma unroll
        for (int m = 0; m < R; ++m) v[j * R + m] = s[sp((t + j * T) + m * (M / R))];
}

// Line element held in register slot (j, m) before the first step.
template <int M>
__device__ __forceinline__ int first_index(int t, int j, int m) {
    constexpr int R = Shape<M>::R0, T = Shape<M>::T;
    return (t + j * T) + m * (M / R);
}

// Barrier between the exchanges of one line team: a team of at most 32
// threads lies within one warp and owns its line buffer, so the warp barrier
// suffices and the block's other lines run on independently; wider teams (512-
// point lines, two warps) synchronise the block.
template <int M>
__device__ __forceinline__ void team_sync() {
    if constexpr (Shape<M>::T <= 32) __syncwarp();
    else __syncthreads();
}

// Full line transform: `v` holds the first step's inputs (first_index order);
// the result (natural order) is left in the team's shared line `s`.  Every
// thread of the block calls this (it synchronises the block).  HALF: the
// line's upper half (elements M/2..M-1) is zero; these are exactly the inputs
// m >= R0/2 of every first-step DFT (element u + m M/R0 with u < M/R0), which
// the half codelets neither read nor add.
template <int M, bool INV, bool HALF = false, class C>
__device__ __forceinline__ void line_fft(C *v, C *s, int t, const C *tw) {
    using SH = Shape<M>;
    constexpr int R0 = SH::R0, R1 = SH::R1, R2 = SH::R2;
    step_regs<M, R0, 1, INV, HALF>(v, t, tw);
    store_step<M, R0, 1>(v, s, t);
    team_sync<M>();
    load_step<M, R1>(v, s, t);
    team_sync<M>();
    step_regs<M, R1, R0, INV>(v, t, tw);
    store_step<M, R1, R0>(v, s, t);
    if constexpr (SH::S == 3) {
        team_sync<M>();
        load_step<M, R2>(v, s, t);
        team_sync<M>();
        step_regs<M, R2, R0 * R1, INV>(v, t, tw);
        store_step<M, R2, R0 * R1>(v, s, t);
    }
    team_sync<M>();
}

template <int M, class C>
__device__ __forceinline__ void load_twiddles(C *stw, const C *__restrict__ tw) {
    for (int i = threadIdx.x; i < M; i += blockDim.x) stw[i] = tw[i];
}

// ------------------------------------------------------------- pass kernels
//
// Spectrum layouts (P = n+1 x-frequencies, row pitch P):
//   S1[z][y][kx]   z < n, y < n           (after the x pass)
//   S2[z][ky][kx]  z < n, ky < m          (after the y pass)
//   S3[zz][ky][kx] zz < n+2 (z = zz-1 mod m), ky < m   (after the fused z pass)
//   S4[zz][yy][kx] zz, yy < n+2           (after the inverse y pass)
// Green's spectrum: Gh[kz][ky][kx], kx, ky, kz <= n (the even octant).

// Source of the x pass: a cube of doubles (rho, or the adjoint's source), or
// the even extension of the Green's function octant table (full m^3 input,
// for its spectrum).  (The tracking solve from the deposit accumulators runs
// in block floating point, below.)
enum XSource { SRC_RHO = 0, SRC_GREEN = 2 };

struct XIn {
    const double *rho;
    const double *g;
};

template <int M, int SRC>
__device__ __forceinline__ double x_value(const XIn &in, int n, int nin, int x, int y, int z) {
    if constexpr (SRC == SRC_GREEN) {
        const int a = min(x, M - x), b = min(y, M - y), c = min(z, M - z), q = n + 1;
        return in.g[((long long)c * q + b) * q + a];
    } else {
        if (x >= nin) return 0.0;
        return in.rho[((long long)z * nin + y) * nin + x];
    }
}

// x pass (forward, real to complex).  Rows (y, y+1) of plane z become one
// complex line a + i b; after the transform A_k = (Z_k + conj Z_{m-k})/2 and
// B_k = (Z_k - conj Z_{m-k})/(2i), k = 0..n.  ny, nz rows/planes are read
// (nin, nin for a source cube of nin^3 nodes: n for rho, n+2 for the adjoint
// source on nodes -1..n; m, m for the Green's function).
// Output out[(z*ny + y)*P + k].
template <int M, int SRC>
__global__ void __launch_bounds__(FFT_TPB) k_fft_x_fwd(XIn in, int n, int ny, int nz,
                                                       const double2 *__restrict__ tw,
                                                       double2 *__restrict__ out,
                                                       const int *gate) {
    if (gate && *gate == 0) return;
    const int nin = ny;
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    extern __shared__ double2 smem[];
    double2 *stw = smem, *sl = smem + M;
    load_twiddles<M>(stw, tw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const long long pairs = (long long)(ny / 2) * nz;
    const long long pr = (long long)blockIdx.x * LPB + team;
    const bool live = pr < pairs;
    const int z = live ? (int)(pr / (ny / 2)) : 0, y = live ? (int)(pr % (ny / 2)) * 2 : 0;
    __syncthreads();
    double2 v[V];
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m);
            v[j * R0 + m] = live ? make_double2(x_value<M, SRC>(in, n, nin, e, y, z),
                                                x_value<M, SRC>(in, n, nin, e, y + 1, z))
                                 : make_double2(0.0, 0.0);
        }
    double2 *s = sl + team * kLineStride<M>;
    if (SRC != SRC_GREEN && 2 * nin == M) line_fft<M, false, true>(v, s, t, stw);  // rows x < M/2
    else line_fft<M, false>(v, s, t, stw);
    if (!live) return;
    const int P = n + 1;
    double2 *oa = out + ((long long)z * ny + y) * P, *ob = oa + P;
    for (int k = t; k <= n; k += T) {
        const double2 zk = s[sp(k)], zc = s[sp((M - k) & (M - 1))];
        oa[k] = make_double2(0.5 * (zk.x + zc.x), 0.5 * (zk.y - zc.y));
        ob[k] = make_double2(0.5 * (zk.y + zc.y), 0.5 * (zc.x - zk.x));
    }
}

// Strided pass over lines (o, kx), o < no, kx < P.  Element e of line (o, kx)
// is in[o*in_o + e*in_e + kx] for e < ne_in; elements ne_in..M-1 are zero.
//   MODE_FWD    forward; writes elements e < nw to out[o*out_o + e*out_e + kx]
//   MODE_INV    inverse; writes node w = 0..nw-1 (element (w-1) mod M) to
//               out[o*out_o + w*out_e + kx]
//   MODE_ZSOLVE forward, times the Green's spectrum at (kx, ky = o, kz = e),
//               inverse; writes like MODE_INV
//   MODE_GREEN  forward; writes the real part of elements e <= n to the
//               octant gh_out[(e*P + o)*P + kx] (lines o = ky <= n)
//   MODE_FWD_EVEN forward like MODE_FWD
// MODE_FWD_EVEN and MODE_GREEN read an even sequence from its first half:
// element e is stored at min(e, M - e).
enum PassMode { MODE_FWD = 0, MODE_INV = 1, MODE_ZSOLVE = 2, MODE_GREEN = 3, MODE_FWD_EVEN = 4 };

template <int M, int MODE>
__global__ void __launch_bounds__(FFT_TPB) k_fft_lines(const double2 *__restrict__ in,
                                                       long long in_o, long long in_e, int ne_in,
                                                       double2 *__restrict__ out,
                                                       long long out_o, long long out_e, int nw,
                                                       int no, int P,
                                                       const double *__restrict__ gh,
                                                       double *__restrict__ gh_out,
                                                       const double2 *__restrict__ tw,
                                                       const int *gate) {
    if (gate && *gate == 0) return;
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    constexpr bool INV1 = MODE == MODE_INV;
    extern __shared__ double2 smem[];
    double2 *stw = smem, *sl = smem + M;
    load_twiddles<M>(stw, tw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const long long line = (long long)blockIdx.x * LPB + team;
    const bool live = line < (long long)no * P;
    const int o = live ? (int)(line / P) : 0, kx = live ? (int)(line % P) : 0;
    __syncthreads();
    double2 v[V];
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
    const double2 *src = in + o * in_o + kx;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            int e = first_index<M>(t, j, m);
            if constexpr (MODE == MODE_GREEN || MODE == MODE_FWD_EVEN) e = min(e, M - e);
            v[j * R0 + m] = (live && e < ne_in) ? src[e * in_e] : make_double2(0.0, 0.0);
        }
    double2 *s = sl + team * kLineStride<M>;
    if ((MODE == MODE_FWD || MODE == MODE_ZSOLVE) && 2 * ne_in == M) line_fft<M, INV1, true>(v, s, t, stw);
    else line_fft<M, INV1>(v, s, t, stw);
    if constexpr (MODE == MODE_ZSOLVE) {
        const int b = min(o, M - o);
        for (int e = t; e < M; e += T) {
            const int c = min(e, M - e);
            const double g = live ? gh[((long long)c * P + b) * P + kx] : 0.0;
            s[sp(e)] = make_double2(s[sp(e)].x * g, s[sp(e)].y * g);
        }
        team_sync<M>();
        load_step<M, R0>(v, s, t);
        team_sync<M>();
        line_fft<M, true>(v, s, t, stw);
    }
    if (!live) return;
    if constexpr (MODE == MODE_FWD || MODE == MODE_FWD_EVEN) {
        double2 *dst = out + o * out_o + kx;
        for (int e = t; e < nw; e += T) dst[e * out_e] = s[sp(e)];
    } else if constexpr (MODE == MODE_GREEN) {
        for (int e = t; e < P; e += T) gh_out[((long long)e * P + o) * P + kx] = s[sp(e)].x;
    } else {
        double2 *dst = out + o * out_o + kx;
        for (int w = t; w < nw; w += T) dst[w * out_e] = s[sp((w + M - 1) & (M - 1))];
    }
}

// x pass (inverse, complex to real) for rows (yy, yy+1) of plane zz of S4:
// Z_k = A_k + i B_k for k <= n and conj(A_{m-k}) + i conj(B_{m-k}) above; the
// real and imaginary parts of the inverse are the two rows.  Writes nodes
// -1..n (element (w-1) mod m) times `scale` to phi[(zz*q + yy)*q + w].
template <int M>
__global__ void __launch_bounds__(FFT_TPB) k_fft_x_inv(const double2 *__restrict__ in, int n,
                                                       double scale,
                                                       const double2 *__restrict__ tw,
                                                       double *__restrict__ phi) {
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    extern __shared__ double2 smem[];
    double2 *stw = smem, *sl = smem + M;
    load_twiddles<M>(stw, tw);
    const int q = n + 2, P = n + 1, team = threadIdx.x / T, t = threadIdx.x % T;
    const long long pairs = (long long)q * (q / 2);
    const long long pr = (long long)blockIdx.x * LPB + team;
    const bool live = pr < pairs;
    const int zz = live ? (int)(pr / (q / 2)) : 0, yy = live ? (int)(pr % (q / 2)) * 2 : 0;
    __syncthreads();
    const double2 *ra = in + ((long long)zz * q + yy) * P, *rb = ra + P;
    double2 v[V];
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m);
            double2 z = make_double2(0.0, 0.0);
            if (live) {
                if (e <= n) {
                    const double2 a = ra[e], b = rb[e];
                    z = make_double2(a.x - b.y, a.y + b.x);
                } else {
                    const double2 a = ra[M - e], b = rb[M - e];
                    z = make_double2(a.x + b.y, b.x - a.y);
                }
            }
            v[j * R0 + m] = z;
        }
    double2 *s = sl + team * kLineStride<M>;
    line_fft<M, true>(v, s, t, stw);
    if (!live) return;
    double *pa = phi + ((long long)zz * q + yy) * q, *pb = pa + q;
    for (int w = t; w < q; w += T) {
        const double2 z = s[sp((w + M - 1) & (M - 1))];
        pa[w] = z.x * scale;
        pb[w] = z.y * scale;
    }
}

__global__ void k_twiddle(double2 *tw, int m) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) {
        double s, c;
        sincospi(2.0 * j / m, &s, &c);
        tw[j] = make_double2(c, -s);
    }
}

// ------------------------------------------------ fixed-point tracking solve
//
// The same passes in block floating point on int64 values, for the tracking
// solve from the deposit accumulators: on this GPU the integer pipes issue
// tens of times more operations per clock than the FP64 pipe.  Every line
// transform carries one exponent E (a stored value v means v 2^E):
//  * on input, a pass aligns its line's elements to the largest exponent
//    among them (rounded right shifts), then shifts the whole line so that
//    the sum of the moduli of its elements, L1, is in (2^59, 2^60];
//  * every intermediate value of a line transform is a sum of its inputs
//    times unit-modulus factors, each input at most once, so it stays below
//    L1 <= 2^60 (sums of a real and an imaginary part below 2^61; products by
//    Q63 constants and twiddles floor(a f 2^-63) need |a| < 2^62);
//  * the line's result keeps the line's exponent (x pass: per row pair;
//    forward y: per (z, kx); z solve: per (ky, kx); inverse y: per (zz, kx)),
//    so each value has the precision of its line, as in floating point with
//    one exponent per line;
//  * the z solve multiplies by the Green's spectrum as round(G^ 2^62 / D),
//    D >= max |G^| (G > 0: max |G^| = G^(0)), then renormalises the line;
//  * phi = value 2^E scale_acc 2^-51 D / m^3.

// Blocks per SM the fixed-point passes are compiled for (latency-bound passes
// whose registers are mostly the line's values): where a thread holds at most
// 8 values of its line, four, except three for the inverse y pass (measured at
// 128^3: x 0.038 -> 0.035 ms, z solve 0.246 -> 0.238, inverse x 0.052 ->
// 0.047, forward y 2 us faster with four; the inverse y pass ran slower with
// four, a few spilled words); else two.  `strided`: the inverse y pass.
template <int M, bool strided = false>
constexpr int fixq_blocks() { return M / Shape<M>::T <= 8 ? (strided ? 3 : 4) : 2; }

constexpr int FIX_EMPTY = -100000;   // exponent of an all-zero line (aligns below any other)

__device__ __forceinline__ long long rshr(long long v, int sh) {
    if (sh <= 0) return v;
    if (sh >= 63) return 0;
    return (v + (1ll << (sh - 1))) >> sh;
}
// v 2^-sh (rounded for sh > 0, exact for sh <= 0 given the L1 bound)
__device__ __forceinline__ longlong2 scale2n(longlong2 v, int sh) {
    if (sh >= 0) return make_longlong2(rshr(v.x, sh), rshr(v.y, sh));
    return make_longlong2((long long)((unsigned long long)v.x << (-sh)),
                          (long long)((unsigned long long)v.y << (-sh)));
}
__device__ __forceinline__ unsigned long long l1_part(longlong2 v) {
    const unsigned long long ax = (unsigned long long)(v.x < 0 ? -v.x : v.x);
    const unsigned long long ay = (unsigned long long)(v.y < 0 ? -v.y : v.y);
    return ((ax + ay) >> 16) + 1;   // an upper bound of |v| / 2^16, no overflow over a line
}

// Reductions over the T threads of a line team (teams are T consecutive
// lanes; a 64-thread team spans two warps and exchanges through `red`, two
// words per team).  Every thread of the block calls them.
template <int T>
__device__ __forceinline__ long long team_max(long long v, long long *red) {
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if constexpr (T > 32) {
        const int team = threadIdx.x / T, half = (threadIdx.x % T) / 32;
        if ((threadIdx.x & 31) == 0) red[2 * team + half] = v;
        __syncthreads();
        v = max(red[2 * team], red[2 * team + 1]);
        __syncthreads();
    }
    return v;
}
// The largest of a 32-bit value over a line team: one warp redux for a team
// of 32 lanes, the shuffle tree of team_max otherwise.
template <int T>
__device__ __forceinline__ int team_max_i32(int v, long long *red) {
    if constexpr (T == 32) return __reduce_max_sync(0xffffffffu, v);
    else return (int)team_max<T>(v, red);
}

template <int T>
__device__ __forceinline__ unsigned long long team_sum(unsigned long long v, long long *red) {
    if constexpr (T == 32) {
        // two 32-bit warp reductions, exact for per-lane values below 2^54: 32
        // low parts of 27 bits, and 32 high parts v >> 27 below 2^27, each sum
        // below 2^32 (a lane's share of a line's L1 bound is at most 8 terms of
        // (|re| + |im|) 2^-16 + 1 with |re|, |im| <= 2^60, below 2^49)
        const unsigned lo = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0x7FFFFFFull));
        const unsigned hi = __reduce_add_sync(0xffffffffu, (unsigned)(v >> 27));
        return ((unsigned long long)hi << 27) + lo;
    }
    constexpr int W = T < 32 ? T : 32;
#pragma unroll
    for (int o = W / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if constexpr (T > 32) {
        const int team = threadIdx.x / T, half = (threadIdx.x % T) / 32;
        if ((threadIdx.x & 31) == 0) red[2 * team + half] = (long long)v;
        __syncthreads();
        v = (unsigned long long)red[2 * team] + (unsigned long long)red[2 * team + 1];
        __syncthreads();
    }
    return v;
}

// Normalisation shift of a line from its L1 bound (in units of 2^16): the
// line times 2^-t has L1 in (2^59, 2^60] (t < 0 shifts left); 0 for an
// all-zero line.
__device__ __forceinline__ int norm_shift(unsigned long long l1_16) {
    if (l1_16 == 0) return 0;
    const int bits = 64 - __clzll((long long)l1_16) + 16;   // L1 < 2^bits
    return bits - 60;
}

// Normalises a line whose values share one exponent: returns the shift t
// applied (the line times 2^-t has L1 in (2^59, 2^60]), or INT_MIN for an
// all-zero line.
template <int M, int V>
__device__ __forceinline__ int normalise_line(longlong2 *v, long long *red) {
    constexpr int T = Shape<M>::T;
    unsigned long long l1 = 0;
#pragma unroll
    for (int i = 0; i < V; ++i) l1 += l1_part(v[i]) - 1 + ((v[i].x | v[i].y) != 0);
    l1 = team_sum<T>(l1, red);
    const int t = norm_shift(l1);
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = scale2n(v[i], t);
    return l1 ? t : INT_MIN;
}


// accumulator value (hi 2^31 + lo, 2^51 per particle)
__device__ __forceinline__ unsigned __int128 acc_value(const unsigned long long *__restrict__ hi,
                                                       const unsigned long long *__restrict__ lo,
                                                       long long i) {
    return ((unsigned __int128)hi[i] << DEP_SPLIT) + lo[i];
}
__device__ __forceinline__ int bitlen128(unsigned __int128 v) {
    const unsigned long long h = (unsigned long long)(v >> 64), l = (unsigned long long)v;
    return h ? 128 - __clzll((long long)h) : (l ? 64 - __clzll((long long)l) : 0);
}
__device__ __forceinline__ long long shift128(unsigned __int128 v, int t) {
    if (t <= 0) return (long long)(v << (-t));
    return (long long)((v + ((unsigned __int128)1 << (t - 1))) >> t);
}

// forward x pass from the accumulators (rows in pairs, as k_fft_x_fwd):
// out[(z*n + y)*P + k], P = n+1; the pair's exponent in e1[z*n + y], e1[z*n + y + 1].
// The pair is normalised by its largest value: L1 < m 2^bits(max).
template <int M>
__global__ void __launch_bounds__(FFT_TPB, fixq_blocks<M>()) k_fftq_x_fwd(const unsigned long long *__restrict__ acc_hi,
                                                        const unsigned long long *__restrict__ acc_lo,
                                                        int n, const longlong2 *__restrict__ tw,
                                                        longlong2 *__restrict__ out,
                                                        int *__restrict__ e1) {
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    extern __shared__ longlong2 smq[];
    __shared__ long long red[2 * LPB];
    longlong2 *stw = smq, *sl = smq + M;
    load_twiddles<M>(stw, tw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const long long pairs = (long long)(n / 2) * n;
    const long long pr = (long long)blockIdx.x * LPB + team;
    const bool live = pr < pairs;
    const int z = live ? (int)(pr / (n / 2)) : 0, y = live ? (int)(pr % (n / 2)) * 2 : 0;
    __syncthreads();
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
    const long long row = ((long long)z * n + y) * n;
    unsigned __int128 va[V], vb[V];
    int mb = 0;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m), i = j * R0 + m;
            va[i] = (live && e < n) ? acc_value(acc_hi, acc_lo, row + e) : 0;
            vb[i] = (live && e < n) ? acc_value(acc_hi, acc_lo, row + n + e) : 0;
            mb = max(mb, max(bitlen128(va[i]), bitlen128(vb[i])));
        }
    mb = team_max_i32<T>(mb, red);
    constexpr int LGM = M == 16 ? 4 : M == 32 ? 5 : M == 64 ? 6 : M == 128 ? 7 : M == 256 ? 8 : 9;
    const int sh = mb + LGM - 60;
    longlong2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = make_longlong2(shift128(va[i], sh), shift128(vb[i], sh));
    longlong2 *s = sl + team * kLineStride<M>;
    line_fft<M, false, true>(v, s, t, stw);  // rows x < M/2
    if (!live) return;
    const int P = n + 1;
    longlong2 *oa = out + ((long long)z * n + y) * P, *ob = oa + P;
    for (int k = t; k <= n; k += T) {
        const longlong2 zk = s[sp(k)], zc = s[sp((M - k) & (M - 1))];
        oa[k] = make_longlong2((zk.x + zc.x) >> 1, (zk.y - zc.y) >> 1);
        ob[k] = make_longlong2((zk.y + zc.y) >> 1, (zc.x - zk.x) >> 1);
    }
    if (t == 0) e1[(long long)z * n + y] = e1[(long long)z * n + y + 1] = mb ? sh : FIX_EMPTY;
}

// rint(v 2^-sh) from the bits (round half to even, integer pipes), for
// |v 2^-sh| < 2^62; zero and subnormal v give 0.
__device__ __forceinline__ long long rint_scaled(double v, int sh) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ex = (int)((b >> 52) & 0x7FF);
    if (ex == 0) return 0;
    const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int e = ex - 1075 - sh;   // v 2^-sh = mant 2^e
    unsigned long long r;
    if (e >= 0) {
        r = mant << e;
    } else if (e < -54) {
        r = 0;
    } else {
        const int k = -e;
        r = mant >> k;
        const unsigned long long rem = mant & ((1ull << k) - 1), half = 1ull << (k - 1);
        r += (rem > half || (rem == half && (r & 1ull))) ? 1ull : 0ull;
    }
    return (b >> 63) ? -(long long)r : (long long)r;
}

// forward x pass from a cube of nin^3 doubles (rows in pairs; nin even, the
// adjoint's source on nodes -1..n); each pair normalised by its largest
// exponent: |value| < 2^(E+1), L1 < 2 nin 2^(E+1) <= 2m 2^(E+1).
template <int M>
__global__ void __launch_bounds__(FFT_TPB, fixq_blocks<M>()) k_fftq_x_fwd_d(const double *__restrict__ src, int n,
                                                          int nin, const longlong2 *__restrict__ tw,
                                                          longlong2 *__restrict__ out,
                                                          int *__restrict__ e1) {
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    extern __shared__ longlong2 smq[];
    __shared__ long long red[2 * LPB];
    longlong2 *stw = smq, *sl = smq + M;
    load_twiddles<M>(stw, tw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const long long pairs = (long long)(nin / 2) * nin;
    const long long pr = (long long)blockIdx.x * LPB + team;
    const bool live = pr < pairs;
    const int z = live ? (int)(pr / (nin / 2)) : 0, y = live ? (int)(pr % (nin / 2)) * 2 : 0;
    __syncthreads();
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
    const long long row = ((long long)z * nin + y) * nin;
    double va[V], vb[V];
    int ef = 0;   // largest biased exponent field
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m), i = j * R0 + m;
            va[i] = (live && e < nin) ? src[row + e] : 0.0;
            vb[i] = (live && e < nin) ? src[row + nin + e] : 0.0;
            const int fa = (int)(((unsigned long long)__double_as_longlong(va[i]) >> 52) & 0x7FF);
            const int fb = (int)(((unsigned long long)__double_as_longlong(vb[i]) >> 52) & 0x7FF);
            ef = max(ef, max(fa, fb));
        }
    ef = team_max_i32<T>(ef, red);
    constexpr int LGM = M == 16 ? 4 : M == 32 ? 5 : M == 64 ? 6 : M == 128 ? 7 : M == 256 ? 8 : 9;
    // |value| < 2^(ef - 1022); L1 < 2m 2^(ef - 1022) <= 2^60 after the shift
    const int sh = (ef - 1022) + LGM + 1 - 60;
    longlong2 v[V];
#pragma unroll
    for (int i = 0; i < V; ++i) v[i] = make_longlong2(rint_scaled(va[i], sh), rint_scaled(vb[i], sh));
    longlong2 *s = sl + team * kLineStride<M>;
    line_fft<M, false>(v, s, t, stw);
    if (!live) return;
    const int P = n + 1;
    longlong2 *oa = out + ((long long)z * nin + y) * P, *ob = oa + P;
    for (int k = t; k <= n; k += T) {
        const longlong2 zk = s[sp(k)], zc = s[sp((M - k) & (M - 1))];
        oa[k] = make_longlong2((zk.x + zc.x) >> 1, (zk.y - zc.y) >> 1);
        ob[k] = make_longlong2((zk.y + zc.y) >> 1, (zc.x - zk.x) >> 1);
    }
    if (t == 0) e1[(long long)z * nin + y] = e1[(long long)z * nin + y + 1] = ef ? sh : FIX_EMPTY;
}

// Strided line passes as k_fft_lines (MODE_FWD: forward y; MODE_ZSOLVE:
// forward z, times the quantised Green's spectrum, inverse z; MODE_INV:
// inverse y).  Element e of line (o, kx) has exponent
// ein[o*ein_o + e*ein_e + kx*ein_k]; the line's exponent goes to eout[o*P + kx].
template <int M, int MODE>
__global__ void __launch_bounds__(FFT_TPB, fixq_blocks<M, MODE == MODE_INV>()) k_fftq_lines(const longlong2 *__restrict__ in,
                                                        long long in_o, long long in_e, int ne_in,
                                                        const int *__restrict__ ein, long long ein_o,
                                                        long long ein_e, long long ein_k,
                                                        longlong2 *__restrict__ out,
                                                        long long out_o, long long out_e, int nw,
                                                        int *__restrict__ eout,
                                                        int no, int P,
                                                        const long long *__restrict__ gq,
                                                        const longlong2 *__restrict__ tw) {
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    constexpr bool INV1 = MODE == MODE_INV;
    extern __shared__ longlong2 smq[];
    __shared__ long long red[2 * LPB];
    longlong2 *stw = smq, *sl = smq + M;
    load_twiddles<M>(stw, tw);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const long long line = (long long)blockIdx.x * LPB + team;
    const bool live = line < (long long)no * P;
    const int o = live ? (int)(line / P) : 0, kx = live ? (int)(line % P) : 0;
    __syncthreads();
    longlong2 v[V];
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
    const longlong2 *src = in + o * in_o + kx;
    const int *esrc = ein + o * ein_o + kx * ein_k;
    // the line's largest exponent, then the values aligned to it (exponents
    // read twice rather than held in registers)
    int emax = FIX_EMPTY;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m);
            if (live && e < ne_in) emax = max(emax, __ldg(&esrc[e * ein_e]));
        }
    emax = team_max_i32<T>(emax, red);
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m), i = j * R0 + m;
            v[i] = (live && e < ne_in) ? scale2n(src[e * in_e], emax - __ldg(&esrc[e * ein_e]))
                                       : make_longlong2(0, 0);
        }
    const int t0 = normalise_line<M, V>(v, red);
    int E = t0 == INT_MIN ? FIX_EMPTY : emax + t0;
    longlong2 *s = sl + team * kLineStride<M>;
    if ((MODE == MODE_FWD || MODE == MODE_ZSOLVE) && 2 * ne_in == M) line_fft<M, INV1, true>(v, s, t, stw);
    else line_fft<M, INV1>(v, s, t, stw);
    if constexpr (MODE == MODE_ZSOLVE) {
        const int b = min(o, M - o);
        for (int e = t; e < M; e += T) {
            const int c = min(e, M - e);
            const long long g = live ? gq[((long long)c * P + b) * P + kx] : 0;
            const longlong2 a = s[sp(e)];
            // floor(a g 2^-62), |a| <= 2^60
            s[sp(e)] = make_longlong2(__mul64hi((long long)((unsigned long long)a.x << 2), g),
                                  __mul64hi((long long)((unsigned long long)a.y << 2), g));
        }
        team_sync<M>();
        load_step<M, R0>(v, s, t);
        team_sync<M>();
        // renormalise the product line (all elements share exponent E)
        const int t1 = normalise_line<M, V>(v, red);
        E = (t1 == INT_MIN || E == FIX_EMPTY) ? FIX_EMPTY : E + t1;
        line_fft<M, true>(v, s, t, stw);
    }
    if (live && t == 0) eout[(long long)o * P + kx] = E;
    if (!live) return;
    longlong2 *dst = out + o * out_o + kx;
    if constexpr (MODE == MODE_FWD) {
        for (int e = t; e < nw; e += T) dst[e * out_e] = s[sp(e)];
    } else {
        for (int w = t; w < nw; w += T) dst[w * out_e] = s[sp((w + M - 1) & (M - 1))];
    }
}

// inverse x pass (complex to real, as k_fft_x_inv); element kx of rows
// (zz, yy), (zz, yy+1) has exponent e4[zz*P + kx]; writes phi[(zz*q + yy)*q + w]
// = value 2^(E + eoff) scale_dev-or-scale D / m^3, nodes -1..n (eoff = -51
// for the accumulators, 2^51 per particle; 0 for a double source).
template <int M>
__global__ void __launch_bounds__(FFT_TPB, fixq_blocks<M>()) k_fftq_x_inv(const longlong2 *__restrict__ in, int n,
                                                        const int *__restrict__ e4,
                                                        const FixScales *__restrict__ fs,
                                                        double scale, const double *scale_dev,
                                                        int eoff,
                                                        const longlong2 *__restrict__ tw,
                                                        double *__restrict__ phi) {
    constexpr int T = Shape<M>::T, LPB = FFT_TPB / T, V = M / T;
    extern __shared__ longlong2 smq[];
    __shared__ long long red[2 * LPB];
    longlong2 *stw = smq, *sl = smq + M;
    load_twiddles<M>(stw, tw);
    const int q = n + 2, P = n + 1, team = threadIdx.x / T, t = threadIdx.x % T;
    const long long pairs = (long long)q * (q / 2);
    const long long pr = (long long)blockIdx.x * LPB + team;
    const bool live = pr < pairs;
    const int zz = live ? (int)(pr / (q / 2)) : 0, yy = live ? (int)(pr % (q / 2)) * 2 : 0;
    __syncthreads();
    const longlong2 *ra = in + ((long long)zz * q + yy) * P, *rb = ra + P;
    const int *er = e4 + (long long)zz * P;
    longlong2 v[V];
    constexpr int R0 = Shape<M>::R0, U0 = (M / R0) / T;
    // exponents first: the packed value A + iB of element e comes from kx = e or m - e
    int emax = FIX_EMPTY;
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m);
            if (live) emax = max(emax, __ldg(&er[e <= n ? e : M - e]));
        }
    emax = team_max_i32<T>(emax, red);
#pragma unroll
    for (int j = 0; j < U0; ++j)
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int e = first_index<M>(t, j, m), i = j * R0 + m;
            longlong2 z = make_longlong2(0, 0);
            if (live) {
                const int d = emax - __ldg(&er[e <= n ? e : M - e]);
                if (e <= n) {
                    const longlong2 a = scale2n(ra[e], d), b = scale2n(rb[e], d);
                    z = make_longlong2(a.x - b.y, a.y + b.x);
                } else {
                    const longlong2 a = scale2n(ra[M - e], d), b = scale2n(rb[M - e], d);
                    z = make_longlong2(a.x + b.y, b.x - a.y);
                }
            }
            v[i] = z;
        }
    // |A + iB| <= |A| + |B| <= 2^61.x: renormalise (now all at exponent emax)
    const int tn = normalise_line<M, V>(v, red);
    const int E = (tn == INT_MIN || emax == FIX_EMPTY) ? FIX_EMPTY : emax + tn;
    longlong2 *s = sl + team * kLineStride<M>;
    line_fft<M, true>(v, s, t, stw);
    if (!live) return;
    const double sc = (scale_dev ? *scale_dev : scale) * fs->F * ldexp(1.0, E + eoff);
    double *pa = phi + ((long long)zz * q + yy) * q, *pb = pa + q;
    for (int w = t; w < q; w += T) {
        const longlong2 z = s[sp((w + M - 1) & (M - 1))];
        pa[w] = (double)z.x * sc;
        pb[w] = (double)z.y * sc;
    }
}

// Twiddles exp(-2 pi i j/m) in Q63 (1 as 2^63 - 1).
__global__ void k_twiddle_q(longlong2 *tw, int m) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) {
        double s, c;
        sincospi(2.0 * j / m, &s, &c);
        auto q = [](double v) {
            return v >= 1.0 ? 0x7FFFFFFFFFFFFFFFll : v <= -1.0 ? -0x7FFFFFFFFFFFFFFFll
                                                               : __double2ll_rn(v * 0x1p63);
        };
        tw[j] = make_longlong2(q(c), q(-s));
    }
}

// round(G^ 2^62 / D) on the spectrum octant, D = G^(0) (1 + 1e-9) >= max |G^|
// (G > 0); fs = {D, D / m^3}.  No usable spectrum: a zero spectrum, phi NaN.
__global__ void k_green_quant(const double *__restrict__ gh, long long cnt, int M,
                              FixScales *__restrict__ fs, long long *__restrict__ gq,
                              const int *gate) {
    if (gate && *gate == 0) return;
    const double g0 = gh[0];
    const bool ok = g0 > 0.0 && isfinite(g0);
    const double D = ok ? g0 * (1.0 + 1e-9) : 0.0, inv = ok ? 0x1p62 / D : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        fs->D = D;
        fs->F = ok ? D / ((double)M * M * M) : __longlong_as_double(0x7FF8000000000000ll);
    }
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < cnt;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = fmin(fmax(gh[i] * inv, -0x1p62), 0x1p62);
        gq[i] = ok ? __double2ll_rn(r) : 0;
    }
}

// ------------------------------------------------------------------ driver

static int team_size(int M) { return M == 512 ? 64 : M == 256 ? 32 : M == 128 ? 16 : M == 64 ? 8 : 4; }

static size_t smem_bytes(int M) {
    return (size_t)(M + (FFT_TPB / team_size(M)) * (M + M / 16)) * sizeof(double2);
}

template <int M>
static void set_attrs() {
    const int sm = (int)smem_bytes(M);
    cudaFuncSetAttribute(k_fft_x_fwd<M, SRC_RHO>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_x_fwd<M, SRC_GREEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_ZSOLVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_GREEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_FWD_EVEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_x_inv<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_x_fwd<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_x_fwd_d<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_ZSOLVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fftq_x_inv<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    // the fixed-point passes are latency-bound: room for several blocks per SM
    cudaFuncSetAttribute(k_fftq_x_fwd<M>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fftq_x_fwd_d<M>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_FWD>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_ZSOLVE>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fftq_lines<M, MODE_INV>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    cudaFuncSetAttribute(k_fftq_x_inv<M>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

cudaError_t fft_plan_init(FftPlan *p, int n) {
    p->n = n;
    p->m = 2 * n;
    p->buf = p->buf2 = p->tw = nullptr;
    p->ghat = nullptr;
    p->twq = nullptr;
    p->ghat_q = nullptr;
    p->fs = nullptr;
    p->fexp = nullptr;
    const long long m = p->m, P = n + 1;
    const long long big = m * m * P;  // largest spectrum (the Green's x pass output)
    cudaError_t e = cudaMalloc(&p->buf, big * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->buf2, big * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->tw, m * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->ghat, P * P * P * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&p->twq, m * sizeof(longlong2));
    if (e == cudaSuccess) e = cudaMalloc(&p->ghat_q, P * P * P * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&p->fs, sizeof(FixScales));
    if (e == cudaSuccess)
        e = cudaMalloc(&p->fexp, ((long long)(n + 2) * (n + 2) + 2 * (n + 2) * P + m * P) * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->fs, 0, sizeof(FixScales));
    if (e != cudaSuccess) {
        fft_plan_free(p);
        return e;
    }
    switch (p->m) {
        case 16: set_attrs<16>(); break;
        case 32: set_attrs<32>(); break;
        case 64: set_attrs<64>(); break;
        case 128: set_attrs<128>(); break;
        case 256: set_attrs<256>(); break;
        case 512: set_attrs<512>(); break;
        default: return cudaErrorInvalidValue;
    }
    BT_LAUNCH(K_TWIDDLE, (cudaStream_t)0, k_twiddle<<<(p->m + 255) / 256, 256>>>(p->tw, p->m));
    BT_LAUNCH(K_TWIDDLE, (cudaStream_t)0, k_twiddle_q<<<(p->m + 255) / 256, 256>>>(p->twq, p->m));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

void fft_plan_free(FftPlan *p) {
    if (p->buf) cudaFree(p->buf);
    if (p->buf2) cudaFree(p->buf2);
    if (p->tw) cudaFree(p->tw);
    if (p->ghat) cudaFree(p->ghat);
    if (p->twq) cudaFree(p->twq);
    if (p->ghat_q) cudaFree(p->ghat_q);
    if (p->fs) cudaFree(p->fs);
    if (p->fexp) cudaFree(p->fexp);
    p->buf = p->buf2 = p->tw = nullptr;
    p->ghat = nullptr;
    p->twq = nullptr;
    p->ghat_q = nullptr;
    p->fs = nullptr;
    p->fexp = nullptr;
}

static inline unsigned blocks_lines(long long lines, int M) {
    const long long lpb = FFT_TPB / team_size(M);
    return (unsigned)((lines + lpb - 1) / lpb);
}

// phi (nodes -1..n) = G (*) source, the source a cube of nin^3 nodes at
// doubled-grid offsets 0..nin-1 (nin = n: rho; nin = n+2: the adjoint source).
template <int M>
static cudaError_t solve_m(const FftPlan *p, const XIn &in, int src, int nin, double *phi,
                           cudaStream_t s) {
    const int n = p->n;
    const long long P = n + 1, q = n + 2;
    const size_t sm = smem_bytes(M);
    double2 *S1 = p->buf, *S2 = p->buf2, *S3 = p->buf, *S4 = p->buf2;
    // x: rows y, z < nin in pairs -> S1[z][y][kx]
    const long long xpairs = (long long)(nin / 2) * nin;
    BT_LAUNCH(K_FFT_X, s, k_fft_x_fwd<M, SRC_RHO><<<blocks_lines(xpairs, M), FFT_TPB, sm, s>>>(
                              in, n, nin, nin, p->tw, S1, nullptr));
    // y: lines (z < nin, kx), inputs y < nin -> S2[z][ky][kx], all ky
    BT_LAUNCH(K_FFT_YZ, s, k_fft_lines<M, MODE_FWD><<<blocks_lines(nin * P, M), FFT_TPB, sm, s>>>(
                               S1, nin * P, P, nin, S2, M * P, P, M, nin, (int)P, nullptr, nullptr,
                               p->tw, nullptr));
    // z fused: lines (ky < m, kx), inputs z < nin -> S3[zz][ky][kx], zz < n+2
    BT_LAUNCH(K_FFT_ZSOLVE, s,
              k_fft_lines<M, MODE_ZSOLVE><<<blocks_lines((long long)M * P, M), FFT_TPB, sm, s>>>(
                  S2, P, (long long)M * P, nin, S3, P, (long long)M * P, (int)q, M, (int)P, p->ghat,
                  nullptr, p->tw, nullptr));
    // inverse y: lines (zz < n+2, kx), all ky -> S4[zz][yy][kx]
    BT_LAUNCH(K_FFT_YZ, s, k_fft_lines<M, MODE_INV><<<blocks_lines(q * P, M), FFT_TPB, sm, s>>>(
                               S3, (long long)M * P, P, M, S4, q * P, P, (int)q, (int)q, (int)P,
                               nullptr, nullptr, p->tw, nullptr));
    // inverse x (complex to real) -> phi on nodes -1..n
    const double scale = 1.0 / ((double)M * M * M);
    BT_LAUNCH(K_FFT_XINV, s, k_fft_x_inv<M><<<blocks_lines(q * (q / 2), M), FFT_TPB, sm, s>>>(
                                 S4, n, scale, p->tw, phi));
    return cudaGetLastError();
}

// The solve in block floating point (passes and layouts as solve_m): the
// source is the accumulators (nin = n) or a cube of nin^3 doubles (src_d);
// line exponents in p->fexp: e1[z][y] (nin^2), e2[z][kx] (nin P),
// e3[ky][kx] (m P), e4[zz][kx] ((n+2) P).
template <int M>
static cudaError_t solve_fix_m(const FftPlan *p, const unsigned long long *acc_hi,
                              const unsigned long long *acc_lo, const double *src_d, int nin,
                              double scale, const double *scale_dev, int eoff, double *phi,
                              cudaStream_t s) {
    const int n = p->n;
    const long long P = n + 1, q = n + 2;
    const size_t sm = smem_bytes(M);
    longlong2 *S1 = (longlong2 *)p->buf, *S2 = (longlong2 *)p->buf2, *S3 = S1, *S4 = S2;
    int *e1 = p->fexp, *e2 = e1 + q * q, *e3 = e2 + q * P, *e4 = e3 + M * P;
    if (src_d)
        BT_LAUNCH(K_FFT_X, s, k_fftq_x_fwd_d<M><<<blocks_lines((long long)(nin / 2) * nin, M), FFT_TPB,
                                                   sm, s>>>(src_d, n, nin, p->twq, S1, e1));
    else
        BT_LAUNCH(K_FFT_X, s, k_fftq_x_fwd<M><<<blocks_lines((long long)(n / 2) * n, M), FFT_TPB, sm,
                                                 s>>>(acc_hi, acc_lo, n, p->twq, S1, e1));
    // y: lines (z, kx), element y with exponent e1[z][y]
    BT_LAUNCH(K_FFT_YZ, s, k_fftq_lines<M, MODE_FWD><<<blocks_lines(nin * P, M), FFT_TPB, sm, s>>>(
                               S1, nin * P, P, nin, e1, nin, 1, 0, S2, M * P, P, M, e2, nin, (int)P,
                               nullptr, p->twq));
    // z: lines (ky, kx), element z with exponent e2[z][kx]
    BT_LAUNCH(K_FFT_ZSOLVE, s,
              k_fftq_lines<M, MODE_ZSOLVE><<<blocks_lines((long long)M * P, M), FFT_TPB, sm, s>>>(
                  S2, P, (long long)M * P, nin, e2, 0, P, 1, S3, P, (long long)M * P, (int)q, e3,
                  M, (int)P, p->ghat_q, p->twq));
    // inverse y: lines (zz, kx), element ky with exponent e3[ky][kx]
    BT_LAUNCH(K_FFT_YZ, s, k_fftq_lines<M, MODE_INV><<<blocks_lines(q * P, M), FFT_TPB, sm, s>>>(
                               S3, (long long)M * P, P, M, e3, 0, P, 1, S4, q * P, P, (int)q, e4,
                               (int)q, (int)P, nullptr, p->twq));
    BT_LAUNCH(K_FFT_XINV, s, k_fftq_x_inv<M><<<blocks_lines(q * (q / 2), M), FFT_TPB, sm, s>>>(
                                 S4, n, e4, p->fs, scale, scale_dev, eoff, p->twq, phi));
    return cudaGetLastError();
}


// Spectrum of the doubled Green's function from its octant table.  The doubled
// G is even in every dimension, so each pass only transforms the lines whose
// outer indices lie in the first half (0..n) and reads mirrored inputs:
// x over rows y <= n+1, z <= n; y over lines z <= n; z over lines ky <= n.
template <int M>
static cudaError_t green_m(const FftPlan *p, const double *gtable, cudaStream_t s, const int *gate) {
    const int n = p->n;
    const long long P = n + 1, ny = n + 2;
    const size_t sm = smem_bytes(M);
    XIn in{};
    in.g = gtable;
    // x: rows y < n+2 (pairs), z <= n -> buf[z][y][kx]
    BT_LAUNCH(K_GREEN_X, s, k_fft_x_fwd<M, SRC_GREEN><<<blocks_lines((ny / 2) * P, M), FFT_TPB, sm, s>>>(
                                in, n, (int)ny, (int)P, p->tw, p->buf, gate));
    // y: lines (z <= n, kx), element y read at min(y, m - y) -> buf2[z][ky][kx], ky <= n
    BT_LAUNCH(K_GREEN_YZ, s, k_fft_lines<M, MODE_FWD_EVEN><<<blocks_lines(P * P, M), FFT_TPB, sm, s>>>(
                                 p->buf, ny * P, P, (int)ny, p->buf2, P * P, P, (int)P, (int)P,
                                 (int)P, nullptr, nullptr, p->tw, gate));
    // z: lines (ky <= n, kx), element z read at min(z, m - z) -> real part at kz <= n
    BT_LAUNCH(K_GREEN_YZ, s, k_fft_lines<M, MODE_GREEN><<<blocks_lines(P * P, M), FFT_TPB, sm, s>>>(
                                 p->buf2, P, P * P, (int)P, nullptr, 0, 0, 0, (int)P, (int)P, nullptr,
                                 p->ghat, p->tw, gate));
    // the block-floating-point solve's quantised spectrum
    return green_quantize(p, s, gate);
}

static cudaError_t solve_any(const FftPlan *p, const XIn &in, int src, int nin, double *phi,
                             cudaStream_t s) {
    switch (p->m) {
        case 16: return solve_m<16>(p, in, src, nin, phi, s);
        case 32: return solve_m<32>(p, in, src, nin, phi, s);
        case 64: return solve_m<64>(p, in, src, nin, phi, s);
        case 128: return solve_m<128>(p, in, src, nin, phi, s);
        case 256: return solve_m<256>(p, in, src, nin, phi, s);
        case 512: return solve_m<512>(p, in, src, nin, phi, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t solve_rho_to_phi(const FftPlan *p, const double *rho, double *phi, cudaStream_t s) {
    XIn in{};
    in.rho = rho;
    return solve_any(p, in, SRC_RHO, p->n, phi, s);
}

// Transpose of the solve (G even, its circulant symmetric): the source
// phibar on nodes -1..n ((n+2)^3, index node + 1) placed at doubled-grid
// offsets 0..n+1 (a shift by one node), convolved with G; the result for
// node j = 0..n-1 is out[j + 2] in each dimension of the (n+2)^3 output.
cudaError_t solve_adjoint_shifted(const FftPlan *p, const double *phibar, double *out,
                                  cudaStream_t s) {
    XIn in{};
    in.rho = phibar;
    return solve_any(p, in, SRC_RHO, p->n + 2, out, s);
}

static cudaError_t solve_fix_dispatch(const FftPlan *p, const unsigned long long *acc_hi,
                                      const unsigned long long *acc_lo, const double *src_d,
                                      int nin, double scale, const double *scale_dev, int eoff,
                                      double *phi, cudaStream_t s) {
    switch (p->m) {
#define BT_FIX_CASE(MM)                                                                          \
    case MM:                                                                                     \
        return solve_fix_m<MM>(p, acc_hi, acc_lo, src_d, nin, scale, scale_dev, eoff, phi, s);
        BT_FIX_CASE(16)
        BT_FIX_CASE(32)
        BT_FIX_CASE(64)
        BT_FIX_CASE(128)
        BT_FIX_CASE(256)
        BT_FIX_CASE(512)
#undef BT_FIX_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t solve_acc_to_phi_fixed(const FftPlan *p, const unsigned long long *acc_hi,
                                   const unsigned long long *acc_lo, double scale, double *phi,
                                   cudaStream_t s, const double *scale_dev) {
    return solve_fix_dispatch(p, acc_hi, acc_lo, nullptr, p->n, scale, scale_dev, -51, phi, s);
}

// The transpose of the solve (as solve_adjoint_shifted) in block floating point.
cudaError_t solve_adjoint_shifted_fixed(const FftPlan *p, const double *phibar, double *out,
                                        cudaStream_t s) {
    return solve_fix_dispatch(p, nullptr, nullptr, phibar, p->n + 2, 1.0, nullptr, 0, out, s);
}

// ghat_q and the scales from ghat (after a build or after loading a stored
// spectrum into ghat).
cudaError_t green_quantize(const FftPlan *p, cudaStream_t s, const int *gate) {
    const long long P = p->n + 1, cnt = P * P * P;
    const unsigned qb = (unsigned)std::min<long long>((cnt + 255) / 256, 148 * 8);
    BT_LAUNCH(K_GREEN_YZ, s, k_green_quant<<<qb, 256, 0, s>>>(p->ghat, cnt, p->m, p->fs, p->ghat_q,
                                                              gate));
    return cudaGetLastError();
}

cudaError_t green_spectrum_from_table(const FftPlan *p, const double *gtable, cudaStream_t s,
                                      const int *gate) {
    switch (p->m) {
        case 16: return green_m<16>(p, gtable, s, gate);
        case 32: return green_m<32>(p, gtable, s, gate);
        case 64: return green_m<64>(p, gtable, s, gate);
        case 128: return green_m<128>(p, gtable, s, gate);
        case 256: return green_m<256>(p, gtable, s, gate);
        case 512: return green_m<512>(p, gtable, s, gate);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bt
