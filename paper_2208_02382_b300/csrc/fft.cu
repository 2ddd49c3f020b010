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
// Design (the FP64 issue rate bounds every pass on this GPU, so the passes do
// as few floating-point operations as the transform allows):
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
//    sincospi), and exchanges values through shared memory between radix steps.
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

// DFT-4 of (v0, v1, v2, v3); HALF: v2 = v3 = 0 (not read).
template <bool INV, bool HALF>
__device__ __forceinline__ void dft4(double2 *v) {
    if constexpr (HALF) {
        const double2 a = v[0], b = v[1], rb = rot90<INV>(b);
        v[0] = cadd(a, b);
        v[1] = cadd(a, rb);
        v[2] = csub(a, b);
        v[3] = csub(a, rb);
    } else {
        double2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        double2 t2 = cadd(v[1], v[3]), t3 = rot90<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
}

// DFT-8; HALF: v4..v7 = 0 (not read).
template <bool INV, bool HALF>
__device__ __forceinline__ void dft8(double2 *v) {
    double2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft4<INV, HALF>(e);
    dft4<INV, HALF>(o);
    v[0] = cadd(e[0], o[0]);
    v[4] = csub(e[0], o[0]);
    bfly_w8_1<INV>(e[1], o[1], v[1], v[5]);
    const double2 r2 = rot90<INV>(o[2]);
    v[2] = cadd(e[2], r2);
    v[6] = csub(e[2], r2);
    bfly_w8_3<INV>(e[3], o[3], v[3], v[7]);
}

// DFT-16; HALF: v8..v15 = 0 (not read).  The twiddles exp(-+ 2 pi i q/16)
// (sg = -1 forward, +1 inverse; S16 = sin(pi/8) = C16 T16) are written as
// C16 (1 + i t) or sg C16 (t + i) with t = +-T16, as RS2 (+-1 +- i), or +-i.
template <bool INV, bool HALF>
__device__ __forceinline__ void dft16(double2 *v) {
    double2 e[8], o[8];
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
    const double2 r4 = rot90<INV>(o[4]);
    v[4] = cadd(e[4], r4);
    v[12] = csub(e[4], r4);
    bfly_st(e[5], o[5], sg * C16, -sg * T16, v[5], v[13]);     // (-S16, sg C16)
    bfly_w8_3<INV>(e[6], o[6], v[6], v[14]);
    bfly_ct(e[7], o[7], -C16, -sg * T16, v[7], v[15]);         // (-C16, sg S16)
}

template <int R, bool INV, bool HALF = false>
__device__ __forceinline__ void dft(double2 *v) {
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
template <> struct Shape<128> { static constexpr int S = 2, R0 = 16, R1 = 8, R2 = 1, T = 8; };
template <> struct Shape<256> { static constexpr int S = 2, R0 = 16, R1 = 16, R2 = 1, T = 16; };
template <> struct Shape<512> { static constexpr int S = 3, R0 = 8, R1 = 8, R2 = 8, T = 64; };

constexpr int FFT_TPB = 256;

// One Stockham radix step on values held in registers.  Thread t of the team
// holds units u = t + j*T (j < U = (M/R)/T); unit u's inputs are the line
// elements u + m*(M/R), in v[j*R + m].  Twiddles W_{L R}^{k m} (k = u mod L)
// are applied before the radix-R DFT; output q of unit u belongs at line
// position (u-k)*R + q*L + k.
template <int M, int R, int L, bool INV, bool HALF = false>
__device__ __forceinline__ void step_regs(double2 *v, int t, const double2 *__restrict__ tw) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j) {
        double2 *x = v + j * R;
        if constexpr (L > 1) {
            const int u = t + j * T, k = u % L;
#pragma unroll
            for (int m = 1; m < R; ++m) {
                double2 w = tw[(k * m) * (M / (L * R))];
                if (INV) w.y = -w.y;
                x[m] = cmul(x[m], w);
            }
        }
        dft<R, INV, HALF>(x);
    }
}

template <int M, int R, int L>
__device__ __forceinline__ void store_step(const double2 *v, double2 *s, int t) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const int u = t + j * T, k = u % L;
#pragma unroll
        for (int q = 0; q < R; ++q) s[(u - k) * R + q * L + k] = v[j * R + q];
    }
}

template <int M, int R>
__device__ __forceinline__ void load_step(double2 *v, const double2 *s, int t) {
    constexpr int T = Shape<M>::T, U = (M / R) / T;
#pragma unroll
    for (int j = 0; j < U; ++j)
#pragma unroll
        for (int m = 0; m < R; ++m) v[j * R + m] = s[(t + j * T) + m * (M / R)];
}

// Line element held in register slot (j, m) before the first step.
template <int M>
__device__ __forceinline__ int first_index(int t, int j, int m) {
    constexpr int R = Shape<M>::R0, T = Shape<M>::T;
    return (t + j * T) + m * (M / R);
}

// Full line transform: `v` holds the first step's inputs (first_index order);
// the result (natural order) is left in the team's shared line `s`.  Every
// thread of the block calls this (it synchronises the block).  HALF: the
// line's upper half (elements M/2..M-1) is zero; these are exactly the inputs
// m >= R0/2 of every first-step DFT (element u + m M/R0 with u < M/R0), which
// the half codelets neither read nor add.
template <int M, bool INV, bool HALF = false>
__device__ __forceinline__ void line_fft(double2 *v, double2 *s, int t, const double2 *tw) {
    using SH = Shape<M>;
    constexpr int R0 = SH::R0, R1 = SH::R1, R2 = SH::R2;
    step_regs<M, R0, 1, INV, HALF>(v, t, tw);
    store_step<M, R0, 1>(v, s, t);
    __syncthreads();
    load_step<M, R1>(v, s, t);
    __syncthreads();
    step_regs<M, R1, R0, INV>(v, t, tw);
    store_step<M, R1, R0>(v, s, t);
    if constexpr (SH::S == 3) {
        __syncthreads();
        load_step<M, R2>(v, s, t);
        __syncthreads();
        step_regs<M, R2, R0 * R1, INV>(v, t, tw);
        store_step<M, R2, R0 * R1>(v, s, t);
    }
    __syncthreads();
}

template <int M>
__device__ __forceinline__ void load_twiddles(double2 *stw, const double2 *__restrict__ tw) {
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

// Source of the x pass: rho as doubles, the fixed-point deposit accumulators
// (rho = scale * (hi * 2^31 + lo) * 2^-51), or the even extension of the
// Green's function octant table (full m^3 input, for its spectrum).
enum XSource { SRC_RHO = 0, SRC_ACC = 1, SRC_GREEN = 2 };

struct XIn {
    const double *rho;
    const unsigned long long *acc_hi, *acc_lo;
    double scale;
    const double *scale_ptr;  // if set, the scale is read from the device
    const double *g;
};

template <int M, int SRC>
__device__ __forceinline__ double x_value(const XIn &in, int n, int nin, int x, int y, int z) {
    if constexpr (SRC == SRC_GREEN) {
        const int a = min(x, M - x), b = min(y, M - y), c = min(z, M - z), q = n + 1;
        return in.g[((long long)c * q + b) * q + a];
    } else {
        if (x >= nin) return 0.0;
        const long long i = ((long long)z * nin + y) * nin + x;
        if constexpr (SRC == SRC_RHO) return in.rho[i];
        return in.scale * (((double)in.acc_hi[i] * 2147483648.0 + (double)in.acc_lo[i]) * 0x1p-51);
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
    if (SRC == SRC_ACC && in.scale_ptr) in.scale = *in.scale_ptr;
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
    double2 *s = sl + team * M;
    if (SRC != SRC_GREEN && 2 * nin == M) line_fft<M, false, true>(v, s, t, stw);  // rows x < M/2
    else line_fft<M, false>(v, s, t, stw);
    if (!live) return;
    const int P = n + 1;
    double2 *oa = out + ((long long)z * ny + y) * P, *ob = oa + P;
    for (int k = t; k <= n; k += T) {
        const double2 zk = s[k], zc = s[(M - k) & (M - 1)];
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
    double2 *s = sl + team * M;
    if ((MODE == MODE_FWD || MODE == MODE_ZSOLVE) && 2 * ne_in == M) line_fft<M, INV1, true>(v, s, t, stw);
    else line_fft<M, INV1>(v, s, t, stw);
    if constexpr (MODE == MODE_ZSOLVE) {
        const int b = min(o, M - o);
        for (int e = t; e < M; e += T) {
            const int c = min(e, M - e);
            const double g = live ? gh[((long long)c * P + b) * P + kx] : 0.0;
            s[e] = make_double2(s[e].x * g, s[e].y * g);
        }
        __syncthreads();
        load_step<M, R0>(v, s, t);
        __syncthreads();
        line_fft<M, true>(v, s, t, stw);
    }
    if (!live) return;
    if constexpr (MODE == MODE_FWD || MODE == MODE_FWD_EVEN) {
        double2 *dst = out + o * out_o + kx;
        for (int e = t; e < nw; e += T) dst[e * out_e] = s[e];
    } else if constexpr (MODE == MODE_GREEN) {
        for (int e = t; e < P; e += T) gh_out[((long long)e * P + o) * P + kx] = s[e].x;
    } else {
        double2 *dst = out + o * out_o + kx;
        for (int w = t; w < nw; w += T) dst[w * out_e] = s[(w + M - 1) & (M - 1)];
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
    double2 *s = sl + team * M;
    line_fft<M, true>(v, s, t, stw);
    if (!live) return;
    double *pa = phi + ((long long)zz * q + yy) * q, *pb = pa + q;
    for (int w = t; w < q; w += T) {
        const double2 z = s[(w + M - 1) & (M - 1)];
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

// ------------------------------------------------------------------ driver

static int team_size(int M) { return M == 512 ? 64 : M == 256 ? 16 : M >= 64 ? 8 : 4; }

static size_t smem_bytes(int M) {
    return (size_t)(M + (FFT_TPB / team_size(M)) * M) * sizeof(double2);
}

template <int M>
static void set_attrs() {
    const int sm = (int)smem_bytes(M);
    cudaFuncSetAttribute(k_fft_x_fwd<M, SRC_RHO>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_x_fwd<M, SRC_ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_x_fwd<M, SRC_GREEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_ZSOLVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_GREEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_lines<M, MODE_FWD_EVEN>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
    cudaFuncSetAttribute(k_fft_x_inv<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
}

cudaError_t fft_plan_init(FftPlan *p, int n) {
    p->n = n;
    p->m = 2 * n;
    p->buf = p->buf2 = p->tw = nullptr;
    p->ghat = nullptr;
    const long long m = p->m, P = n + 1;
    const long long big = m * m * P;  // largest spectrum (the Green's x pass output)
    cudaError_t e = cudaMalloc(&p->buf, big * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->buf2, big * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->tw, m * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->ghat, P * P * P * sizeof(double));
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
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

void fft_plan_free(FftPlan *p) {
    if (p->buf) cudaFree(p->buf);
    if (p->buf2) cudaFree(p->buf2);
    if (p->tw) cudaFree(p->tw);
    if (p->ghat) cudaFree(p->ghat);
    p->buf = p->buf2 = p->tw = nullptr;
    p->ghat = nullptr;
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
    if (src == SRC_ACC)
        BT_LAUNCH(K_FFT_X, s, k_fft_x_fwd<M, SRC_ACC><<<blocks_lines(xpairs, M), FFT_TPB, sm, s>>>(
                                  in, n, nin, nin, p->tw, S1, nullptr));
    else
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
    return cudaGetLastError();
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

cudaError_t solve_acc_to_phi(const FftPlan *p, const unsigned long long *acc_hi,
                             const unsigned long long *acc_lo, double scale, double *phi,
                             cudaStream_t s, const double *scale_dev) {
    XIn in{};
    in.acc_hi = acc_hi;
    in.acc_lo = acc_lo;
    in.scale = scale;
    in.scale_ptr = scale_dev;
    return solve_any(p, in, SRC_ACC, p->n, phi, s);
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
