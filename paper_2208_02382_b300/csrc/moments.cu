// Beam statistics (ABLASTR beam statistics; the paper's FODO and IOTA
// benchmarks check second moments and emittances): means, then centred second
// moments.
//
// Means: per-block FP64 partial sums over fixed contiguous chunks with a fixed
// shared-memory tree, then a fixed-order sum of the partials (bitwise
// reproducible for a given particle order); the same pass takes each
// coordinate's min and max (order-preserving integer keys).
// Second moments: the 21 sums of d_a d_b (d = coordinate minus its mean) run on
// the integer pipes instead of the FP64 pipe (21 FP64 FMAs a particle were the
// bound): d_c is rounded to an integer at 2^s_c, with s_c chosen from the
// coordinate's extent about its mean and the particle count so that every sum
// of products fits a signed 128-bit integer; the 64x64 -> 128-bit products are
// summed exactly (the sums do not depend on particle order or blocking) and
// converted to double once.  The rounding of d_c (to nearest, unbiased) is at
// most 2^-44 of the extent; summed over the bunch these errors stay far below
// the FP64 sum's own.
#include "common.cuh"

namespace bt {

constexpr int MOM_TPB = 256;
constexpr int MOM_P1 = 18;   // pass-1 partial per block: 6 sums, 6 min keys, 6 max keys
constexpr int MOM_P2 = 42;   // pass-2 partial per block: 21 x (hi, lo) of 128-bit sums

// at most MOM_PPT particles per thread (the per-thread integer sums' bound),
// in whole waves of the second-moment pass (128 registers: two blocks of 256
// threads per SM), so that no wave runs a few long blocks on an idle GPU
constexpr int MOM_PPT = 256;
int moments_blocks(int64_t n) {
    const int64_t resident = 148 * 2;
    const int64_t per = (int64_t)MOM_TPB * MOM_PPT;
    int64_t waves = (n + resident * per - 1) / (resident * per);
    if (waves < 1) waves = 1;
    int64_t b = resident * waves;
    if (b > (n + MOM_TPB - 1) / MOM_TPB) b = (n + MOM_TPB - 1) / MOM_TPB;
    return (int)(b < 1 ? 1 : b);
}

// doubles of scratch the moments need for `nblocks` blocks (pass-2 partials,
// reused by pass 1, plus the per-coordinate scales)
size_t moments_scratch_doubles(int nblocks) { return (size_t)nblocks * MOM_P2 + 8; }

template <int K>
__device__ void block_tree_sum(double (&v)[K], double *out) {
    __shared__ double sm[K][MOM_TPB];
#pragma unroll
    for (int k = 0; k < K; ++k) sm[k][threadIdx.x] = v[k];
    __syncthreads();
    for (int s = MOM_TPB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
#pragma unroll
            for (int k = 0; k < K; ++k) sm[k][threadIdx.x] += sm[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; ++k) out[k] = sm[k][0];
}

__global__ void k_mom_sum(const double *__restrict__ x, const double *__restrict__ px,
                          const double *__restrict__ y, const double *__restrict__ py,
                          const double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                          double *__restrict__ partial) {
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double v[6] = {0, 0, 0, 0, 0, 0};
    long long lo[6], hi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        lo[c] = LLONG_MAX;
        hi[c] = LLONG_MIN;
    }
    for (int64_t p = b0 + threadIdx.x; p < b1; p += MOM_TPB) {
        const double q[6] = {x[p], px[p], y[p], py[p], t[p], pt[p]};
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            v[c] += q[c];
            const long long k = dkey(q[c]);
            lo[c] = min(lo[c], k);
            hi[c] = max(hi[c], k);
        }
    }
    double *out = partial + (size_t)blockIdx.x * MOM_P1;
    block_tree_sum<6>(v, out);
    // min/max keys: warp, then block (exact, any order)
    __shared__ long long sk[12][MOM_TPB / 32];
#pragma unroll
    for (int c = 0; c < 6; ++c)
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = min(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = max(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            sk[c][threadIdx.x >> 5] = lo[c];
            sk[6 + c][threadIdx.x >> 5] = hi[c];
        }
    __syncthreads();
    if (threadIdx.x < 12) {
        long long r = sk[threadIdx.x][0];
        for (int w = 1; w < MOM_TPB / 32; ++w)
            r = threadIdx.x < 6 ? min(r, sk[threadIdx.x][w]) : max(r, sk[threadIdx.x][w]);
        reinterpret_cast<long long *>(out)[6 + threadIdx.x] = r;
    }
}

// Means (a fixed-order reduction of the partials) into out[0..5], and the
// scale exponents s_c into scale[0..5].  One block.
__global__ void __launch_bounds__(MOM_TPB) k_mom_means(const double *__restrict__ partial,
                                                     int nblocks, int64_t n,
                                                     double *__restrict__ out,
                                                     int *__restrict__ scale) {
    // each thread folds blocks t, t + 256, ... (in that order), then a fixed
    // shared-memory tree: the same result for the same partials every time
    __shared__ double ss[6][MOM_TPB];
    __shared__ long long slo[6][MOM_TPB], shi[6][MOM_TPB];
    double v[6] = {0, 0, 0, 0, 0, 0};
    long long lo[6], hi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        lo[c] = LLONG_MAX;
        hi[c] = LLONG_MIN;
    }
    for (int b = threadIdx.x; b < nblocks; b += MOM_TPB) {
        const double *pb = partial + (size_t)b * MOM_P1;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            v[c] += pb[c];
            lo[c] = min(lo[c], reinterpret_cast<const long long *>(pb)[6 + c]);
            hi[c] = max(hi[c], reinterpret_cast<const long long *>(pb)[12 + c]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        ss[c][threadIdx.x] = v[c];
        slo[c][threadIdx.x] = lo[c];
        shi[c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int st = MOM_TPB / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                ss[c][threadIdx.x] += ss[c][threadIdx.x + st];
                slo[c][threadIdx.x] = min(slo[c][threadIdx.x], slo[c][threadIdx.x + st]);
                shi[c][threadIdx.x] = max(shi[c][threadIdx.x], shi[c][threadIdx.x + st]);
            }
        __syncthreads();
    }
    const int c = threadIdx.x;
    if (c >= 6) return;
    // scale exponent s_c: 2^s_c times the extent of coordinate c about its
    // mean stays below 2^43, so a product is below 2^87, a thread's sum of at
    // most 256 of them below 2^95 (its high word fits a signed 32-bit
    // integer), and the sum over up to 2^31 particles below 2^118
    const double mean = ss[c][0] / (double)n;
    out[c] = mean;
    const double ext = fmax(dkey_inv(shi[c][0]) - mean, mean - dkey_inv(slo[c][0]));
    const int B = 43;
    int sc = 0;
    if (ext > 0.0 && isfinite(ext)) sc = B - (ilogb(ext) + 1);  // ext < 2^(ilogb + 1)
    scale[c] = isfinite(mean) && isfinite(ext) ? sc : INT_MIN;
}

// round(d * 2^s) for |d * 2^s| < 2^62, by exponent/mantissa arithmetic on the
// integer pipes (ties away from zero; |d * 2^s| < 1/2 gives 0).
__device__ __forceinline__ long long fix_round(double d, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = e - 1075 + s;  // |d| 2^s = m 2^sh
    unsigned long long v;
    if (e == 0 || sh < -54) v = 0;
    else if (sh >= 0) v = m << min(sh, 9);
    else v = (m + (1ull << (-sh - 1))) >> (-sh);
    return (b >> 63) ? -(long long)v : (long long)v;
}

__device__ __forceinline__ void add128(long long &hi, unsigned long long &lo, long long phi,
                                       unsigned long long plo) {
    const unsigned long long r = lo + plo;
    hi += phi + (r < lo ? 1 : 0);
    lo = r;
}

__global__ void __launch_bounds__(MOM_TPB) k_mom_cov(
    const double *__restrict__ x, const double *__restrict__ px, const double *__restrict__ y,
    const double *__restrict__ py, const double *__restrict__ t, const double *__restrict__ pt,
    int64_t n, const double *__restrict__ mean, const int *__restrict__ scale,
    unsigned long long *__restrict__ partial) {
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double m[6];
    int sc[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        m[k] = mean[k];
        sc[k] = scale[k] == INT_MIN ? 0 : scale[k];
    }
    // per-thread sums: (high 32-bit word, low 64-bit word), at most 256 terms
    int hi32[21];
    unsigned long long alo[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) {
        hi32[k] = 0;
        alo[k] = 0;
    }
    for (int64_t p = b0 + threadIdx.x; p < b1; p += MOM_TPB) {
        const long long f[6] = {fix_round(x[p] - m[0], sc[0]), fix_round(px[p] - m[1], sc[1]),
                                fix_round(y[p] - m[2], sc[2]), fix_round(py[p] - m[3], sc[3]),
                                fix_round(t[p] - m[4], sc[4]), fix_round(pt[p] - m[5], sc[5])};
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b, ++k) {
                const unsigned long long plo = (unsigned long long)f[a] * (unsigned long long)f[b];
                const unsigned long long r = alo[k] + plo;
                hi32[k] += (int)__mul64hi(f[a], f[b]) + (r < alo[k] ? 1 : 0);
                alo[k] = r;
            }
    }
    long long ahi[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) ahi[k] = hi32[k];
    // exact block sum: warp shuffles, then the warps in order
#pragma unroll
    for (int k = 0; k < 21; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            const long long h = __shfl_xor_sync(0xffffffffu, ahi[k], o);
            const unsigned long long l = __shfl_xor_sync(0xffffffffu, alo[k], o);
            add128(ahi[k], alo[k], h, l);
        }
    __shared__ long long sh[21][MOM_TPB / 32];
    __shared__ unsigned long long sl[21][MOM_TPB / 32];
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int k = 0; k < 21; ++k) {
            sh[k][threadIdx.x >> 5] = ahi[k];
            sl[k][threadIdx.x >> 5] = alo[k];
        }
    __syncthreads();
    if (threadIdx.x < 21) {
        long long h = 0;
        unsigned long long l = 0;
        for (int w = 0; w < MOM_TPB / 32; ++w) add128(h, l, sh[threadIdx.x][w], sl[threadIdx.x][w]);
        partial[(size_t)blockIdx.x * MOM_P2 + 2 * threadIdx.x] = (unsigned long long)h;
        partial[(size_t)blockIdx.x * MOM_P2 + 2 * threadIdx.x + 1] = l;
    }
}

// out[6 + k] = (sum over blocks of the 128-bit partial k) 2^-(s_a + s_b) / n,
// one warp per k (exact integer sums: any order).
__global__ void k_mom_cov_final(const unsigned long long *__restrict__ partial, int nblocks,
                                int64_t n, const int *__restrict__ scale,
                                double *__restrict__ out) {
    const int k = blockIdx.x, lane = threadIdx.x;
    long long h = 0;
    unsigned long long l = 0;
    for (int q = lane; q < nblocks; q += 32)
        add128(h, l, (long long)partial[(size_t)q * MOM_P2 + 2 * k], partial[(size_t)q * MOM_P2 + 2 * k + 1]);
    for (int o = 16; o > 0; o >>= 1) {
        const long long hh = __shfl_xor_sync(0xffffffffu, h, o);
        const unsigned long long ll = __shfl_xor_sync(0xffffffffu, l, o);
        add128(h, l, hh, ll);
    }
    if (lane != 0) return;
    int a = 0, r = k;
    while (r >= 6 - a) {
        r -= 6 - a;
        ++a;
    }
    const int b = a + r;
    if (scale[a] == INT_MIN || scale[b] == INT_MIN) {
        out[6 + k] = NAN;
        return;
    }
    const double v = (double)h * 18446744073709551616.0 + (double)l;
    out[6 + k] = ldexp(v, -(scale[a] + scale[b])) / (double)n;
}

cudaError_t launch_moments(double *const c[6], int64_t n, double *partials, int nblocks,
                           double *out, cudaStream_t s) {
    int *scale = reinterpret_cast<int *>(partials + (size_t)nblocks * MOM_P2);
    BT_LAUNCH(K_MOMENTS, s, k_mom_sum<<<nblocks, MOM_TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, partials));
    BT_LAUNCH(K_MOMENTS, s, k_mom_means<<<1, MOM_TPB, 0, s>>>(partials, nblocks, n, out, scale));
    BT_LAUNCH(K_MOMENTS, s, k_mom_cov<<<nblocks, MOM_TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, out, scale,
                                                                    reinterpret_cast<unsigned long long *>(partials)));
    BT_LAUNCH(K_MOMENTS, s, k_mom_cov_final<<<21, 32, 0, s>>>(reinterpret_cast<const unsigned long long *>(partials),
                                                              nblocks, n, scale, out));
    return cudaGetLastError();
}

// Moments (means, then the row-major upper triangle of the centred second
// moments) taken through a linear map of the MapCoef class: mean' = M mean,
// C' = M C M^T.  One thread.
__global__ void k_moments_transform(double *__restrict__ mom, const MapCoef *map) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const MapCoef &c = *map;
    double M[6][6] = {{c.m00, c.m01, 0, 0, 0, c.m05}, {c.m10, c.m11, 0, 0, 0, c.m15},
                      {0, 0, c.m22, c.m23, 0, 0},     {0, 0, c.m32, c.m33, 0, 0},
                      {c.m40, c.m41, 0, 0, 1, c.m45}, {0, 0, 0, 0, 0, 1}};
    double mean[6], C[6][6], T[6][6];
    for (int i = 0; i < 6; ++i) mean[i] = mom[i];
    int k = 6;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) C[i][j] = C[j][i] = mom[k];
    for (int i = 0; i < 6; ++i) {
        double s = 0.0;
        for (int j = 0; j < 6; ++j) s += M[i][j] * mean[j];
        mom[i] = s;
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int l = 0; l < 6; ++l) s += M[i][l] * C[l][j];
            T[i][j] = s;
        }
    k = 6;
    for (int i = 0; i < 6; ++i)
        for (int j = i; j < 6; ++j, ++k) {
            double s = 0.0;
            for (int l = 0; l < 6; ++l) s += T[i][l] * M[j][l];
            mom[k] = s;
        }
}

cudaError_t launch_moments_transform(double *mom, const MapCoef *map, cudaStream_t s) {
    BT_LAUNCH(K_MOMENTS, s, k_moments_transform<<<1, 32, 0, s>>>(mom, map));
    return cudaGetLastError();
}

}  // namespace bt
