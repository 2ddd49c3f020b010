// Beam statistics (ABLASTR beam statistics; the paper's FODO and IOTA
// benchmarks check second moments and emittances): means and centred second
// moments.
//
// Pass 1 takes each coordinate's exact extent (min/max of order-preserving
// integer keys, order-free).  From it, per coordinate, a scale 2^k that brings
// the half-extent below 2^42 and an origin R 2^-k (the extent's midpoint
// rounded to a multiple of 2^-k).  Pass 2 rounds every coordinate to the
// integer q = round(x 2^k) - R (integer operations only: no FP64) and forms
// the exact sums of q and of the 21 products q_a q_b, the products from 21-bit
// limbs (q = qh 2^21 + ql: q_a q_b = qh_a qh_b 2^42 + (qh_a ql_b + ql_a qh_b)
// 2^21 + ql_a ql_b, three 64-bit sums of 32 x 32 -> 64-bit products).  Its
// blocks stage chunks of 1024 particles in shared memory with asynchronous
// copies (the next chunk loads while the current one is summed), and each warp
// sums the pairs of one row group of the 6 x 6 matrix.  The blocks' integer
// sums are added in 128-bit integers and converted once: mean = (R + sum q/N)
// 2^-k, centred second moment = (sum q_a q_b/N - (sum q_a/N)(sum q_b/N))
// 2^-(k_a + k_b).  Every sum is exact, so the result does not depend on particle
// order or blocking; the only roundings are q's (at most 2^-43 of the extent)
// and the final conversions.
#include "common.cuh"
#include "dd.cuh"

namespace bt {

constexpr int MOM_TPB = 256;            // eight warps: two per row group of the 6 x 6 matrix
constexpr int MOM_CHUNK = 1024;         // particles per staged chunk (48 KB of shared memory)
constexpr int MOM_REC = 72;             // per-block record: 21 x 3 pair sums, 6 sums of q
constexpr int MOM_HDR = 32;             // scratch header: keys, origins and scales, flags

int moments_blocks(int64_t n) {
    const int64_t chunks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    const int64_t cap = 148 * 2;        // two blocks of 2 x 48 KB per SM
    int64_t b = chunks < cap ? chunks : cap;
    return (int)(b < 1 ? 1 : b);
}

size_t moments_scratch_doubles(int nblocks) { return MOM_HDR + (size_t)nblocks * MOM_REC; }

// The pairs of warp w (of a row group): row 0 (which also sums q), row 1, row 2
// and (5, 5), rows 3 and 4; entry p is pair index mom_k(w, p) in row-major
// upper-triangle order (-1: none).
__host__ __device__ constexpr int mom_np(int w) { return w == 0 ? 6 : 5; }
__host__ __device__ constexpr int mom_k(int w, int p) {
    constexpr int K[4][6] = {{0, 1, 2, 3, 4, 5}, {6, 7, 8, 9, 10, -1}, {11, 12, 13, 14, 20, -1},
                             {15, 16, 17, 18, 19, -1}};
    return K[w][p];
}
__host__ __device__ constexpr int mom_a(int k) {
    constexpr int A[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
    return A[k];
}
__host__ __device__ constexpr int mom_b(int k) {
    constexpr int B[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};
    return B[k];
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

// Coordinate k of the six arrays (a uniform select, no indexed local array).
__device__ __forceinline__ const double *coord6(const double *x, const double *px,
                                                const double *y, const double *py,
                                                const double *t, const double *pt, int k) {
    return k == 0 ? x : k == 1 ? px : k == 2 ? y : k == 3 ? py : k == 4 ? t : pt;
}

// Scratch header (as long long): [0..5] min keys, [6..11] max keys, [12..17]
// scales k, [18..23] origins R, [24..29] the origin's FP64 value (far origins),
// [30] flags (1: a coordinate not finite; 2 << c: coordinate c far from its
// origin relative to its extent, q taken from the FP64 difference).
__global__ void k_mom_init(long long *hdr) {
    if (threadIdx.x < 6) {
        hdr[threadIdx.x] = LLONG_MAX;
        hdr[6 + threadIdx.x] = LLONG_MIN;
    }
}

// Pass 1: exact per-coordinate min/max keys (order-free integer atomics).
__global__ void __launch_bounds__(256) k_mom_extent(
    const double *__restrict__ x, const double *__restrict__ px, const double *__restrict__ y,
    const double *__restrict__ py, const double *__restrict__ t, const double *__restrict__ pt,
    int64_t n, long long *hdr) {
    long long lo[6], hi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        lo[k] = LLONG_MAX;
        hi[k] = LLONG_MIN;
    }
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; p + 3 * stride < n; p += 4 * stride) {   // four particles' loads in flight
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double *c = coord6(x, px, y, py, t, pt, k);
            const long long k0 = dkey(c[p]), k1 = dkey(c[p + stride]), k2 = dkey(c[p + 2 * stride]),
                            k3 = dkey(c[p + 3 * stride]);
            lo[k] = min(lo[k], min(min(k0, k1), min(k2, k3)));
            hi[k] = max(hi[k], max(max(k0, k1), max(k2, k3)));
        }
    }
    for (; p < n; p += stride)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const long long kk = dkey(coord6(x, px, y, py, t, pt, k)[p]);
            lo[k] = min(lo[k], kk);
            hi[k] = max(hi[k], kk);
        }
    __shared__ long long s_lo[6][8], s_hi[6][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = min(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = max(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
        if (lane == 0) {
            s_lo[k][warp] = lo[k];
            s_hi[k][warp] = hi[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        long long a = s_lo[threadIdx.x][0], b = s_hi[threadIdx.x][0];
        for (int w = 1; w < 8; ++w) {
            a = min(a, s_lo[threadIdx.x][w]);
            b = max(b, s_hi[threadIdx.x][w]);
        }
        atomicMin(&hdr[threadIdx.x], a);
        atomicMax(&hdr[6 + threadIdx.x], b);
    }
}

// Scales and origins from the extents (one thread per coordinate).
__global__ void k_mom_prep(long long *hdr) {
    const int c = threadIdx.x;
    if (c == 0) hdr[30] = 0;
    __syncwarp();
    if (c >= 6) return;
    const double mn = dkey_inv(hdr[c]), mx = dkey_inv(hdr[6 + c]);
    const double mid = __dmul_rn(0.5, __dadd_rn(mn, mx));
    const double half = fmax(__dsub_rn(mx, mid), __dsub_rn(mid, mn));
    int sc = 0;
    long long flag = 0, R = 0;
    if (!(isfinite(mid) && isfinite(half))) {
        flag = 1;
    } else {
        if (half > 0.0) sc = 42 - (ilogb(half) + 1);   // half 2^sc < 2^42
        if (mid != 0.0 && ilogb(mid) + sc >= 60) flag = 2ll << c;   // far origin: FP64 difference
        else R = fix_round(mid, sc);
    }
    hdr[12 + c] = sc;
    hdr[18 + c] = R;
    hdr[24 + c] = __double_as_longlong(mid);
    if (flag) atomicOr(reinterpret_cast<unsigned long long *>(&hdr[30]), (unsigned long long)flag);
}

// acc + a b for 32-bit a, b and a 64-bit accumulator: one wide multiply-add
// (signed, and unsigned for the low limbs).
__device__ __forceinline__ long long mad_wide_s(int a, int b, long long acc) {
    long long d;
    asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(acc));
    return d;
}
__device__ __forceinline__ long long mad_wide_u(unsigned a, unsigned b, long long acc) {
    long long d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(acc));
    return d;
}

__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Pass 2.  The block's j-th chunk (chunk blockIdx.x + j gridDim.x) goes to
// buffer j & 1; the six coordinate rows of 1024 doubles are copied
// asynchronously (the next chunk's copies run while this one is summed),
// converted in place to q, then summed.
__global__ void __launch_bounds__(MOM_TPB, 2) k_mom_sums(
    const double *__restrict__ x, const double *__restrict__ px, const double *__restrict__ y,
    const double *__restrict__ py, const double *__restrict__ t, const double *__restrict__ pt,
    int64_t n, const long long *__restrict__ hdr, long long *__restrict__ rec) {
    extern __shared__ double sbuf[];                 // [2][6][MOM_CHUNK]
    __shared__ int s_sc[6];
    __shared__ long long s_R[6];
    __shared__ double s_mid[6];
    __shared__ long long s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, grp = warp & 3, half = warp >> 2;
    if (tid < 6) {
        s_sc[tid] = (int)hdr[12 + tid];
        s_R[tid] = hdr[18 + tid];
        s_mid[tid] = __longlong_as_double(hdr[24 + tid]);
    }
    if (tid == 0) s_flag = hdr[30];
    const int64_t nchunks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    auto issue = [&](int64_t ch, int j) {
        if (ch < nchunks) {
            const int64_t b0 = ch * MOM_CHUNK;
            const int cnt = (int)min((int64_t)MOM_CHUNK, n - b0);
            double *buf = sbuf + (size_t)(j & 1) * 6 * MOM_CHUNK;
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const double *src = coord6(x, px, y, py, t, pt, k) + b0;
                for (int i = tid; i < cnt; i += MOM_TPB) cp_async8(buf + k * MOM_CHUNK + i, src + i);
            }
        }
        cp_async_commit();
    };
    // per-lane exact sums over all of the block's chunks (a lane sums at most
    // 2^11 products below 2^43 per chunk share: far from 2^63)
    constexpr int NPMAX = 6;
    long long hh[NPMAX], mid[NPMAX], ll[NPMAX], sq[6];
#pragma unroll
    for (int p = 0; p < NPMAX; ++p) hh[p] = mid[p] = ll[p] = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) sq[k] = 0;
    issue(blockIdx.x, 0);
    __syncthreads();
    const long long flag = s_flag;
    int j = 0;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++j) {
        issue(ch + gridDim.x, j + 1);          // the next chunk, into the other buffer
        cp_async_wait<1>();                     // this chunk's copies are done
        __syncthreads();
        const int64_t b0 = ch * MOM_CHUNK;
        const int cnt = (int)min((int64_t)MOM_CHUNK, n - b0);
        double *buf = sbuf + (size_t)(j & 1) * 6 * MOM_CHUNK;
        long long *q = reinterpret_cast<long long *>(buf);
        // coordinates to integers, in place
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int sc = s_sc[k];
            const bool far = (flag >> (k + 1)) & 1;
            const long long R = s_R[k];
            const double m = s_mid[k];
            for (int i = tid; i < cnt; i += MOM_TPB) {
                const double v = buf[k * MOM_CHUNK + i];
                q[k * MOM_CHUNK + i] = far ? fix_round(v - m, sc) : fix_round(v, sc) - R;
            }
        }
        __syncthreads();
        // warp (grp, half): the pairs of row group grp over half the chunk
        const int i0 = half * (MOM_CHUNK / 2), i1 = min(cnt, i0 + MOM_CHUNK / 2);
        for (int i = i0 + lane; i < i1; i += 32) {
            int qh[6], ql[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const long long v = q[k * MOM_CHUNK + i];
                qh[k] = (int)(v >> 21);
                ql[k] = (int)(v & 0x1FFFFF);
                if (grp == 0) sq[k] += v;
            }
            switch (grp) {
#define MOM_ROWS(W)                                                              \
    case W:                                                                      \
        _Pragma("unroll") for (int p = 0; p < mom_np(W); ++p) {                  \
            const int a = mom_a(mom_k(W, p)), b = mom_b(mom_k(W, p));            \
            hh[p] = mad_wide_s(qh[a], qh[b], hh[p]);                             \
            mid[p] = mad_wide_s(ql[a], qh[b], mad_wide_s(qh[a], ql[b], mid[p])); \
            ll[p] = mad_wide_u((unsigned)ql[a], (unsigned)ql[b], ll[p]);         \
        }                                                                        \
        break;
                MOM_ROWS(0)
                MOM_ROWS(1)
                MOM_ROWS(2)
                MOM_ROWS(3)
#undef MOM_ROWS
            }
        }
        __syncthreads();                        // the buffer is free for the chunk after next
    }
    cp_async_wait<0>();
    // warp sums (each below 2^62), then the two warps of a row group add theirs
    __shared__ long long s_rec[2][MOM_REC];
#pragma unroll
    for (int p = 0; p < NPMAX; ++p)
        for (int o = 16; o > 0; o >>= 1) {
            hh[p] += __shfl_xor_sync(0xffffffffu, hh[p], o);
            mid[p] += __shfl_xor_sync(0xffffffffu, mid[p], o);
            ll[p] += __shfl_xor_sync(0xffffffffu, ll[p], o);
        }
#pragma unroll
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) sq[k] += __shfl_xor_sync(0xffffffffu, sq[k], o);
    if (lane == 0) {
        for (int p = 0; p < mom_np(grp); ++p) {
            const int kk = grp == 0 ? mom_k(0, p) : grp == 1 ? mom_k(1, p) : grp == 2 ? mom_k(2, p) : mom_k(3, p);
            s_rec[half][3 * kk] = hh[p];
            s_rec[half][3 * kk + 1] = mid[p];
            s_rec[half][3 * kk + 2] = ll[p];
        }
        if (grp == 0)
            for (int k = 0; k < 6; ++k) s_rec[half][63 + k] = sq[k];
    }
    __syncthreads();
    if (tid < 69) rec[(size_t)blockIdx.x * MOM_REC + tid] = s_rec[0][tid] + s_rec[1][tid];
}

// 128-bit integer to double-double.
__device__ __forceinline__ dd i128_to_dd(__int128 v) {
    const double hi = (double)v;
    const double lo = (double)(v - (__int128)hi);
    return fast_two_sum(hi, lo);
}

// The blocks' records added in 128-bit integers (exact), then the 27 moments
// (one warp; lane j < 27 takes output j).
__global__ void k_mom_final(const long long *__restrict__ hdr, const long long *__restrict__ rec,
                            int nblocks, int64_t n, double *__restrict__ out) {
    const int lane = threadIdx.x;
    __shared__ double s_m[6][2];
    __int128 a = 0, b = 0, c = 0;               // sum q (lanes < 6) or HH, MID, LL
    if (lane < 27)
        for (int blk = 0; blk < nblocks; ++blk) {
            const long long *r = rec + (size_t)blk * MOM_REC;
            if (lane < 6) {
                a += r[63 + lane];
            } else {
                const int k = lane - 6;
                a += r[3 * k];
                b += r[3 * k + 1];
                c += r[3 * k + 2];
            }
        }
    const bool bad = (hdr[30] & 1) != 0;
    const double N = (double)n;
    if (lane < 6) {
        const dd mq = dd_div_d(i128_to_dd(a), N);            // mean of q
        s_m[lane][0] = mq.hi;
        s_m[lane][1] = mq.lo;
    }
    __syncwarp();
    if (lane < 6) {
        const int sc = (int)hdr[12 + lane];
        const bool far = (hdr[30] >> (lane + 1)) & 1;
        const dd mq{s_m[lane][0], s_m[lane][1]};
        // origin: R 2^-k, or the FP64 midpoint for a far origin
        const dd org = far ? dd_make(__longlong_as_double(hdr[24 + lane]))
                           : dd_scale(i128_to_dd((__int128)hdr[18 + lane]), ldexp(1.0, -sc));
        out[lane] = bad ? NAN : dd_add(org, dd_scale(mq, ldexp(1.0, -sc))).hi;
    } else if (lane < 27) {
        const int k = lane - 6, ia = mom_a(k), ib = mom_b(k);
        const int sa = (int)hdr[12 + ia], sb = (int)hdr[12 + ib];
        // sum q_a q_b = HH 2^42 + MID 2^21 + LL
        const dd S = dd_add(dd_scale(i128_to_dd(a), 0x1p42),
                            dd_add(dd_scale(i128_to_dd(b), 0x1p21), i128_to_dd(c)));
        const dd ma{s_m[ia][0], s_m[ia][1]}, mb{s_m[ib][0], s_m[ib][1]};
        const dd v = dd_sub(dd_div_d(S, N), dd_mul(ma, mb));
        out[lane] = bad ? NAN : ldexp(v.hi, -(sa + sb));
    }
}

cudaError_t launch_moments(double *const c[6], int64_t n, double *partials, int nblocks,
                           double *out, cudaStream_t s) {
    long long *hdr = reinterpret_cast<long long *>(partials);
    long long *rec = hdr + MOM_HDR;
    const size_t sm = (size_t)2 * 6 * MOM_CHUNK * sizeof(double);
    cudaFuncSetAttribute(k_mom_sums, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int eb = (int)((n + 255) / 256);
    if (eb > 148 * 8) eb = 148 * 8;
    if (eb < 1) eb = 1;
    BT_LAUNCH(K_MOMENTS, s, k_mom_init<<<1, 32, 0, s>>>(hdr));
    BT_LAUNCH(K_MOMENTS, s, k_mom_extent<<<eb, 256, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, hdr));
    BT_LAUNCH(K_MOMENTS, s, k_mom_prep<<<1, 32, 0, s>>>(hdr));
    BT_LAUNCH(K_MOMENTS, s, k_mom_sums<<<nblocks, MOM_TPB, sm, s>>>(c[0], c[1], c[2], c[3], c[4],
                                                                     c[5], n, hdr, rec));
    BT_LAUNCH(K_MOMENTS, s, k_mom_final<<<1, 32, 0, s>>>(hdr, rec, nblocks, n, out));
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
