// Beam statistics (ABLASTR beam statistics; the paper's FODO and IOTA
// benchmarks check second moments and emittances): means and centred second
// moments.
//
// Both passes read the particles the same way: each block's chunks of 1024
// particles arrive in shared memory by bulk asynchronous copies (TMA), four
// chunks in flight per block, each completing on an mbarrier whose wait is
// bounded in time (plain loads when an array is not 16-byte aligned).  Pass 1
// takes each block's exact per-coordinate extent (min/max of order-preserving
// integer keys).  Pass 2 first reduces those records and derives per
// coordinate a scale 2^k that brings the half-extent below 2^42 and an origin
// R 2^-k (the extent's midpoint rounded to a multiple of 2^-k); it then rounds
// every coordinate to the integer q = round(x 2^k) - R (x 2^k formed exactly
// from the exponent field, no FP64 arithmetic) and forms the exact sums of q
// and of the 21 products q_a q_b, the products from 21-bit limbs (q = qh 2^21
// + ql, s = qh + ql: q_a q_b = qh_a qh_b 2^42 + (s_a s_b - qh_a qh_b - ql_a
// ql_b) 2^21 + ql_a ql_b, three 64-bit sums of 32 x 32 -> 64-bit products).
// One thread takes a whole particle and keeps all 69 sums in registers.  The
// threads' sums are added per block in 128-bit integers, the blocks' by 64-bit
// atomics with carry into a 128-bit total, and the last block converts them
// once: mean = (R + sum q/N) 2^-k, centred second moment = (sum q_a q_b/N -
// (sum q_a/N)(sum q_b/N)) 2^-(k_a + k_b).  Every sum is exact, so the result
// does not depend on particle order or blocking; the only roundings are q's
// (to nearest: at most 2^-43 of the extent) and the final conversions.  No
// state is kept between calls.
#include "common.cuh"
#include "dd.cuh"
#include "tma.cuh"

namespace bt {

constexpr int MOM_TPB = 256;            // one particle per thread and step
constexpr int MOM_CHUNK = 1024;         // particles per staged chunk (48 KB of shared memory)
constexpr int MOM_STAGES = 4;           // chunks in flight per block
constexpr int MOM_NV = 69;              // sums per thread: 21 x 3 pair sums, 6 sums of q
constexpr int MOM_ACC = 2 * MOM_NV + 2; // global 128-bit sums (lo, hi words), block counter, flags
constexpr int MOM_EXT = 16;             // per-block extent record: 6 min keys, 6 max keys, marker
constexpr int MOM_EXT_MAX = 148 * 4;    // extent blocks at most
constexpr unsigned long long MOM_WAIT_NS = 2000000000ull;  // bound of one staging wait: 2 s
constexpr size_t MOM_SMEM = (size_t)MOM_STAGES * 6 * MOM_CHUNK * sizeof(double);
static_assert((size_t)MOM_TPB * MOM_NV * 8 <= MOM_SMEM, "block sums reuse the staging buffers");

// One block per SM (all 69 sums of a particle live in registers).  A thread
// sums at most n / (148 * 256) particles' products below 2^43 (about 2^17 for
// the 5.6e9 particles that fit in memory), far from 2^63.
int moments_blocks(int64_t n) {
    const int64_t chunks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    const int64_t b = chunks < 148 ? chunks : 148;
    return (int)(b < 1 ? 1 : b);
}

// Scratch (as long long): the global sums, then the extent records.
size_t moments_scratch_doubles(int) { return MOM_ACC + (size_t)MOM_EXT_MAX * MOM_EXT; }

__host__ __device__ constexpr int mom_a(int k) {
    constexpr int A[21] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 4, 4, 5};
    return A[k];
}
__host__ __device__ constexpr int mom_b(int k) {
    constexpr int B[21] = {0, 1, 2, 3, 4, 5, 1, 2, 3, 4, 5, 2, 3, 4, 5, 3, 4, 5, 4, 5, 5};
    return B[k];
}

// round(d * 2^s) for |d * 2^s| < 2^62, to nearest, in one of two ways that
// give the same integer except on exact ties (within 1/2 either way):
//
// fix_round_cvt: d 2^s formed exactly by adding s to the exponent field, then
// one hardware conversion to a 64-bit integer (ties to even; FP64 pipe).  A
// value that would fall below the normal range (|d 2^s| < 2^-1022; zeros and
// subnormals) keeps only its sign and low word, a subnormal, which rounds to 0.
__device__ __forceinline__ long long fix_round_cvt(double d, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned hi = (unsigned)(b >> 32);
    const int e = (int)((hi >> 20) & 0x7FF);
    const unsigned hs = (e > 0 && e + s > 0) ? hi + ((unsigned)s << 20) : (hi & 0x80000000u);
    return __double2ll_rn(__hiloint2double((int)hs, (int)(unsigned)b));
}

// fix_round_int: exponent and mantissa arithmetic on the integer pipes, no
// branches (ties away from zero): with the significand m (53 bits) shifted to
// t = m 2^10 < 2^63, |d| 2^s = t 2^-r and the rounded magnitude is
// floor((floor(t 2^-(r-1)) + 1) / 2), which is 0 for r >= 64 (r is limited to
// 64: t 2^-63 < 1); zeros and subnormals take r = 64.
__device__ __forceinline__ long long fix_round_int(double d, int s) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FF);
    const unsigned long long t = ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) << 10;
    const int r1 = e == 0 ? 63 : min(max(1085 - s - e, 1), 64) - 1;
    const unsigned long long v = ((t >> r1) + 1) >> 1;
    const long long sg = (long long)b >> 63;
    return ((long long)v ^ sg) - sg;
}

// Coordinates whose q takes the hardware conversion (bit k for coordinate k);
// the others take the integer pipes, so that both pipes share the work (four
// of six measured fastest: 2.5e7 particles, 0.626 ms against 0.677 with none
// and 0.648 with all six).
#ifndef MOM_CVT_MASK
#define MOM_CVT_MASK 0x0F
#endif
template <int K>
__device__ __forceinline__ long long fix_round_k(double d, int s) {
    if constexpr ((MOM_CVT_MASK >> K) & 1) return fix_round_cvt(d, s);
    else return fix_round_int(d, s);
}

// The six coordinate arrays (indexed with unrolled, compile-time k only).
struct Coords6 {
    const double *p[6];
};

__device__ __forceinline__ void key_minmax(double v, long long &lo, long long &hi) {
    const long long k = dkey(v);
    lo = min(lo, k);
    hi = max(hi, k);
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

// The block's chunks of 1024 particles (chunk blockIdx.x + j gridDim.x for
// j = 0, 1, ...), handed to body(ld, cnt) with ld(k, i) = coordinate k of the
// chunk's particle i.  TMA: chunk j arrives in stage j % 4 of the shared
// buffers by bulk copies of its six rows (the even part of a ragged chunk;
// thread 0 copies its odd last particle), four chunks in flight; thread 0
// refills a stage once every thread is done with it.  pre() runs while the
// first copies are in flight.  Every wait is bounded: if one runs out, the
// timeout goes to *status, the copies still in flight are waited for (bounded
// again) and the result is false.  Not TMA: ld reads global memory.
template <bool TMA, class Pre, class Body>
__device__ __forceinline__ bool staged_chunks(const Coords6 c, int64_t n, double *sbuf,
                                              unsigned long long *bar, unsigned long long wait_ns,
                                              int *status, Pre &&pre, Body &&body) {
    const int tid = threadIdx.x;
    const int64_t nchunks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    const int J = blockIdx.x < nchunks ? (int)((nchunks - 1 - blockIdx.x) / gridDim.x + 1) : 0;
    auto chunk_at = [&](int j) { return (blockIdx.x + (int64_t)j * gridDim.x) * MOM_CHUNK; };
    if constexpr (!TMA) {
        pre();
        for (int j = 0; j < J; ++j) {
            const int64_t b0 = chunk_at(j);
            const int cnt = (int)min((int64_t)MOM_CHUNK, n - b0);
            body([&](int k, int i) { return c.p[k][b0 + i]; }, cnt);
        }
        return true;
    } else {
        auto issue = [&](int j) {                      // thread 0: chunk j into stage j % 4
            const int64_t b0 = chunk_at(j);
            const unsigned bytes = (unsigned)(min((int64_t)MOM_CHUNK, n - b0) & ~1ll) * 8u;
            const int st = j % MOM_STAGES;
            const unsigned b = smem_u32(&bar[st]);
            fence_proxy_async();
            mbar_arrive_expect(b, 6 * bytes);
            if (bytes)
#pragma unroll
                for (int k = 0; k < 6; ++k)
                    bulk_copy_g2s(smem_u32(sbuf + (size_t)(st * 6 + k) * MOM_CHUNK), c.p[k] + b0, bytes, b);
        };
        if (tid == 0) {
            for (int st = 0; st < MOM_STAGES; ++st) mbar_init(smem_u32(&bar[st]), 1);
            fence_proxy_async();
            for (int j = 0; j < min(J, MOM_STAGES); ++j) issue(j);
        }
        __syncthreads();
        pre();
        int j = 0;
        bool ok_all = true;
        for (; j < J; ++j) {
            const int st = j % MOM_STAGES;
            const int64_t b0 = chunk_at(j);
            const int cnt = (int)min((int64_t)MOM_CHUNK, n - b0);
            double *sg = sbuf + (size_t)st * 6 * MOM_CHUNK;
            const bool ok = mbar_wait(smem_u32(&bar[st]), (unsigned)(j / MOM_STAGES) & 1u, wait_ns);
            if (ok && tid == 0 && (cnt & 1))
#pragma unroll
                for (int k = 0; k < 6; ++k) sg[k * MOM_CHUNK + cnt - 1] = c.p[k][b0 + cnt - 1];
            if (__syncthreads_or(!ok)) {
                ok_all = false;
                break;
            }
            body([&](int k, int i) { return sg[k * MOM_CHUNK + i]; }, cnt);
            __syncthreads();                            // every thread is done with stage st
            if (tid == 0 && j + MOM_STAGES < J) issue(j + MOM_STAGES);
        }
        if (!ok_all && tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            for (int jj = j; jj < min(J, j + MOM_STAGES); ++jj)
                mbar_wait(smem_u32(&bar[jj % MOM_STAGES]), (unsigned)(jj / MOM_STAGES) & 1u, wait_ns);
        }
        return ok_all;
    }
}

// Pass 1: each block's exact per-coordinate min/max keys (order-preserving
// integer keys of the doubles) into its extent record, with a completion
// marker (0 if a staging wait ran out).  Block 0 also clears the global sums,
// block counter and flags that pass 2 adds into.
template <bool TMA>
__global__ void __launch_bounds__(MOM_TPB, 1) k_mom_extent(Coords6 c, int64_t n,
                                                           long long *__restrict__ ext,
                                                           long long *__restrict__ acc, int *status,
                                                           unsigned long long wait_ns) {
    if (blockIdx.x == 0 && threadIdx.x < MOM_ACC) acc[threadIdx.x] = 0;
    extern __shared__ __align__(128) double sbuf[];
    __shared__ __align__(8) unsigned long long s_bar[MOM_STAGES];
    __shared__ long long s_lo[6][MOM_TPB / 32], s_hi[6][MOM_TPB / 32];
    long long lo[6], hi[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        lo[k] = LLONG_MAX;
        hi[k] = LLONG_MIN;
    }
    const bool ok = staged_chunks<TMA>(c, n, sbuf, s_bar, wait_ns, status, [] {},
                                       [&](auto ld, int cnt) {
                                           for (int i = threadIdx.x; i < cnt; i += MOM_TPB)
#pragma unroll
                                               for (int k = 0; k < 6; ++k) key_minmax(ld(k, i), lo[k], hi[k]);
                                       });
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
    if (threadIdx.x < 12) {
        const int k = threadIdx.x % 6;
        const bool mx = threadIdx.x >= 6;
        long long v = mx ? s_hi[k][0] : s_lo[k][0];
        for (int w = 1; w < MOM_TPB / 32; ++w) v = mx ? max(v, s_hi[k][w]) : min(v, s_lo[k][w]);
        ext[(size_t)blockIdx.x * MOM_EXT + threadIdx.x] = v;
    }
    if (threadIdx.x == 12) ext[(size_t)blockIdx.x * MOM_EXT + 12] = ok ? 1 : 0;
}

// 128-bit integer to double-double: v = c2 2^86 + c1 2^43 + c0 with c1, c0 in
// [0, 2^43), each part an exact double (hardware 64-bit conversions only).
__device__ __forceinline__ dd i128_to_dd(__int128 v) {
    constexpr long long M43 = (1ll << 43) - 1;
    const double c2 = (double)(long long)(v >> 86);
    const double c1 = (double)((long long)(v >> 43) & M43);
    const double c0 = (double)((long long)v & M43);
    return dd_add_d(two_sum(c2 * 0x1p86, c1 * 0x1p43), c0);
}

// Pass 2.  Prologue (while the first copies are in flight): the extent from
// the extent records, and from it per coordinate the scale 2^k (half-extent
// 2^k < 2^42) and the origin R (the midpoint rounded at 2^-k), or, for a
// coordinate far from its origin relative to its extent or of zero extent,
// the FP64 midpoint itself (q from the FP64 difference, then exact); every
// block derives the same values.  Then every particle's q and its exact sums:
// per pair, with s = qh + ql, the sums of qh_a qh_b, ql_a ql_b and
// K = s_a s_b (three wide products; the cross sum is K - hh - ll).  The
// block's sums, added in 128-bit integers, go into the global sums by 64-bit
// atomics (the low word's wrap carried into the high word: exact in any
// order).  The last block to finish converts them into the 27 moments.
template <bool TMA>
__global__ void __launch_bounds__(MOM_TPB, 1) k_mom_sums(Coords6 c, int64_t n,
                                                         const long long *__restrict__ ext, int next,
                                                         long long *__restrict__ acc, double *out,
                                                         int *status, unsigned long long wait_ns) {
    extern __shared__ __align__(128) double sbuf[];   // [4][6][MOM_CHUNK], then the block sums
    __shared__ __align__(8) unsigned long long s_bar[MOM_STAGES];
    __shared__ long long s_key[13];
    __shared__ int s_sc[6];
    __shared__ long long s_R[6];
    __shared__ double s_mid[6];
    __shared__ unsigned s_flag;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int sc[6];
    long long R[6];
    double mid[6];
    unsigned flag = 0;
    auto pre = [&] {
        for (int k = warp; k < 13; k += MOM_TPB / 32) {   // 6 min keys, 6 max keys, the markers
            const bool is_max = k >= 6 && k < 12;
            long long v = is_max ? LLONG_MIN : LLONG_MAX;
            for (int r = lane; r < next; r += 32) {
                const long long x = ext[(size_t)r * MOM_EXT + k];
                v = is_max ? max(v, x) : min(v, x);
            }
            for (int o = 16; o > 0; o >>= 1) {
                const long long y = __shfl_xor_sync(0xffffffffu, v, o);
                v = is_max ? max(v, y) : min(v, y);
            }
            if (lane == 0) s_key[k] = v;
        }
        __syncthreads();
        if (warp == 0) {
            unsigned f = 0;
            if (tid < 6) {
                const double mn = dkey_inv(s_key[tid]), mx = dkey_inv(s_key[6 + tid]);
                const double m = __dmul_rn(0.5, __dadd_rn(mn, mx));
                const double half = fmax(__dsub_rn(mx, m), __dsub_rn(m, mn));
                int k2 = 0;
                long long r0 = 0;
                if (!(isfinite(m) && isfinite(half))) {
                    f = 1;
                } else {
                    if (half > 0.0) k2 = 42 - (ilogb(half) + 1);   // half 2^k < 2^42
                    if (half == 0.0 || (m != 0.0 && ilogb(m) + k2 >= 60)) f = 2u << tid;
                    else r0 = fix_round_int(m, k2);
                }
                s_sc[tid] = k2;
                s_R[tid] = r0;
                s_mid[tid] = m;
            }
            if (tid == 6 && s_key[12] != 1) f = 1;   // an extent block's wait ran out
            f = __reduce_or_sync(0xffffffffu, f);
            if (tid == 0) s_flag = f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            sc[k] = s_sc[k];
            R[k] = s_R[k];
            mid[k] = s_mid[k];
        }
        flag = s_flag;
    };
    long long hh[21], md[21], ll[21], sq[6];
#pragma unroll
    for (int p = 0; p < 21; ++p) hh[p] = md[p] = ll[p] = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) sq[k] = 0;
    // a particle's q per coordinate, as 21-bit limbs
    struct Limbs {
        int h[6];
        unsigned l[6];
    };
    auto convert = [&](auto ld, int i, auto far_tag) {
        constexpr bool ANYFAR = decltype(far_tag)::value;
        Limbs L;
        auto one = [&](auto kc) {
            constexpr int k = decltype(kc)::value;
            const double v = ld(k, i);
            long long q;
            if constexpr (ANYFAR)
                q = ((flag >> (k + 1)) & 1) ? fix_round_k<k>(v - mid[k], sc[k]) : fix_round_k<k>(v, sc[k]) - R[k];
            else
                q = fix_round_k<k>(v, sc[k]) - R[k];
            sq[k] += q;
            L.h[k] = (int)(q >> 21);
            L.l[k] = (unsigned)q & 0x1FFFFFu;
        };
        one(std::integral_constant<int, 0>{});
        one(std::integral_constant<int, 1>{});
        one(std::integral_constant<int, 2>{});
        one(std::integral_constant<int, 3>{});
        one(std::integral_constant<int, 4>{});
        one(std::integral_constant<int, 5>{});
        return L;
    };
    // its limb products: hh, ll and K = (qh_a + ql_a)(qh_b + ql_b) per pair
    // (|qh + ql| < 2^22, so |K| < 2^44)
    auto accumulate = [&](const Limbs &L) {
        int sl[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) sl[k] = L.h[k] + (int)L.l[k];
#pragma unroll
        for (int p = 0; p < 21; ++p) {
            const int a = mom_a(p), b = mom_b(p);
            hh[p] = mad_wide_s(L.h[a], L.h[b], hh[p]);
            md[p] = mad_wide_s(sl[a], sl[b], md[p]);
            ll[p] = mad_wide_u(L.l[a], L.l[b], ll[p]);
        }
    };
    // two particles per step (twelve independent conversions in flight)
    auto chunk = [&](auto ld, int cnt, auto far_tag) {
        int i = tid;
        for (; i + MOM_TPB < cnt; i += 2 * MOM_TPB) {
            const Limbs L0 = convert(ld, i, far_tag);
            const Limbs L1 = convert(ld, i + MOM_TPB, far_tag);
            accumulate(L0);
            accumulate(L1);
        }
        if (i < cnt) accumulate(convert(ld, i, far_tag));
    };
    const bool ok = staged_chunks<TMA>(c, n, sbuf, s_bar, wait_ns, status, pre, [&](auto ld, int cnt) {
        if (flag & 0x7Eu) chunk(ld, cnt, std::true_type{});
        else chunk(ld, cnt, std::false_type{});
    });
    __shared__ __int128 s_tot[MOM_NV];
    __shared__ int s_last;
    if (ok) {
        // block sums in 128-bit integers: the threads' sums through shared
        // memory (the staging buffers are free: every copy has been waited for)
        __syncthreads();
        long long *s64 = reinterpret_cast<long long *>(sbuf);
#pragma unroll
        for (int p = 0; p < 21; ++p) {
            s64[tid * MOM_NV + 3 * p] = hh[p];
            s64[tid * MOM_NV + 3 * p + 1] = md[p];
            s64[tid * MOM_NV + 3 * p + 2] = ll[p];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) s64[tid * MOM_NV + 63 + k] = sq[k];
        __syncthreads();
        if (tid < MOM_NV) {
            __int128 t0 = 0, t1 = 0, t2 = 0, t3 = 0;    // four chains: loads overlap
            for (int i = 0; i < MOM_TPB; i += 4) {
                t0 += s64[i * MOM_NV + tid];
                t1 += s64[(i + 1) * MOM_NV + tid];
                t2 += s64[(i + 2) * MOM_NV + tid];
                t3 += s64[(i + 3) * MOM_NV + tid];
            }
            const __int128 t = (t0 + t1) + (t2 + t3);
            unsigned long long *g = reinterpret_cast<unsigned long long *>(acc + 2 * tid);
            const unsigned long long lo = (unsigned long long)t;
            const unsigned long long old = atomicAdd(g, lo);
            atomicAdd(g + 1, (unsigned long long)(t >> 64) + (old + lo < old ? 1ull : 0ull));
            __threadfence();
        }
    } else if (tid == 0) {
        atomicOr(reinterpret_cast<unsigned long long *>(acc + 2 * MOM_NV + 1), 1ull);   // incomplete
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) {
        const unsigned long long done =
            atomicAdd(reinterpret_cast<unsigned long long *>(acc + 2 * MOM_NV), 1ull);
        s_last = done == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block: every block's sums are in
    __threadfence();
    if (tid < MOM_NV)
        s_tot[tid] = (__int128)(unsigned long long)__ldcg(acc + 2 * tid) |
                     ((__int128)__ldcg(acc + 2 * tid + 1) << 64);
    __syncthreads();
    if (warp != 0) return;
    __shared__ double s_m[6][2];
    const bool bad = (flag & 1u) || __ldcg(acc + 2 * MOM_NV + 1) != 0;
    const double N = (double)n;
    if (lane < 6) {
        const dd mq = dd_div_d(i128_to_dd(s_tot[63 + lane]), N);   // mean of q
        s_m[lane][0] = mq.hi;
        s_m[lane][1] = mq.lo;
    }
    __syncwarp();
    if (lane < 6) {
        const bool far = (flag >> (lane + 1)) & 1u;
        const dd mq{s_m[lane][0], s_m[lane][1]};
        // origin: R 2^-k, or the FP64 midpoint for a far origin
        const int k2 = s_sc[lane];
        const dd org = far ? dd_make(s_mid[lane]) : dd_scale(i128_to_dd((__int128)s_R[lane]), ldexp(1.0, -k2));
        out[lane] = bad ? NAN : dd_add(org, dd_scale(mq, ldexp(1.0, -k2))).hi;
    } else if (lane < 27) {
        const int k = lane - 6, ia = mom_a(k), ib = mom_b(k);
        // sum q_a q_b = HH 2^42 + (K - HH - LL) 2^21 + LL, exact in 128 bits
        // (|sum| < N 2^84)
        const __int128 HH = s_tot[3 * k], K = s_tot[3 * k + 1], LL = s_tot[3 * k + 2];
        const dd S = i128_to_dd(HH * ((__int128)1 << 42) + (K - HH - LL) * ((__int128)1 << 21) + LL);
        const dd ma{s_m[ia][0], s_m[ia][1]}, mb{s_m[ib][0], s_m[ib][1]};
        const dd v = dd_sub(dd_div_d(S, N), dd_mul(ma, mb));
        out[lane] = bad ? NAN : ldexp(v.hi, -(s_sc[ia] + s_sc[ib]));
    }
}


static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

cudaError_t launch_moments(double *const c[6], int64_t n, double *partials, int nblocks,
                           double *out, int *status, cudaStream_t s) {
    long long *acc = reinterpret_cast<long long *>(partials);
    long long *ext = acc + MOM_ACC;
    Coords6 cc;
    bool al = true;
    for (int k = 0; k < 6; ++k) {
        cc.p[k] = c[k];
        al = al && aligned16(c[k]);
    }
    // staged: one block per SM; plain loads: up to four blocks per SM
    const int64_t chunks = (n + MOM_CHUNK - 1) / MOM_CHUNK;
    const int eb = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, al ? 148 : MOM_EXT_MAX));
    if (al) {
        cudaFuncSetAttribute(k_mom_extent<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MOM_SMEM);
        cudaFuncSetAttribute(k_mom_sums<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MOM_SMEM);
        BT_LAUNCH(K_MOMENTS, s, k_mom_extent<true><<<eb, MOM_TPB, MOM_SMEM, s>>>(cc, n, ext, acc, status,
                                                                                MOM_WAIT_NS));
        BT_LAUNCH(K_MOMENTS, s, k_mom_sums<true><<<nblocks, MOM_TPB, MOM_SMEM, s>>>(cc, n, ext, eb, acc, out,
                                                                                   status, MOM_WAIT_NS));
    } else {
        const size_t sm = (size_t)MOM_TPB * MOM_NV * 8;   // the block sums only
        cudaFuncSetAttribute(k_mom_sums<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        BT_LAUNCH(K_MOMENTS, s, k_mom_extent<false><<<eb, MOM_TPB, 0, s>>>(cc, n, ext, acc, status, MOM_WAIT_NS));
        BT_LAUNCH(K_MOMENTS, s, k_mom_sums<false><<<nblocks, MOM_TPB, sm, s>>>(cc, n, ext, eb, acc, out,
                                                                              status, MOM_WAIT_NS));
    }
    return cudaGetLastError();
}

// Self-test of the bounded staging wait: one block arms a barrier for 16
// bytes of copies that are never issued, waits on it like the moments'
// staging does, and records the timeout in the status word.
__global__ void k_wait_selftest(int *status, unsigned long long wait_ns) {
    __shared__ __align__(8) unsigned long long bar;
    if (threadIdx.x == 0) {
        mbar_init(smem_u32(&bar), 1);
        mbar_arrive_expect(smem_u32(&bar), 16);
    }
    __syncthreads();
    const bool ok = mbar_wait(smem_u32(&bar), 0, wait_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
}

cudaError_t launch_wait_selftest(int *status, double limit_ms, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, (unsigned long long)(limit_ms * 1e6));
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
