// Binning of particles by grid brick: a stable counting sort that keeps the
// particles of each brick contiguous, so the fused particle kernel's blocks
// each touch a compact set of cells and accumulate their charge in a
// shared-memory tile.  Stable and deterministic: the order after sorting is a
// fixed function of the order before (ties keep their relative order).
//
//   keys:    brick of each particle's cell (bricks of be^3 cells; be = 8, or
//            n/16 above n = 128, unless the context sets it; at most 16^3
//            bricks), plus a per-chunk brick histogram (chunks of SORT_CHUNK
//            particles)
//   scan:    exclusive prefix over the histograms in brick-major, chunk-minor
//            order -> the destination of each (brick, chunk) run
//   scatter: within a chunk, each particle's rank among the earlier particles
//            of its brick (warp match_any, warps taking turns in order);
//            writes the six coordinates and the id to scratch arrays, which
//            are then copied back over the caller's arrays.
// Cell order (bx_set_binning's cell_order): a first pass keyed by the cell's
// index within its brick writes the scratch arrays, a second (stable) pass
// keyed by the brick writes the caller's arrays back: particles ordered by
// brick and within a brick by cell: consecutive particles share cells and
// field nodes, which the gather's loads find in L1 (the deposit then spreads
// its atomics over the block's particles, particles.cu).
#include <algorithm>

#include "common.cuh"
#include "fixed.cuh"

namespace bt {

constexpr int SORT_TPB = 256;
constexpr int SORT_ROUNDS = 64;
constexpr int SORT_CHUNK = SORT_TPB * SORT_ROUNDS;   // 16384 particles per block
constexpr int SCAN_TILE = 2048;                      // elements per scan block

int sort_brick_edge(int nn, int be_opt) {
    if (be_opt > 0) return be_opt;
    return nn <= 128 ? 8 : nn / 16;
}
int sort_bricks(int nn, int be) {
    int nb = nn / be;
    return nb * nb * nb;
}
bool sort_brick_edge_valid(int nn, int be) {
    return be >= 2 && be <= nn / 2 && (be & (be - 1)) == 0 && sort_bricks(nn, be) <= 4096;
}
int64_t sort_chunks(int64_t n) { return (n + SORT_CHUNK - 1) / SORT_CHUNK; }

// Sort key of a particle: its brick (mode 0) or its cell's index within the
// brick, x fastest (mode 1).
__device__ __forceinline__ int brick_of(double x, double y, double t, double nbg, const Box &b,
                                        int nn, int be, int mode) {
    const double u[3] = {(x - b.lo[0]) * b.inv_h[0], (y - b.lo[1]) * b.inv_h[1],
                         (__dmul_rn(nbg, t) - b.lo[2]) * b.inv_h[2]};
    const int lb = __ffs(be) - 1;   // be is a power of two
    const int nb = nn >> lb;
    int k[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        long long c = (long long)(to_fixed52(u[d]) >> 52);  // outside: clamped
        if (c > nn - 2) c = nn - 2;
        k[d] = mode ? (int)(c & (be - 1)) : (int)(c >> lb);
    }
    return mode ? (k[2] * be + k[1]) * be + k[0] : (k[2] * nb + k[1]) * nb + k[0];
}

__global__ void k_sort_keys(const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ t, int64_t n, double nbg,
                            const Box *__restrict__ box, int nn, int be, int nbricks,
                            int64_t nchunks, int *__restrict__ keys,
                            long long *__restrict__ counts, const int *gate,
                            const double *const *ptrs, int mode) {
    if (gate && *gate == 0) return;
    if (ptrs) {
        x = ptrs[0];
        y = ptrs[2];
        t = ptrs[4];
    }
    extern __shared__ int hist[];
    for (int i = threadIdx.x; i < nbricks; i += SORT_TPB) hist[i] = 0;
    __syncthreads();
    const Box b = *box;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t p = base + r * SORT_TPB + threadIdx.x;
        if (p >= n) break;
        const int k = brick_of(x[p], y[p], t[p], nbg, b, nn, be, mode);
        keys[p] = k;
        atomicAdd(&hist[k], 1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbricks; i += SORT_TPB)
        counts[(long long)i * nchunks + blockIdx.x] = hist[i];
}

// Exclusive scan, three kernels: per-tile sums, scan of the sums, tiles.
__global__ void k_scan_tiles(const long long *__restrict__ in, long long len,
                             long long *__restrict__ sums, const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ long long sm[SORT_TPB];
    const long long b0 = (long long)blockIdx.x * SCAN_TILE;
    long long s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SORT_TPB)
        if (b0 + i < len) s += in[b0 + i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = SORT_TPB / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sm[threadIdx.x] += sm[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = sm[0];
}

__global__ void k_scan_sums(long long *sums, long long nt, const int *gate) {
    if (gate && *gate == 0) return;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        long long run = 0;
        for (long long i = 0; i < nt; ++i) {
            long long v = sums[i];
            sums[i] = run;
            run += v;
        }
    }
}

__global__ void k_scan_apply(const long long *__restrict__ in, long long len,
                             const long long *__restrict__ sums, long long *__restrict__ out,
                             const int *gate) {
    if (gate && *gate == 0) return;
    __shared__ long long sm[SORT_TPB];
    constexpr int PER = SCAN_TILE / SORT_TPB;
    const long long b0 = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * PER;
    long long v[PER], s = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = (b0 + k < len) ? in[b0 + k] : 0;
        s += v[k];
    }
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < SORT_TPB; o <<= 1) {  // inclusive Hillis-Steele
        long long add = threadIdx.x >= o ? sm[threadIdx.x - o] : 0;
        __syncthreads();
        sm[threadIdx.x] += add;
        __syncthreads();
    }
    long long run = sums[blockIdx.x] + sm[threadIdx.x] - s;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (b0 + k < len) out[b0 + k] = run;
        run += v[k];
    }
}

__global__ void k_sort_scatter(const int *__restrict__ keys, const long long *__restrict__ offs,
                               int64_t n, int nbricks, int64_t nchunks,
                               const double *const *__restrict__ src,
                               const long long *__restrict__ id_src,
                               double *const *__restrict__ dst, long long *__restrict__ id_dst,
                               const int *gate, int *__restrict__ dest_out) {
    if (gate && *gate == 0) return;
    extern __shared__ int running[];
    for (int i = threadIdx.x; i < nbricks; i += SORT_TPB) running[i] = 0;
    __shared__ int s_base[SORT_TPB];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
    for (int r = 0; r < SORT_ROUNDS; ++r) {
        const int64_t p = base + r * SORT_TPB + threadIdx.x;
        const bool valid = p < n;
        const int key = valid ? keys[p] : -1 - lane;  // invalid lanes never match valid ones
        const unsigned same = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(same & lt), cnt = __popc(same);
        const int leader = __ffs(same) - 1;
        for (int w = 0; w < SORT_TPB / 32; ++w) {  // warps take turns, in order
            if (warp == w && valid && lane == leader) {
                s_base[threadIdx.x] = running[key];
                running[key] += cnt;
            }
            __syncthreads();
        }
        const int gbase = s_base[(threadIdx.x & ~31) + leader];
        if (valid) {
            const long long d = offs[(long long)key * nchunks + blockIdx.x] + gbase + rank;
#pragma unroll
            for (int c = 0; c < 6; ++c) dst[c][d] = src[c][p];
            id_dst[d] = id_src[p];
            if (dest_out) dest_out[p] = (int)d;
        }
        __syncthreads();
    }
}

// Copy the sorted scratch arrays back over the caller's arrays.
__global__ void k_sort_copy_back(double *const *__restrict__ ptrs, const long long *__restrict__ ids,
                                 long long *__restrict__ id_dst, int64_t n, const int *gate) {
    if (gate && *gate == 0) return;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 6; ++c) ptrs[c][p] = ptrs[6 + c][p];
        id_dst[p] = ids[p];
    }
}

// dev_ptrs (device, 24 pointers) must hold the six coordinate arrays then the
// six scratch arrays, then the same twelve with the halves swapped
// (sort_set_pointers).  With `gate`, every kernel returns at once unless *gate
// is set.
cudaError_t sort_set_pointers(double *const c[6], double *const scratch[6], double **dev_ptrs,
                              cudaStream_t s) {
    double *h[24];
    for (int k = 0; k < 6; ++k) {
        h[k] = h[18 + k] = c[k];
        h[6 + k] = h[12 + k] = scratch[k];
    }
    return cudaMemcpyAsync(dev_ptrs, h, sizeof(h), cudaMemcpyHostToDevice, s);
}

int sort_bins(int nn, int be, bool cell_order) {
    const int nb = sort_bricks(nn, be);
    return cell_order ? std::max(nb, be * be * be) : nb;
}

// One stable counting-sort pass over the keys of `mode` (see brick_of): the
// coordinates named by ptrs[0..5] and ids id_src go to ptrs[6..11] and id_dst.
static cudaError_t sort_pass(int64_t n, double nbg, const Box *box, int nn, int be, int mode,
                             int *keys, long long *counts, long long *offs, long long *sums,
                             const long long *id_src, long long *id_dst, double **ptrs,
                             cudaStream_t s, const int *gate, int *dest_out) {
    const int nb = mode ? be * be * be : sort_bricks(nn, be);
    const int64_t nch = sort_chunks(n);
    const size_t hsm = (size_t)nb * sizeof(int);
    cudaFuncSetAttribute(k_sort_keys, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    cudaFuncSetAttribute(k_sort_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsm);
    const double *const *dp = (const double *const *)ptrs;
    BT_LAUNCH(K_SORT, s, k_sort_keys<<<(unsigned)nch, SORT_TPB, hsm, s>>>(
                             nullptr, nullptr, nullptr, n, nbg, box, nn, be, nb, nch, keys,
                             counts, gate, dp, mode));
    const long long len = (long long)nb * nch;
    const long long nt = (len + SCAN_TILE - 1) / SCAN_TILE;
    BT_LAUNCH(K_SORT, s, k_scan_tiles<<<(unsigned)nt, SORT_TPB, 0, s>>>(counts, len, sums, gate));
    BT_LAUNCH(K_SORT, s, k_scan_sums<<<1, 32, 0, s>>>(sums, nt, gate));
    BT_LAUNCH(K_SORT, s, k_scan_apply<<<(unsigned)nt, SORT_TPB, 0, s>>>(counts, len, sums, offs, gate));
    BT_LAUNCH(K_SORT, s, k_sort_scatter<<<(unsigned)nch, SORT_TPB, hsm, s>>>(
                             keys, offs, n, nb, nch, dp, id_src, (double *const *)(ptrs + 6),
                             id_dst, gate, dest_out));
    return cudaGetLastError();
}

cudaError_t launch_sort(double *const c[6], long long *id, int64_t n, double betagamma,
                        const Box *box, int nn, int be, int *keys, long long *counts,
                        long long *offs, long long *sums, double *const scratch[6],
                        long long *id_scratch, double **dev_ptrs, cudaStream_t s,
                        const int *gate, int *dest_out, bool cell_order) {
    if (n <= 0) return cudaSuccess;
    (void)c;
    (void)scratch;
    if (cell_order && !dest_out) {
        // by cell within brick into the scratch arrays, then (stable) by brick
        // back into the caller's arrays: ordered by brick, then by cell
        cudaError_t e = sort_pass(n, -betagamma, box, nn, be, 1, keys, counts, offs, sums, id,
                                  id_scratch, dev_ptrs, s, gate, nullptr);
        if (e != cudaSuccess) return e;
        return sort_pass(n, -betagamma, box, nn, be, 0, keys, counts, offs, sums, id_scratch, id,
                         dev_ptrs + 12, s, gate, nullptr);
    }
    cudaError_t e = sort_pass(n, -betagamma, box, nn, be, 0, keys, counts, offs, sums, id,
                              id_scratch, dev_ptrs, s, gate, dest_out);
    if (e != cudaSuccess) return e;
    const int cb = (int)((n + 255) / 256) < 148 * 16 ? (int)((n + 255) / 256) : 148 * 16;
    BT_LAUNCH(K_SORT, s, k_sort_copy_back<<<cb, 256, 0, s>>>(dev_ptrs, id_scratch, id, n, gate));
    return cudaGetLastError();
}

}  // namespace bt
