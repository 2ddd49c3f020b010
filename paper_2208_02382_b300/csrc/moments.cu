// Beam statistics (ABLASTR beam statistics; the paper's FODO and IOTA
// benchmarks check second moments and emittances): means, then centred second
// moments, each as per-block partial sums over fixed contiguous chunks with a
// fixed shared-memory tree, then a fixed-order sum of the partials, so the
// result is bitwise reproducible for a given particle order.
#include "common.cuh"

namespace bt {

constexpr int MOM_TPB = 256;

int moments_blocks(int64_t n) {
    int64_t b = (n + MOM_TPB * 8 - 1) / (MOM_TPB * 8);
    if (b > 148 * 8) b = 148 * 8;
    return (int)(b < 1 ? 1 : b);
}

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
    for (int64_t p = b0 + threadIdx.x; p < b1; p += MOM_TPB) {
        v[0] += x[p];
        v[1] += px[p];
        v[2] += y[p];
        v[3] += py[p];
        v[4] += t[p];
        v[5] += pt[p];
    }
    block_tree_sum<6>(v, partial + (size_t)blockIdx.x * 6);
}

__global__ void k_mom_cov(const double *__restrict__ x, const double *__restrict__ px,
                          const double *__restrict__ y, const double *__restrict__ py,
                          const double *__restrict__ t, const double *__restrict__ pt, int64_t n,
                          const double *__restrict__ mean, double *__restrict__ partial) {
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b0 = blockIdx.x * chunk, b1 = min(n, b0 + chunk);
    double m[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) m[k] = mean[k];
    double v[21];
#pragma unroll
    for (int k = 0; k < 21; ++k) v[k] = 0.0;
    for (int64_t p = b0 + threadIdx.x; p < b1; p += MOM_TPB) {
        double d[6] = {x[p] - m[0], px[p] - m[1], y[p] - m[2], py[p] - m[3], t[p] - m[4], pt[p] - m[5]};
        int k = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int b = a; b < 6; ++b) v[k++] += d[a] * d[b];
    }
    block_tree_sum<21>(v, partial + (size_t)blockIdx.x * 21);
}

// out[off + k] = (sum over blocks of partial[b*K + k]) / n, in block order.
__global__ void k_mom_final(const double *__restrict__ partial, int nblocks, int K, int64_t n,
                            double *__restrict__ out, int off) {
    int k = threadIdx.x;
    if (k < K) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * K + k];
        out[off + k] = s / (double)n;
    }
}

cudaError_t launch_moments(double *const c[6], int64_t n, double *partials, int nblocks,
                           double *out, cudaStream_t s) {
    BT_LAUNCH(K_MOMENTS, s, k_mom_sum<<<nblocks, MOM_TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, partials));
    BT_LAUNCH(K_MOMENTS, s, k_mom_final<<<1, 32, 0, s>>>(partials, nblocks, 6, n, out, 0));
    BT_LAUNCH(K_MOMENTS, s, k_mom_cov<<<nblocks, MOM_TPB, 0, s>>>(c[0], c[1], c[2], c[3], c[4], c[5], n, out, partials));
    BT_LAUNCH(K_MOMENTS, s, k_mom_final<<<1, 32, 0, s>>>(partials, nblocks, 21, n, out, 6));
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
