// Open-boundary Poisson solve on the doubled (Hockney) grid with hand-written
// shared-memory FFTs.
//
// Paper anchor (arXiv:2208.02382, Model Assumptions): the Poisson equation is
// solved in the bunch rest frame with open boundaries.  Reading: phi = G (*) rho
// as an aperiodic convolution, computed as a circular one on the zero-padded
// (2n)^3 grid, where the doubled Green's function holds offset k for k <= n and
// k - 2n above (G is even, so entry k is G(min(k, 2n-k)); offset +-n carries
// the true value).  phi is then exact on nodes -1..n.
//
// Each 1D transform of length m = 2n runs in shared memory: the line is loaded
// in bit-reversed order, then log2(m) in-place radix-2 decimation-in-time
// stages with twiddles exp(-2 pi i j/m) from a table built on the device with
// sincospi.  Lines along x are contiguous; lines along y and z are loaded as
// tiles of TX adjacent x-columns so every global access is a contiguous run.
#include "common.cuh"

namespace bt {

constexpr int FFT_TPB = 256;
constexpr int FFT_LPB = 8;  // x-lines per block
constexpr int FFT_TX = 8;   // x-columns per block for y/z lines

__global__ void k_twiddle(double2 *tw, int m) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m / 2) {
        double s, c;
        sincospi(2.0 * j / m, &s, &c);
        tw[j] = make_double2(c, -s);
    }
}

__device__ __forceinline__ int bitrev(int e, int logm) { return (int)(__brev((unsigned)e) >> (32 - logm)); }

template <bool INV>
__device__ void fft_lines_smem(double2 *s, int m, int nlines, const double2 *__restrict__ tw) {
    const int half = m >> 1;
    for (int hsz = 1; hsz < m; hsz <<= 1) {
        const int tstride = half / hsz;
        for (int t = threadIdx.x; t < nlines * half; t += blockDim.x) {
            int line = t / half, k = t - line * half;
            int j = k & (hsz - 1);
            int i0 = ((k - j) << 1) + j;
            int i1 = i0 + hsz;
            double2 w = tw[j * tstride];
            if (INV) w.y = -w.y;
            double2 *L = s + (size_t)line * m;
            double2 a = L[i0], b = L[i1];
            double2 wb = make_double2(w.x * b.x - w.y * b.y, w.x * b.y + w.y * b.x);
            L[i0] = make_double2(a.x + wb.x, a.y + wb.y);
            L[i1] = make_double2(a.x - wb.x, a.y - wb.y);
        }
        __syncthreads();
    }
}

template <bool INV>
__global__ void k_fft_x(double2 *__restrict__ buf, int m, int logm, const double2 *__restrict__ tw) {
    extern __shared__ double2 sm[];
    const long long line0 = (long long)blockIdx.x * FFT_LPB;
    for (int t = threadIdx.x; t < FFT_LPB * m; t += blockDim.x) {
        int l = t / m, e = t - l * m;
        sm[l * m + bitrev(e, logm)] = buf[(line0 + l) * m + e];
    }
    __syncthreads();
    fft_lines_smem<INV>(sm, m, FFT_LPB, tw);
    for (int t = threadIdx.x; t < FFT_LPB * m; t += blockDim.x) {
        int l = t / m, e = t - l * m;
        buf[(line0 + l) * m + e] = sm[l * m + e];
    }
}

// axis 1: lines along y for fixed z = blockIdx.y; axis 2: lines along z for fixed y.
template <bool INV>
__global__ void k_fft_yz(double2 *__restrict__ buf, int m, int logm, int axis,
                         const double2 *__restrict__ tw) {
    extern __shared__ double2 sm[];
    const long long o = blockIdx.y;
    const int x0 = blockIdx.x * FFT_TX;
    for (int t = threadIdx.x; t < FFT_TX * m; t += blockDim.x) {
        int xl = t % FFT_TX, e = t / FFT_TX;
        long long a = axis == 1 ? ((o * m + e) * m + x0 + xl) : (((long long)e * m + o) * m + x0 + xl);
        sm[xl * m + bitrev(e, logm)] = buf[a];
    }
    __syncthreads();
    fft_lines_smem<INV>(sm, m, FFT_TX, tw);
    for (int t = threadIdx.x; t < FFT_TX * m; t += blockDim.x) {
        int xl = t % FFT_TX, e = t / FFT_TX;
        long long a = axis == 1 ? ((o * m + e) * m + x0 + xl) : (((long long)e * m + o) * m + x0 + xl);
        buf[a] = sm[xl * m + e];
    }
}

__global__ void k_pad_rho(const double *__restrict__ rho, int n, int m, double2 *__restrict__ buf) {
    const long long total = (long long)m * m * m;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx % m), j = (int)((idx / m) % m), l = (int)(idx / ((long long)m * m));
        double v = (i < n && j < n && l < n) ? rho[((long long)l * n + j) * n + i] : 0.0;
        buf[idx] = make_double2(v, 0.0);
    }
}

__global__ void k_mul_real(double2 *__restrict__ buf, const double *__restrict__ g, long long total) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        double2 v = buf[idx];
        double s = g[idx];
        buf[idx] = make_double2(v.x * s, v.y * s);
    }
}

// phi on nodes -1..n: array index k holds node k-1, i.e. doubled index (k-1) mod m.
__global__ void k_extract_phi(const double2 *__restrict__ buf, int n, int m, double scale,
                              double *__restrict__ phi) {
    const int q = n + 2;
    const long long total = (long long)q * q * q;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int a = (int)(idx % q), b = (int)((idx / q) % q), c = (int)(idx / ((long long)q * q));
        int i = (a + m - 1) % m, j = (b + m - 1) % m, l = (c + m - 1) % m;
        phi[idx] = buf[((long long)l * m + j) * m + i].x * scale;
    }
}

__global__ void k_fill_green(const double *__restrict__ g, int n, int m, double2 *__restrict__ buf) {
    const long long total = (long long)m * m * m;
    const int q = n + 1;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int i = (int)(idx % m), j = (int)((idx / m) % m), l = (int)(idx / ((long long)m * m));
        int a = min(i, m - i), b = min(j, m - j), c = min(l, m - l);
        buf[idx] = make_double2(g[((long long)c * q + b) * q + a], 0.0);
    }
}

__global__ void k_take_real(const double2 *__restrict__ buf, double *__restrict__ out, long long total) {
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x)
        out[idx] = buf[idx].x;
}

static int log2i(int m) {
    int l = 0;
    while ((1 << l) < m) ++l;
    return l;
}

static inline int blocks_for(long long total) {
    long long b = (total + FFT_TPB - 1) / FFT_TPB;
    if (b > 148 * 32) b = 148 * 32;
    return (int)b;
}

cudaError_t fft_plan_init(FftPlan *p, int n) {
    p->n = n;
    p->m = 2 * n;
    p->buf = nullptr;
    p->tw = nullptr;
    p->ghat = nullptr;
    const long long m3 = (long long)p->m * p->m * p->m;
    cudaError_t e = cudaMalloc(&p->buf, m3 * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->tw, (p->m / 2) * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(&p->ghat, m3 * sizeof(double));
    if (e != cudaSuccess) {
        fft_plan_free(p);
        return e;
    }
    int smem = (FFT_LPB > FFT_TX ? FFT_LPB : FFT_TX) * p->m * (int)sizeof(double2);
    cudaFuncSetAttribute(k_fft_x<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_fft_x<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_fft_yz<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_fft_yz<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    BT_LAUNCH(K_TWIDDLE, (cudaStream_t)0, k_twiddle<<<(p->m / 2 + 255) / 256, 256>>>(p->tw, p->m));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e;
}

void fft_plan_free(FftPlan *p) {
    if (p->buf) cudaFree(p->buf);
    if (p->tw) cudaFree(p->tw);
    if (p->ghat) cudaFree(p->ghat);
    p->buf = nullptr;
    p->tw = nullptr;
    p->ghat = nullptr;
}

template <bool INV>
static cudaError_t fft3d(const FftPlan *p, cudaStream_t s) {
    const int m = p->m, logm = log2i(m);
    const size_t smx = (size_t)FFT_LPB * m * sizeof(double2);
    const size_t smyz = (size_t)FFT_TX * m * sizeof(double2);
    dim3 gyz(m / FFT_TX, m);
    if (!INV) {
        BT_LAUNCH(K_FFT_X, s, k_fft_x<INV><<<(m * m) / FFT_LPB, FFT_TPB, smx, s>>>(p->buf, m, logm, p->tw));
        BT_LAUNCH(K_FFT_YZ, s, k_fft_yz<INV><<<gyz, FFT_TPB, smyz, s>>>(p->buf, m, logm, 1, p->tw));
        BT_LAUNCH(K_FFT_YZ, s, k_fft_yz<INV><<<gyz, FFT_TPB, smyz, s>>>(p->buf, m, logm, 2, p->tw));
    } else {
        BT_LAUNCH(K_FFT_YZ, s, k_fft_yz<INV><<<gyz, FFT_TPB, smyz, s>>>(p->buf, m, logm, 2, p->tw));
        BT_LAUNCH(K_FFT_YZ, s, k_fft_yz<INV><<<gyz, FFT_TPB, smyz, s>>>(p->buf, m, logm, 1, p->tw));
        BT_LAUNCH(K_FFT_X, s, k_fft_x<INV><<<(m * m) / FFT_LPB, FFT_TPB, smx, s>>>(p->buf, m, logm, p->tw));
    }
    return cudaGetLastError();
}

cudaError_t solve_rho_to_phi(const FftPlan *p, const double *rho, double *phi, cudaStream_t s) {
    const int n = p->n, m = p->m;
    const long long m3 = (long long)m * m * m;
    BT_LAUNCH(K_FFT_PAD, s, k_pad_rho<<<blocks_for(m3), FFT_TPB, 0, s>>>(rho, n, m, p->buf));
    cudaError_t e = fft3d<false>(p, s);
    if (e != cudaSuccess) return e;
    BT_LAUNCH(K_FFT_MUL, s, k_mul_real<<<blocks_for(m3), FFT_TPB, 0, s>>>(p->buf, p->ghat, m3));
    e = fft3d<true>(p, s);
    if (e != cudaSuccess) return e;
    const long long q3 = (long long)(n + 2) * (n + 2) * (n + 2);
    BT_LAUNCH(K_FFT_EXTRACT, s, k_extract_phi<<<blocks_for(q3), FFT_TPB, 0, s>>>(p->buf, n, m, 1.0 / (double)m3, phi));
    return cudaGetLastError();
}

cudaError_t green_spectrum_from_table(const FftPlan *p, const double *gtable, cudaStream_t s) {
    const int n = p->n, m = p->m;
    const long long m3 = (long long)m * m * m;
    BT_LAUNCH(K_GREEN_FILL, s, k_fill_green<<<blocks_for(m3), FFT_TPB, 0, s>>>(gtable, n, m, p->buf));
    cudaError_t e = fft3d<false>(p, s);
    if (e != cudaSuccess) return e;
    BT_LAUNCH(K_GREEN_TAKE, s, k_take_real<<<blocks_for(m3), FFT_TPB, 0, s>>>(p->buf, p->ghat, m3));
    return cudaGetLastError();
}

}  // namespace bt
