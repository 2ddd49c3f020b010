// Charge deposition for callers that cannot allocate device memory.
//
// Some programs that embed this library may not allocate device memory after
// they start: on-line models in an accelerator control loop that set up all
// memory once and then must run with a fixed footprint, or host frameworks
// that own every device allocation through their own pool and forbid stray
// cudaMalloc calls.  bx_deposit needs a context, and creating one allocates
// its scratch.  bx_deposit_noalloc instead keeps the fixed-point accumulators
// of the deposition in a file-scope device array of fixed size that the
// library holds on every GPU that loads it, until the process exits.  The
// caller passes the particles and the output grid; nothing is allocated or
// freed by the call.
//
// Limits and sharing: at most NOALLOC_MAX_NODES = 64^3 grid nodes (n <= 64),
// i.e. 2 x 64^3 x 8 bytes = 4 MiB of accumulators.  Every call on a device
// uses the same array and clears it first, so calls whose work overlaps on
// the GPU (different streams, or host threads without ordering) race and
// corrupt each other's result; order them on one stream.  The first call on a
// device looks up the array's device address (cudaGetSymbolAddress) with that
// device current and caches it; make that first call before any stream
// capture.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace bt {

constexpr int NOALLOC_MAX_N = 64;
constexpr long long NOALLOC_MAX_NODES = (long long)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N;

// hi words of the accumulators, then lo words (same split as the context path)
static __device__ __align__(256) unsigned long long g_noalloc_acc[2 * NOALLOC_MAX_NODES];

namespace {

struct BoxV {
    double lo[3], h[3], inv_h[3];
};

__device__ __forceinline__ unsigned long long na_to_fixed52(double u) {
    unsigned long long b = (unsigned long long)__double_as_longlong(u);
    int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -60 || u <= 0.0) return 0ull;
    unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    return e >= 0 ? (mant << e) : (mant >> (-e));
}

__device__ __forceinline__ unsigned long long na_mulshr52(unsigned long long a,
                                                         unsigned long long b) {
    unsigned long long lo = a * b, hi = __umul64hi(a, b);
    return (hi << 12) | (lo >> 52);
}

// Same arithmetic as the context deposit: CIC weights in unsigned fixed point,
// summed by integer atomics (order-independent).  Particles outside the box
// are skipped.
__global__ void k_deposit_noalloc(const double *__restrict__ x, const double *__restrict__ y,
                                  const double *__restrict__ t, int64_t n, double nbg, BoxV box,
                                  int nn, unsigned long long *__restrict__ acc) {
    unsigned long long *acc_hi = acc, *acc_lo = acc + (long long)nn * nn * nn;
    const unsigned long long one = 1ull << 52;
    const unsigned long long umax = (unsigned long long)(nn - 1) << 52;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        double u[3];
        u[0] = (x[p] - box.lo[0]) * box.inv_h[0];
        u[1] = (y[p] - box.lo[1]) * box.inv_h[1];
        u[2] = (__dmul_rn(nbg, t[p]) - box.lo[2]) * box.inv_h[2];
        int cell[3];
        unsigned long long w[3][2];
        bool outside = false;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            outside |= !(u[d] >= 0.0) || u[d] > (double)(nn - 1) + 1e-6;
            unsigned long long U = na_to_fixed52(u[d]);
            if (U > umax) U = umax;
            unsigned long long i = U >> 52;
            if (i > (unsigned long long)(nn - 2)) i = nn - 2;
            unsigned long long f = U - (i << 52);
            cell[d] = (int)i;
            w[d][0] = one - f;
            w[d][1] = f;
        }
        if (outside) continue;
        const long long base = ((long long)cell[2] * nn + cell[1]) * nn + cell[0];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                unsigned long long wyz = na_mulshr52(w[1][dy], w[2][dz]);
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    unsigned long long v = na_mulshr52(w[0][dx], wyz) >> 1;
                    long long node = base + ((long long)dz * nn + dy) * nn + dx;
                    atomicAdd(&acc_hi[node], v >> DEP_SPLIT);
                    atomicAdd(&acc_lo[node], v & ((1ull << DEP_SPLIT) - 1));
                }
            }
    }
}

__global__ void k_acc_to_rho_noalloc(const unsigned long long *__restrict__ acc, int nn,
                                     double scale, double *__restrict__ rho) {
    const long long nodes = (long long)nn * nn * nn;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        double w = ((double)acc[i] * 2147483648.0 + (double)acc[nodes + i]) * 0x1p-51;
        rho[i] = scale * w;
    }
}

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[256] = {};

}  // namespace

// Looks up (once per device, with that device current) the device address of
// the static accumulator array.
static cudaError_t noalloc_scratch(unsigned long long **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_acc);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = (unsigned long long *)g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace bt

extern "C" int32_t bx_deposit_noalloc(const bx_beam *beam, const double lo[3], const double hi[3],
                                      int32_t n, double *rho, void *stream) {
    using namespace bt;
    if (!beam || !lo || !hi || !rho) return set_noctx_error(BX_BAD_ARG, "NULL argument");
    if (n < 8 || n > NOALLOC_MAX_N || (n & (n - 1)) != 0)
        return set_noctx_error(BX_BAD_ARG,
                               "bx_deposit_noalloc: n must be a power of two in [8, 64] "
                               "(its static scratch holds at most 64^3 nodes)");
    if (beam->n < 0) return set_noctx_error(BX_BAD_ARG, "beam n < 0");
    if (beam->n > 0)
        for (int k = 0; k < 6; ++k)
            if (!beam->coord[k]) return set_noctx_error(BX_BAD_ARG, "beam coordinate pointer is NULL");
    if (!(beam->mass_MeV > 0.0) || !(beam->kinetic_MeV > 0.0) ||
        !(beam->charge_sign == 1.0 || beam->charge_sign == -1.0) ||
        !std::isfinite(beam->bunch_charge_C))
        return set_noctx_error(BX_BAD_ARG, "beam species or charge invalid");
    BoxV b;
    for (int d = 0; d < 3; ++d) {
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return set_noctx_error(BX_BAD_ARG, "box needs finite lo < hi");
        b.lo[d] = lo[d];
        b.h[d] = (hi[d] - lo[d]) / (double)(n - 1);
        b.inv_h[d] = 1.0 / b.h[d];
    }
    unsigned long long *acc = nullptr;
    cudaError_t e = noalloc_scratch(&acc);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    const long long nodes = (long long)n * n * n;
    e = cudaMemsetAsync(acc, 0, 2 * nodes * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    const double gamma = 1.0 + beam->kinetic_MeV / beam->mass_MeV;
    const double bg = std::sqrt(gamma * gamma - 1.0);
    if (beam->n > 0) {
        long long blocks = (beam->n + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        k_deposit_noalloc<<<(int)blocks, 256, 0, s>>>(beam->coord[0], beam->coord[2],
                                                      beam->coord[4], beam->n, -bg, b, n, acc);
    }
    const double q = beam->n > 0 ? beam->charge_sign * std::fabs(beam->bunch_charge_C) /
                                       (double)beam->n
                                 : 0.0;
    const double scale = q / (b.h[0] * b.h[1] * b.h[2]);
    k_acc_to_rho_noalloc<<<(int)((nodes + 255) / 256), 256, 0, s>>>(acc, n, scale, rho);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    return BX_OK;
}
