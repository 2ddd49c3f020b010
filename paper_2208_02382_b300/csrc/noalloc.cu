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
// caller passes the particles, the output grid and, optionally, a word for the
// flags of skipped particles; nothing is allocated or freed by the call.
//
// The per-particle arithmetic is the context deposit's (bx_deposit with
// use_box = 1): the same box constants, u = (X - lo)/h, cells and 52-bit
// fractions (cell_frac), fixed-point CIC weights (cic_weights) and the
// same split of the 51-bit weights into the two integer accumulators, so the
// two give bitwise the same charge density.
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

#include "ctx.cuh"
#include "particle_math.cuh"

namespace bt {

constexpr int NOALLOC_MAX_N = 64;
constexpr long long NOALLOC_MAX_NODES = (long long)NOALLOC_MAX_N * NOALLOC_MAX_N * NOALLOC_MAX_N;

// hi words of the accumulators, then lo words (same split as the context path)
static __device__ __align__(256) unsigned long long g_noalloc_acc[2 * NOALLOC_MAX_NODES];

namespace {

// One particle per thread (grid-stride): its cell and weights as the context
// deposit forms them, added to the 8 nodes with 64-bit integer atomics
// (order-independent sums).  Particles outside the box (as the context
// deposit decides it) and particles with a non-finite position are skipped
// and reported in *flags (when given).
template <bool EX>
__global__ void k_deposit_noalloc(const double *__restrict__ x, const double *__restrict__ y,
                                  const double *__restrict__ t, int64_t n, double nbg, Box box,
                                  int nn, unsigned long long *__restrict__ acc,
                                  int32_t *__restrict__ flags) {
    unsigned long long *acc_hi = acc, *acc_lo = acc + (long long)nn * nn * nn;
    bool any_out = false, any_bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const double xp = x[p], yp = y[p], tp = t[p];
        any_bad |= nonfinite_bits(xp) || nonfinite_bits(yp) || nonfinite_bits(tp);
        double u0, u1, u2;
        box_u<EX>(box, nbg, xp, yp, tp, u0, u1, u2);
        int c0, c1, c2;
        unsigned long long F0, F1, F2;
        bool outside = false;
        cell_frac(u0, nn, c0, F0, outside);
        cell_frac(u1, nn, c1, F1, outside);
        cell_frac(u2, nn, c2, F2, outside);
        if (outside) {
            any_out = true;
            continue;
        }
        unsigned long long wc[8];
        cic_weights(F0, F1, F2, wc);
        const long long base = ((long long)c2 * nn + c1) * nn + c0;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    const unsigned long long v = wc[(dz * 2 + dy) * 2 + dx];
                    const long long node = base + ((long long)dz * nn + dy) * nn + dx;
                    atomicAdd(&acc_hi[node], v >> DEP_SPLIT);
                    atomicAdd(&acc_lo[node], v & ((1ull << DEP_SPLIT) - 1));
                }
            }
    }
    if (flags && (any_out || any_bad))
        atomicOr(flags, (any_out ? BX_NOALLOC_OUTSIDE : 0) | (any_bad ? BX_NOALLOC_NONFINITE : 0));
}

// rho[node] = q W / (hx hy hz), W = (hi 2^31 + lo) 2^-51 (the context's conversion).
__global__ void k_acc_to_rho_noalloc(const unsigned long long *__restrict__ acc, int nn, Box box,
                                     double q_macro, double *__restrict__ rho) {
    const long long nodes = (long long)nn * nn * nn;
    const double vol = box.h[0] * box.h[1] * box.h[2];
    const double scale = q_macro / vol;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nodes;
         i += (long long)gridDim.x * blockDim.x) {
        const double w = ((double)acc[i] * 2147483648.0 + (double)acc[nodes + i]) * 0x1p-51;
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
                                      int32_t n, double *rho, int32_t *flags_device,
                                      void *stream) {
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
    for (int d = 0; d < 3; ++d)
        if (!(hi[d] > lo[d]) || !std::isfinite(lo[d]) || !std::isfinite(hi[d]))
            return set_noctx_error(BX_BAD_ARG, "box needs finite lo < hi");
    const Ref r = make_ref(beam);
    const Box b = explicit_box(lo, hi, n, r.bg);
    unsigned long long *acc = nullptr;
    cudaError_t e = noalloc_scratch(&acc);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    cudaStream_t s = (cudaStream_t)stream;
    const long long nodes = (long long)n * n * n;
    e = cudaMemsetAsync(acc, 0, 2 * nodes * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    if (beam->n > 0) {
        long long blocks = (beam->n + 255) / 256;
        if (blocks > 148 * 16) blocks = 148 * 16;
        if (box_far_offset(b))
            k_deposit_noalloc<true><<<(int)blocks, 256, 0, s>>>(
                beam->coord[0], beam->coord[2], beam->coord[4], beam->n, -r.bg, b, n, acc,
                flags_device);
        else
            k_deposit_noalloc<false><<<(int)blocks, 256, 0, s>>>(
                beam->coord[0], beam->coord[2], beam->coord[4], beam->n, -r.bg, b, n, acc,
                flags_device);
    }
    const double q = beam->n > 0 ? r.sign * std::fabs(beam->bunch_charge_C) / (double)beam->n : 0.0;
    k_acc_to_rho_noalloc<<<(int)((nodes + 255) / 256), 256, 0, s>>>(acc, n, b, q, rho);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    return BX_OK;
}
