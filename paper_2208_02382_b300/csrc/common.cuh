// Internal declarations shared by the CUDA translation units of libbeamtrack.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "beamtrack.h"

namespace bt {

// Device status word bits (read by bx_sync).
enum : int32_t { ST_NONFINITE = 1, ST_TIMEOUT = 2, ST_OUTSIDE = 4 };

// Linear map with the structure shared by drift, quadrupole and sector bend
// and closed under composition (pt is unchanged, t enters its own row with
// coefficient 1, y decouples).  In the per-call map table the three padding
// slots carry the kick factors of the slice (transverse, longitudinal) and the
// map's structure class:
//   x'  = m00 x + m01 px + m05 pt        y'  = m22 y + m23 py
//   px' = m10 x + m11 px + m15 pt        py' = m32 y + m33 py
//   t'  = t + m40 x + m41 px + m45 pt    pt' = pt
struct MapCoef {
    double m00, m01, m05, m10, m11, m15, m22, m23, m32, m33, m40, m41, m45;
    double kick_t, kick_z, kind;
    double aux;   // kind MAP_SPLIT: offset, in entries, from this entry to its SplitRec
};

// Map structure classes (see MapCoef): drift (x += m01 px, y += m23 py,
// t += m45 pt), no dispersion (2x2 blocks and the t-pt term), general;
// MAP_BEND: general in x, px, t with a drift in y (y += m23 py, py unchanged:
// the merged half maps inside a sector bend); MAP_TABLE selects the per-call
// table in the particle kernels; MAP_SPLIT (stored kind only): two linear parts
// with thin multipoles between them, in the entry's SplitRec.
enum MapKind { MAP_NONE = 0, MAP_DRIFT = 1, MAP_QUAD = 2, MAP_GENERAL = 3, MAP_TABLE = 4,
               MAP_SPLIT = 5, MAP_BEND = 6 };

// Thin multipoles of orders 1..MP_MAX: kick polynomial terms z^0..z^(MP_MAX-1).
constexpr int MP_MAX = 12;
static_assert(MP_MAX == BX_MULTIPOLE_MAX_ORDER, "multipole orders of the ABI");

// A map-table entry with thin multipoles at the slice boundary inside it:
// z -> after(N(before(z))) with the thin kick N: px -= Re P, py += Im P,
// P = sum_{j < nc} (cr[j] + i ci[j]) (x + i y)^j (all multipoles at that
// boundary summed: their kicks depend on x, y only, so they commute with each
// other and with the linear thin elements there, which `after` holds).
struct SplitRec {
    MapCoef before, after;
    double nc;
    double cr[MP_MAX], ci[MP_MAX];
};
// table entries (MapCoef units) one SplitRec takes, appended after the entries
constexpr int SPLIT_UNITS = (int)((sizeof(SplitRec) + sizeof(MapCoef) - 1) / sizeof(MapCoef));

// Pre-scaled field at a node (momentum change per unit CIC weight) in int64
// fixed point: E_fix = rint(E * 2^e_d) per component (exponents kept
// separately), so the interpolation runs on the integer pipes; padded to 32
// bytes so that a node's x, y components are one aligned 16-byte load.
struct __align__(32) EFix {
    long long x, y, z, w;
};

// Grid box as the kernels read it (device resident for tracking).
// off = -lo * (1/h) and tz = -(beta gamma) * (1/h_z) are the per-box constants
// of u = X * (1/h) + off (Z = -beta gamma t: u_z = t * tz + off_z), formed once
// per box rule (or per explicit box) instead of in every particle thread.
struct Box {
    double lo[3], hi[3], h[3], inv_h[3];
    double off[3], tz;
};

__host__ __device__ inline void box_finish(Box &b, double nbg) {
    for (int d = 0; d < 3; ++d) b.off[d] = -b.lo[d] * b.inv_h[d];
    b.tz = nbg * b.inv_h[2];
}

// Tracking state kept on the device between kicks.
struct TrackState {
    Box box;
    long long mm[6];        // order-preserving keys of min X,Y,Z then max X,Y,Z
    int32_t has_box;        // a box exists
    int32_t regrid;         // the box rule made a new box at the last decision
    int32_t green_stale;    // h differs from the h of the current Green's function
    int32_t pad;
    double green_h[3];      // h the Green's function spectrum was built for
    long long kick;         // kick counter (since creation / reset)
    long long nlog;         // regrid log length
    // Device-driven tracking: the box rule of each kick sets these gates,
    // which the later kernels of the kick read (a gated kernel whose gate is
    // 0 returns at once), so a call needs no host decision between kicks.
    int32_t k_in_call;      // kick index within the current bx_track call
    int32_t nkicks_call;    // kicks in the call
    int32_t deposit_gate;   // deposit the current positions (first kick or new box)
    int32_t sort_gate;      // re-bin the particles now
    int32_t next_gate;      // a next kick follows in this call (deposit for it)
    int32_t exact_u;        // box far from the origin: u = (X - lo)/h unfused
    int32_t sort_interval;  // kicks between re-binning (0: never)
    int32_t halt;           // non-finite box: skip the space-charge work
    double q_macro;         // macroparticle charge [C]
    double rho_scale;       // q_macro / (hx hy hz)
    double nbg;             // -beta gamma of the beam being tracked
    // Differentiation runs (null otherwise; indexed by the kick counter):
    Box *box_hist;          // the box of every kick is recorded here
    const Box *box_replay;  // the box of every kick is taken from here
    int32_t *slot_hist;     // index of the Green's function build in use
    int32_t green_builds;   // Green's function builds so far
    int32_t pro_dep;        // the call's prologue deposited into the box kept from before
};

// Order-preserving map between doubles and signed 64-bit keys (monotone for
// all non-NaN values), used for exact, order-free min/max with integer atomics.
__host__ __device__ __forceinline__ long long dkey(double v) {
    long long b;
    memcpy(&b, &v, 8);
    return b >= 0 ? b : (b ^ 0x7FFFFFFFFFFFFFFFLL);
}
__host__ __device__ __forceinline__ double dkey_inv(long long k) {
    long long b = k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFLL);
    double v;
    memcpy(&v, &b, 8);
    return v;
}

// Fixed-point deposit: CIC weights carry 51 fractional bits; the global
// accumulator splits each value into hi (bits >= 31) and lo (bits < 31) so
// neither 64-bit sum can overflow for fewer than 2^32 contributions of < 2^62.
constexpr int DEP_FRAC_BITS = 51;
constexpr int DEP_SPLIT = 31;

// ---- kernel-level profiler (profile.cu) -----------------------------------
// Every kernel launch goes through BT_LAUNCH, which counts launches per kernel
// and, when timing is on for the calling context, brackets the launch with a
// pair of CUDA events on the launch stream.
enum KernelId : int {
    K_PUSH, K_MINMAX, K_BOX, K_IGF_CORNER, K_IGF_SUM, K_DEPOSIT, K_ACC_TO_RHO, K_FFT_X,
    K_FFT_YZ, K_FFT_ZSOLVE, K_FFT_XINV, K_GREEN_X, K_GREEN_YZ, K_FIELD, K_GATHER, K_MOMENTS,
    K_TWIDDLE, K_EFIX, K_SORT, K_ADJ_PART, K_ADJ_GRID, K_ZERO, K_REDEPOSIT, K_COUNT
};

struct Profiler;
const char *kernel_name(int id);
void prof_begin(int id, cudaStream_t s);
void prof_end(int id, cudaStream_t s);
Profiler *profiler_new();
bool profiler_timing(const Profiler *p);
void profiler_free(Profiler *p);
void profiler_enable(Profiler *p, bool on);
cudaError_t profiler_read(Profiler *p, double *ms, long long *launches, int cap);
// Makes `p` the profiler of the calling thread for the current scope.
struct ProfScope {
    explicit ProfScope(Profiler *p);
    ~ProfScope();
    Profiler *prev;
};

#define BT_LAUNCH(id, s, ...)               \
    do {                                     \
        ::bt::prof_begin((id), (s));         \
        __VA_ARGS__;                         \
        ::bt::prof_end((id), (s));           \
    } while (0)

// Records `msg` as the error text returned by bx_last_error(NULL) and returns
// `code` (for entry points that take no context).
int32_t set_noctx_error(int32_t code, const char *msg);

// ---- launchers (defined in the .cu files) --------------------------------
// particles.cu
cudaError_t launch_push_maps(double *const c[6], int64_t n, const MapCoef *maps, int nmaps,
                             cudaStream_t s, int32_t *status, TrackState *st = nullptr,
                             double betagamma = 0.0);
cudaError_t launch_minmax(double *const c[6], int64_t n, double betagamma, TrackState *st,
                          int32_t *status, cudaStream_t s);
cudaError_t launch_deposit(double *const c[6], int64_t n, double betagamma, const Box *box,
                           const Box &box_host, int nn, unsigned long long *acc_hi,
                           unsigned long long *acc_lo, int32_t *status, cudaStream_t s, int shape = 1);
cudaError_t launch_acc_to_rho(const unsigned long long *acc_hi, const unsigned long long *acc_lo,
                              int nn, double q_macro, const Box *box, double *rho,
                              cudaStream_t s);
cudaError_t launch_kick_push_deposit(double *const c[6], int64_t n, double betagamma,
                                     const Box *box, const Box &box_host, int nn, const EFix *ef,
                                     const int *escale,
                                     const MapCoef *map_host, bool deposit,
                                     unsigned long long *acc_hi, unsigned long long *acc_lo,
                                     TrackState *st, int32_t *status, cudaStream_t s, int shape = 1);
cudaError_t launch_box_rule(TrackState *st, int nn, int64_t n, long long *log, int64_t log_cap,
                            bool advance, cudaStream_t s);
cudaError_t launch_field(const double *phi, int nn, const Box *box, double kx, double ky,
                         double kz, unsigned long long *emax, EFix *efix, int *escale,
                         cudaStream_t s, const TrackState *st = nullptr,
                         const MapCoef *maps = nullptr);
cudaError_t launch_call_init(TrackState *st, int nkicks, double q_macro, int sort_interval,
                             long long kick0, cudaStream_t s, double betagamma,
                             bool fused_prologue = false);
// First half map of a tracking call (table entry 0) with the min/max keys and,
// when a box was kept from the previous call, the first kick's deposit into it.
// `cells` (3 n, or null): the deposits store each particle's cells there and
// the gather of the same kick reads them instead of recomputing them.
cudaError_t launch_track_prologue(double *const c[6], int64_t n, double betagamma, const Box *box,
                                  int nn, const MapCoef *maps, unsigned long long *acc_hi,
                                  unsigned long long *acc_lo, TrackState *st, int32_t *status,
                                  cudaStream_t s, int shape, unsigned long long *cells = nullptr,
                                  const MapCoef *map0 = nullptr);
cudaError_t launch_zero_acc(unsigned long long *a, unsigned long long *b, int nn, const int *gate,
                            cudaStream_t s);
cudaError_t launch_track_particles(double *const c[6], int64_t n, double betagamma,
                                   const Box *box, int nn, const EFix *ef, const int *escale,
                                   const MapCoef *maps, unsigned long long *acc_hi,
                                   unsigned long long *acc_lo, TrackState *st, int32_t *status,
                                   cudaStream_t s, int part = 3, int shape = 1,
                                   unsigned long long *cells = nullptr, bool spread = false);
cudaError_t launch_box_rule_graph(TrackState *st, int nn, long long *log, int64_t cap,
                                  cudaGraphConditionalHandle hg, cudaGraphConditionalHandle hs,
                                  cudaGraphConditionalHandle hd, cudaGraphConditionalHandle hn,
                                  cudaStream_t s, cudaGraphConditionalHandle hl = 0,
                                  bool has_loop = false);
cudaError_t launch_state_reset(TrackState *st, int nkicks, double q_macro, int sort_interval,
                               cudaStream_t s, double betagamma);
cudaError_t launch_track_particles_oop(double *const cin[6], double *const cout[6], int64_t n,
                                       double betagamma, const Box *box, int nn, const EFix *ef,
                                       const int *escale, const MapCoef *maps,
                                       unsigned long long *acc_hi, unsigned long long *acc_lo,
                                       TrackState *st, int32_t *status, cudaStream_t s, int shape = 1);
cudaError_t launch_track_deposit(double *const c[6], int64_t n, double betagamma, const Box *box,
                                 int nn, unsigned long long *acc_hi, unsigned long long *acc_lo,
                                 TrackState *st, int32_t *status, cudaStream_t s, int shape = 1,
                                 unsigned long long *cells = nullptr, bool spread = false);
int map_kind(const MapCoef &m);
// sort.cu
int sort_brick_edge(int nn, int be_opt);
bool sort_brick_edge_valid(int nn, int be);
cudaError_t sort_set_pointers(double *const c[6], double *const scratch[6], double **dev_ptrs,
                              cudaStream_t s);
int sort_bricks(int nn, int be);
int64_t sort_chunks(int64_t n);
cudaError_t launch_sort(double *const c[6], long long *id, int64_t n, double betagamma,
                        const Box *box, int nn, int be, int *keys, long long *counts,
                        long long *offs, long long *sums, double *const scratch[6],
                        long long *id_scratch, double **dev_ptrs, cudaStream_t s,
                        const int *gate = nullptr, int *dest_out = nullptr,
                        bool cell_order = false);
// Histogram bins the sort scratch needs (cell order adds a pass over the cells
// of a brick).
int sort_bins(int nn, int be, bool cell_order);
// moments.cu
cudaError_t launch_moments(double *const c[6], int64_t n, double *partials, int nblocks,
                           double *out, int *status, cudaStream_t s);
cudaError_t launch_wait_selftest(int *status, double limit_ms, cudaStream_t s);
int moments_blocks(int64_t n);
size_t moments_scratch_doubles(int nblocks);
cudaError_t launch_moments_transform(double *mom, const MapCoef *map, cudaStream_t s);
// fft.cu
// Scales of the block-floating-point tracking solve (fft.cu), set with each
// Green's spectrum: D >= max |G^| (the spectrum is stored as round(G^ 2^62 / D))
// and the output factor D / m^3.
struct FixScales {
    double D, F;
};

struct FftPlan {
    int n;            // physical grid nodes per dim
    int m;            // doubled size 2n
    double2 *buf;     // spectrum work buffers, m*m*(n+1) complex each
    double2 *buf2;
    double2 *tw;      // m twiddles exp(-2 pi i j/m)
    double *ghat;     // (n+1)^3 real even octant of the doubled Green's function spectrum
    longlong2 *twq;   // the twiddles in Q63 (fixed-point solve)
    long long *ghat_q;   // the spectrum octant as round(G^ 2^62 / D)
    FixScales *fs;       // device
    int *fexp;           // line exponents of the fixed-point passes
};
cudaError_t fft_plan_init(FftPlan *p, int n);
void fft_plan_free(FftPlan *p);
cudaError_t solve_rho_to_phi(const FftPlan *p, const double *rho, double *phi, cudaStream_t s);
cudaError_t solve_acc_to_phi_fixed(const FftPlan *p, const unsigned long long *acc_hi,
                                   const unsigned long long *acc_lo, double scale, double *phi,
                                   cudaStream_t s, const double *scale_dev);
cudaError_t solve_adjoint_shifted_fixed(const FftPlan *p, const double *phibar, double *out,
                                        cudaStream_t s);
cudaError_t green_quantize(const FftPlan *p, cudaStream_t s, const int *gate = nullptr);
cudaError_t green_spectrum_from_table(const FftPlan *p, const double *gtable, cudaStream_t s,
                                      const int *gate = nullptr);
cudaError_t solve_adjoint_shifted(const FftPlan *p, const double *phibar, double *out,
                                  cudaStream_t s);
// adjoint.cu
struct P6 {
    double *p[6];
};
// One reverse kick (see adjoint.cu): P = state before the kick, A = adjoint
// (in place), the kick's field/box/map, scatter and grid scratch.
struct AdjKick {
    P6 P, A;
    const EFix *ef;
    const int *escale;
    const Box *box;
    const MapCoef *map;             // table entry 1 + k
    double betagamma, q_macro;
    int nn;
    int64_t n;
    long long kick;                 // kick index (for the Green's function slot)
    const unsigned long long *amax_in;
    unsigned long long *amax_out;
    long long *kbar;                // 3 nn^3
    int *sexp;                      // 3
    double *part;                   // adj_blocks(n) * 13
    double *mbar;                   // 13 (out)
    double *phibar, *rb;            // (nn+2)^3 each
    const FftPlan *plan;
    const int32_t *slot_hist;
    const double *ghat_store;
    long long ghat_count;
    int ghat_cap;
};
int adj_blocks(int64_t n);
cudaError_t launch_adj_seed(P6 c, int64_t n, const double *mom, const double w[4], P6 A,
                            unsigned long long *amax, cudaStream_t s);
cudaError_t launch_adj_kick(const AdjKick &k, cudaStream_t s);
// Six arrays through a re-binning map dest (particle p went to slot dest[p]):
// gather out[p] = in[dest[p]] (back to the order before), else scatter
// out[dest[p]] = in[p] (forward).
cudaError_t launch_permute6(P6 in, const int *dest, int64_t n, P6 out, bool gather,
                            cudaStream_t s);
cudaError_t launch_adj_initial(P6 A, P6 z0, int64_t n, const MapCoef *map0, P6 out, double *part,
                               double *sums, cudaStream_t s);
cudaError_t launch_ghat_store(const TrackState *st, double *store, double *ghat, long long count,
                              int cap, int dir, int32_t *status, cudaStream_t s);
cudaError_t launch_set_deposit_gate(TrackState *st, cudaStream_t s);
cudaError_t launch_ghat_fetch(const int32_t *slot_hist, long long k, const double *store,
                              double *ghat, long long count, int cap, cudaStream_t s);
cudaError_t launch_twiss_beam(P6 xi, int64_t n, const double c[8], P6 out, cudaStream_t s);
struct Coef9 {
    double c[9];
};
cudaError_t launch_distribution(int kind, P6 z, const double *uni, int64_t n, Coef9 c, P6 out,
                                cudaStream_t s);
// igf.cu
// Doubles of IGF scratch for grid n: the (n+2)^3 corner table in
// double-double, then the far-field series coefficients.
inline long long igf_scratch_doubles(int n) {
    return 2LL * (n + 2) * (n + 2) * (n + 2) + 256;
}
cudaError_t launch_igf_table(int n, const double h[3], double *fcorner, double *gtable,
                             cudaStream_t s, const TrackState *gate = nullptr);
cudaError_t launch_green_commit(TrackState *st, cudaStream_t s);

}  // namespace bt
