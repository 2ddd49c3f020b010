// The library context and the host helpers shared by the C-ABI translation
// units (api.cu: tracking and the step calls; grad.cu: differentiation).
#pragma once

#include <string>
#include <vector>

#include "common.cuh"

namespace bt {
struct GradTape;
}

using bt::Box;
using bt::EFix;
using bt::FftPlan;
using bt::MapCoef;
using bt::Profiler;
using bt::TrackState;

struct bx_ctx {
    int n = 0;
    FftPlan plan{};
    unsigned long long *acc_hi = nullptr, *acc_lo = nullptr;
    double *rho = nullptr, *phi = nullptr;
    double *fcorner = nullptr, *gtable = nullptr;
    TrackState *st = nullptr;      // device
    Box *tmp_box = nullptr;        // device scratch for explicit boxes
    int32_t *status = nullptr;     // device
    long long *log = nullptr;      // device regrid log
    int64_t log_cap = 1 << 20;
    double *mom_partial = nullptr;
    int mom_partial_cap = 0;
    MapCoef *maps = nullptr;       // device map table
    size_t maps_cap = 0;
    bool green_valid = false;
    double green_h[3] = {0, 0, 0};
    long long kick = 0;
    EFix *efix = nullptr;                  // field in fixed point
    unsigned long long *emax = nullptr;    // max |E'| per component (bits)
    int *escale = nullptr;                 // fixed-point exponents
    // particle binning scratch, sized for sort_n particles
    int64_t sort_n = 0;
    // each particle's cells as the deposit of the current kick computed them
    // (3 n codes), read by that kick's gather
    unsigned long long *cells = nullptr;
    int64_t cells_n = 0;
    int *keys = nullptr;
    long long *counts = nullptr, *offs = nullptr, *sums = nullptr, *id_scr = nullptr;
    double *scr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double **dev_ptrs = nullptr;
    int shape = 1;                         // particle shape: 1 CIC, 2 TSC
    int sort_interval = 16;                // kicks between re-binning (0: never)
    int bin_edge = 0;                      // cells per bin edge (0: default)
    bool cell_order = false;               // re-bin by cell within brick; run deposit
    int sort_nb = 0;                       // bins the sort scratch is sized for
    // per-kick CUDA graph (conditional nodes), rebuilt when the bunch changes
    cudaGraphExec_t kick_exec = nullptr;
    double *graph_c[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t *graph_id = nullptr;
    int64_t graph_n = -1;
    double graph_bg = 0.0;
    MapCoef *graph_maps = nullptr;         // map table and sort scratch the graph was built with
    int64_t graph_sort_n = -1;
    unsigned long long *graph_cells = nullptr;
    cudaStream_t cap_stream = nullptr, body_stream = nullptr;
    bool graphs_off = false;               // the graph path failed once: plain launches
    Profiler *prof = nullptr;
    bt::GradTape *grad = nullptr;          // differentiation tape (grad.cu)
    bx_shard shard{};                      // sharded run: the collective hook (allreduce set)
    std::string err;
};

namespace bt {

extern thread_local std::string g_create_err;

int32_t fail(bx_ctx *c, int32_t code, const std::string &msg);
int32_t cuda_fail(bx_ctx *c, cudaError_t e, const char *what);

#define CK(call, what)                                          \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::bt::cuda_fail(ctx, e_, what); \
    } while (0)

struct Ref {
    double gamma, bg, beta, mass_eV, sign;
};
Ref make_ref(const bx_beam *b);

typedef double Mat[6][6];
struct Mat6 {
    double a[6][6];
};
bool element_is_thin(const bx_element &e);
bool lattice_has_multipoles(const bx_lattice *lat);
void mat_inverse(const Mat a, Mat out);
// Products of the linear thin elements ahead of every slice (pre[j]: between
// slice j-1 and slice j) and past the last slice (post), in beamline order.
void thin_maps(const bx_lattice *lat, const Ref &r, std::vector<Mat6> &pre, Mat6 &post);
// Summed kick polynomials of the thin multipoles at the same places.
struct MpPoly {
    int nc = 0;
    double cr[MP_MAX] = {}, ci[MP_MAX] = {};
};
void thin_multipoles(const bx_lattice *lat, std::vector<MpPoly> &pre, MpPoly &post);
void mat_identity(Mat m);
void focus_block(double ds, double k, double out[2][2]);
void element_map(const bx_element &e, double ds, const Ref &r, Mat m);
void mat_mul(const Mat a, const Mat b, Mat out);
MapCoef to_coef(const Mat m);

// Slice schedule of a lattice: element index and slice length per kick.
void slice_schedule(const bx_lattice *lat, std::vector<int> &sel, std::vector<double> &sds);
// Map table of kicks [first, first + nkicks): entry 0 the first half map,
// entry 1 + k the map after kick k (merged halves) with the kick factors of
// kick k and the map class; entries at a slice boundary with thin multipoles
// are MAP_SPLIT, their SplitRecs appended after the nkicks + 1 entries.
void build_map_table(const bx_lattice *lat, const std::vector<int> &sel,
                     const std::vector<double> &sds, int64_t first, int64_t nkicks, const Ref &r,
                     std::vector<MapCoef> &tab);

int32_t check_beam(bx_ctx *ctx, const bx_beam *b);
int32_t check_lattice(bx_ctx *ctx, const bx_lattice *l);
int32_t check_grid(bx_ctx *ctx, const bx_grid *g, bool need_rho, bool need_phi);
Box explicit_box(const double lo[3], const double hi[3], int n, double betagamma);
int32_t ensure_green(bx_ctx *ctx, const double h[3], cudaStream_t s);
int32_t ensure_maps(bx_ctx *ctx, size_t count);
int32_t ensure_sort_scratch(bx_ctx *ctx, int64_t n);
int32_t ensure_cells(bx_ctx *ctx, int64_t n);
// The cell codes the deposit hands to the gather, or null (the gather computes
// them): shared for CIC; for TSC the deposit's extra stores cost more than the
// gather's own nearest-node computation.
inline unsigned long long *shared_cells(bx_ctx *ctx) {
    return ctx->shape == 1 ? ctx->cells : nullptr;
}
int32_t ensure_moment_scratch(bx_ctx *ctx, int64_t n);
int32_t read_state(bx_ctx *ctx, TrackState *h, cudaStream_t s);
void init_state(TrackState *h);
void grad_free(bx_ctx *ctx);

// kick.cu: the pieces of one device-driven kick and its graphs
struct KickArgs {
    bx_ctx *ctx;
    double *const *c;
    int64_t *id;
    int64_t n;
    double bg;
    bool binning;
};
cudaError_t kick_plain(const KickArgs &k, cudaStream_t s);
// One kick of a sharded run: the plain launches of kick_plain with the
// caller's allreduce of the box keys before the box rule and of the charge
// accumulators before the solve.  Returns BX_OK, BX_COLLECTIVE (the callback
// failed) or BX_CUDA (*err holds the CUDA error).
int32_t kick_sharded(const KickArgs &k, cudaStream_t s, cudaError_t *err);
inline bool ctx_sharded(const bx_ctx *ctx) { return ctx->shard.allreduce != nullptr; }
cudaError_t build_kick_graph(const KickArgs &k, cudaGraphExec_t *exec);

}  // namespace bt
