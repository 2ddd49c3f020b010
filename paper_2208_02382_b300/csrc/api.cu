// C ABI of libbeamtrack (declared in include/beamtrack.h): argument checks,
// the context and its device scratch, the host-built map table of the slice
// schedule, and the split-operator tracking loop.
//
// Paper anchors (arXiv:2208.02382): Listing 1 (ImpactX(), set_particle_shape,
// set_space_charge, init_grids, add_particles, ref_particle().set_energy_MeV,
// lattice of Drift/Quad with nslice, evolve) and Model Assumptions (linear
// maps, rest-frame electrostatic field, split-operator step).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "common.cuh"

using namespace bt;

struct bx_ctx {
    int n = 0;
    FftPlan plan{};
    unsigned long long *acc_hi = nullptr, *acc_lo = nullptr;
    double *rho = nullptr, *phi = nullptr, *efield = nullptr;
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
    int *keys = nullptr;
    long long *counts = nullptr, *offs = nullptr, *sums = nullptr, *id_scr = nullptr;
    double *scr[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    double **dev_ptrs = nullptr;
    int sort_interval = 16;                // kicks between re-binning
    // per-kick CUDA graph (conditional nodes), rebuilt when the bunch changes
    cudaGraphExec_t kick_exec = nullptr;
    double *graph_c[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int64_t *graph_id = nullptr;
    int64_t graph_n = -1;
    double graph_bg = 0.0;
    cudaStream_t cap_stream = nullptr, body_stream = nullptr;
    bool graphs_off = false;               // the graph path failed once: plain launches
    Profiler *prof = nullptr;
    std::string err;
};

namespace {

thread_local std::string g_create_err;

int32_t fail(bx_ctx *c, int32_t code, const std::string &msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

int32_t cuda_fail(bx_ctx *c, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(c, e == cudaErrorMemoryAllocation ? BX_OUT_OF_MEMORY : BX_CUDA, m);
}

#define CK(call, what)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

struct Ref {
    double gamma, bg, beta, mass_eV, sign;
};

// Reference particle from kinetic energy (Listing 1 set_energy_MeV, read as
// kinetic): gamma = 1 + W/mc^2, beta gamma = sqrt(gamma^2 - 1).
Ref make_ref(const bx_beam *b) {
    Ref r;
    r.gamma = 1.0 + b->kinetic_MeV / b->mass_MeV;
    r.bg = std::sqrt(r.gamma * r.gamma - 1.0);
    r.beta = r.bg / r.gamma;
    r.mass_eV = b->mass_MeV * 1e6;
    r.sign = b->charge_sign;
    return r;
}

typedef double Mat[6][6];

void mat_identity(Mat m) {
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) m[i][j] = i == j ? 1.0 : 0.0;
}

void focus_block(double ds, double k, double out[2][2]) {
    if (k > 0.0) {
        double w = std::sqrt(k), c = std::cos(w * ds), s = std::sin(w * ds);
        out[0][0] = c; out[0][1] = s / w; out[1][0] = -w * s; out[1][1] = c;
    } else if (k < 0.0) {
        double w = std::sqrt(-k), c = std::cosh(w * ds), s = std::sinh(w * ds);
        out[0][0] = c; out[0][1] = s / w; out[1][0] = w * s; out[1][1] = c;
    } else {
        out[0][0] = 1.0; out[0][1] = ds; out[1][0] = 0.0; out[1][1] = 1.0;
    }
}

// Linear map of a piece ds of an element (Model Assumptions: linear order).
// Drift: x += ds px, y += ds py, t += ds/(beta gamma)^2 pt.  Quadrupole: k > 0
// focuses x.  Sector bend of radius rho = length/angle, theta = ds/rho:
//   x'  = cos x + rho sin px - rho(1-cos)/beta pt
//   px' = -sin/rho x + cos px - sin/beta pt
//   t'  = t + sin/beta x + rho(1-cos)/beta px + rho(sin/beta^2 - theta) pt.
void element_map(const bx_element &e, double ds, const Ref &r, Mat m) {
    mat_identity(m);
    if (e.type == BX_SBEND && e.angle != 0.0) {
        double rho = e.length / e.angle, th = ds / rho;
        double c = std::cos(th), s = std::sin(th), b = r.beta;
        m[0][0] = c; m[0][1] = rho * s; m[0][5] = -rho * (1.0 - c) / b;
        m[1][0] = -s / rho; m[1][1] = c; m[1][5] = -s / b;
        m[2][3] = ds;
        m[4][0] = s / b; m[4][1] = rho * (1.0 - c) / b; m[4][5] = rho * (s / (b * b) - th);
        return;
    }
    m[4][5] = ds / (r.bg * r.bg);
    if (e.type == BX_QUAD) {
        double bx[2][2], by[2][2];
        focus_block(ds, e.k, bx);
        focus_block(ds, -e.k, by);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                m[i][j] = bx[i][j];
                m[2 + i][2 + j] = by[i][j];
            }
    } else {
        m[0][1] = ds;
        m[2][3] = ds;
    }
}

// out = a * b (apply b first).
void mat_mul(const Mat a, const Mat b, Mat out) {
    Mat t;
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += a[i][k] * b[k][j];
            t[i][j] = s;
        }
    memcpy(out, t, sizeof(Mat));
}

MapCoef to_coef(const Mat m) {
    MapCoef c;
    memset(&c, 0, sizeof(c));
    c.m00 = m[0][0]; c.m01 = m[0][1]; c.m05 = m[0][5];
    c.m10 = m[1][0]; c.m11 = m[1][1]; c.m15 = m[1][5];
    c.m22 = m[2][2]; c.m23 = m[2][3];
    c.m32 = m[3][2]; c.m33 = m[3][3];
    c.m40 = m[4][0]; c.m41 = m[4][1]; c.m45 = m[4][5];
    return c;
}

int32_t check_beam(bx_ctx *ctx, const bx_beam *b) {
    if (!b) return fail(ctx, BX_BAD_ARG, "beam is NULL");
    if (b->n < 0) return fail(ctx, BX_BAD_ARG, "beam n < 0");
    if (b->n > 0)
        for (int k = 0; k < 6; ++k)
            if (!b->coord[k]) return fail(ctx, BX_BAD_ARG, "beam coordinate pointer is NULL");
    if (!(b->charge_sign == 1.0 || b->charge_sign == -1.0))
        return fail(ctx, BX_BAD_ARG, "charge_sign must be +1 or -1");
    if (!(b->mass_MeV > 0.0) || !std::isfinite(b->mass_MeV))
        return fail(ctx, BX_BAD_ARG, "mass_MeV must be > 0");
    if (!(b->kinetic_MeV > 0.0) || !std::isfinite(b->kinetic_MeV))
        return fail(ctx, BX_BAD_ARG, "kinetic_MeV must be > 0");
    if (!std::isfinite(b->bunch_charge_C)) return fail(ctx, BX_BAD_ARG, "bunch charge not finite");
    return BX_OK;
}

int32_t check_lattice(bx_ctx *ctx, const bx_lattice *l) {
    if (!l) return fail(ctx, BX_BAD_ARG, "lattice is NULL");
    if (l->count < 0 || (l->count > 0 && !l->elements))
        return fail(ctx, BX_BAD_ARG, "lattice elements missing");
    for (int i = 0; i < l->count; ++i) {
        const bx_element &e = l->elements[i];
        if (e.type != BX_DRIFT && e.type != BX_QUAD && e.type != BX_SBEND)
            return fail(ctx, BX_BAD_ARG, "unknown element type");
        if (!(e.length > 0.0) || !std::isfinite(e.length))
            return fail(ctx, BX_BAD_ARG, "element length must be > 0");
        if (e.nslice <= 0) return fail(ctx, BX_BAD_ARG, "element nslice must be >= 1");
        if (!std::isfinite(e.k) || !std::isfinite(e.angle))
            return fail(ctx, BX_BAD_ARG, "element k/angle not finite");
    }
    return BX_OK;
}

int32_t check_grid(bx_ctx *ctx, const bx_grid *g, bool need_rho, bool need_phi) {
    if (!g) return fail(ctx, BX_BAD_ARG, "grid is NULL");
    if (g->n != ctx->n) return fail(ctx, BX_BAD_ARG, "grid n differs from the context's n_grid");
    if (need_rho && !g->rho) return fail(ctx, BX_BAD_ARG, "grid rho is NULL");
    if (need_phi && !g->phi) return fail(ctx, BX_BAD_ARG, "grid phi is NULL");
    return BX_OK;
}

Box explicit_box(const double lo[3], const double hi[3], int n) {
    Box b;
    for (int d = 0; d < 3; ++d) {
        b.lo[d] = lo[d];
        b.hi[d] = hi[d];
        b.h[d] = (hi[d] - lo[d]) / (double)(n - 1);
        b.inv_h[d] = 1.0 / b.h[d];
    }
    return b;
}

int32_t ensure_green(bx_ctx *ctx, const double h[3], cudaStream_t s) {
    if (ctx->green_valid && ctx->green_h[0] == h[0] && ctx->green_h[1] == h[1] &&
        ctx->green_h[2] == h[2])
        return BX_OK;
    CK(launch_igf_table(ctx->n, h, ctx->fcorner, ctx->gtable, s), "green table");
    CK(green_spectrum_from_table(&ctx->plan, ctx->gtable, s), "green spectrum");
    ctx->green_valid = true;
    memcpy(ctx->green_h, h, sizeof(ctx->green_h));
    // the tracking loop decides on the device from the state's copy of h
    CK(cudaMemcpyAsync(ctx->st->green_h, ctx->green_h, sizeof(ctx->green_h),
                       cudaMemcpyHostToDevice, s),
       "green h");
    return BX_OK;
}

int32_t ensure_maps(bx_ctx *ctx, size_t count) {
    if (count <= ctx->maps_cap) return BX_OK;
    if (ctx->maps) cudaFree(ctx->maps);
    ctx->maps = nullptr;
    size_t cap = count < 1024 ? 1024 : count;
    CK(cudaMalloc(&ctx->maps, cap * sizeof(MapCoef)), "map table");
    ctx->maps_cap = cap;
    return BX_OK;
}

// Binning scratch for n particles, allocated on the first call for a larger n.
int32_t ensure_sort_scratch(bx_ctx *ctx, int64_t n) {
    if (n <= ctx->sort_n) return BX_OK;
    cudaDeviceSynchronize();
    void **ps[] = {(void **)&ctx->keys, (void **)&ctx->counts, (void **)&ctx->offs,
                   (void **)&ctx->sums, (void **)&ctx->id_scr, (void **)&ctx->scr[0],
                   (void **)&ctx->scr[1], (void **)&ctx->scr[2], (void **)&ctx->scr[3],
                   (void **)&ctx->scr[4], (void **)&ctx->scr[5]};
    for (void **p : ps)
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    ctx->sort_n = 0;
    const long long len = (long long)sort_bricks(ctx->n) * sort_chunks(n);
    CK(cudaMalloc(&ctx->keys, n * sizeof(int)), "sort keys");
    CK(cudaMalloc(&ctx->counts, len * sizeof(long long)), "sort counts");
    CK(cudaMalloc(&ctx->offs, len * sizeof(long long)), "sort offsets");
    CK(cudaMalloc(&ctx->sums, (len / 2048 + 2) * sizeof(long long)), "sort sums");
    CK(cudaMalloc(&ctx->id_scr, n * sizeof(long long)), "sort ids");
    for (int k = 0; k < 6; ++k) CK(cudaMalloc(&ctx->scr[k], n * sizeof(double)), "sort arrays");
    ctx->sort_n = n;
    return BX_OK;
}

int32_t read_state(bx_ctx *ctx, TrackState *h, cudaStream_t s) {
    CK(cudaMemcpyAsync(h, ctx->st, sizeof(TrackState), cudaMemcpyDeviceToHost, s), "read state");
    CK(cudaStreamSynchronize(s), "sync");
    return BX_OK;
}

void init_state(TrackState *h) {
    memset(h, 0, sizeof(*h));
    for (int d = 0; d < 3; ++d) {
        h->mm[d] = dkey(INFINITY);
        h->mm[3 + d] = dkey(-INFINITY);
    }
}

// The kernels of one device-driven kick, in pieces (so the graph builder can
// put the gated pieces into conditional bodies).
struct KickArgs {
    bx_ctx *ctx;
    double *const *c;
    int64_t *id;
    int64_t n;
    double bg;
    bool binning;
};

cudaError_t kick_green(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = launch_igf_table(ctx->n, nullptr, ctx->fcorner, ctx->gtable, s, ctx->st);
    if (e == cudaSuccess) e = green_spectrum_from_table(&ctx->plan, ctx->gtable, s, &ctx->st->green_stale);
    if (e == cudaSuccess) e = launch_green_commit(ctx->st, s);
    return e;
}

cudaError_t kick_sort(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_sort(k.c, (long long *)k.id, k.n, k.bg, &ctx->st->box, ctx->n, ctx->keys,
                       ctx->counts, ctx->offs, ctx->sums, ctx->scr, ctx->id_scr, ctx->dev_ptrs, s,
                       &ctx->st->sort_gate);
}

cudaError_t kick_deposit(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_track_deposit(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->acc_hi, ctx->acc_lo,
                                ctx->st, ctx->status, s);
}

cudaError_t kick_solve_field_push(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = solve_acc_to_phi(&ctx->plan, ctx->acc_hi, ctx->acc_lo, 0.0, ctx->phi, s,
                                     &ctx->st->rho_scale);
    if (e == cudaSuccess)
        e = launch_field(ctx->phi, ctx->n, &ctx->st->box, 0.0, 0.0, 0.0, ctx->efield, ctx->emax,
                         ctx->efix, ctx->escale, s, ctx->st, ctx->maps);
    if (e == cudaSuccess)
        e = launch_track_particles(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->efix, ctx->escale,
                                   ctx->maps, ctx->acc_hi, ctx->acc_lo, ctx->st, ctx->status, s, 1);
    return e;
}

cudaError_t kick_next_deposit(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_track_particles(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->efix, ctx->escale,
                                  ctx->maps, ctx->acc_hi, ctx->acc_lo, ctx->st, ctx->status, s, 2);
}

// Plain launches of one kick (gated kernels return at once when not needed).
cudaError_t kick_plain(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = launch_box_rule(ctx->st, ctx->n, k.n, ctx->log, ctx->log_cap, true, s);
    if (e == cudaSuccess) e = kick_green(k, s);
    if (e == cudaSuccess && k.binning) e = kick_sort(k, s);
    if (e == cudaSuccess) e = kick_deposit(k, s);
    if (e == cudaSuccess) e = kick_solve_field_push(k, s);
    if (e == cudaSuccess) e = kick_next_deposit(k, s);
    return e;
}

// Adds an IF node on condition `h` at the current point of the capture on
// `cs` and captures `body` into it on `bs`.
template <class F>
cudaError_t capture_if(cudaStream_t cs, cudaStream_t bs, cudaGraph_t cg,
                       cudaGraphConditionalHandle h, F body) {
    cudaStreamCaptureStatus status;
    const cudaGraphNode_t *deps = nullptr;
    size_t ndeps = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, cg, deps, nullptr, ndeps, &p);
    if (e != cudaSuccess) return e;
    cudaGraph_t g = p.conditional.phGraph_out[0];
    e = cudaStreamUpdateCaptureDependencies(cs, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCaptureToGraph(bs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t eb = body(bs);
    e = cudaStreamEndCapture(bs, &g);
    return eb != cudaSuccess ? eb : e;
}

// One kick as a CUDA graph: box rule (sets the conditions), IF(Green's
// function stale){rebuild}, IF(re-bin due){sort}, IF(deposit needed){deposit},
// solve + field + gather/kick/map, IF(next kick){deposit for it}.
cudaError_t build_kick_graph(const KickArgs &k, cudaGraphExec_t *exec) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = cudaSuccess;
    if (!ctx->cap_stream) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->body_stream)
        e = cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaStream_t cs = ctx->cap_stream, bs = ctx->body_stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaGraph_t cg = nullptr;
    cudaStreamCaptureStatus status;
    e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle hg = 0, hs = 0, hd = 0, hn = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hg, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hs, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hd, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hn, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = launch_box_rule_graph(ctx->st, ctx->n, ctx->log, ctx->log_cap, hg, hs, hd, hn, cs);
    if (e == cudaSuccess) e = capture_if(cs, bs, cg, hg, [&](cudaStream_t b) { return kick_green(k, b); });
    if (e == cudaSuccess && k.binning)
        e = capture_if(cs, bs, cg, hs, [&](cudaStream_t b) { return kick_sort(k, b); });
    if (e == cudaSuccess) e = capture_if(cs, bs, cg, hd, [&](cudaStream_t b) { return kick_deposit(k, b); });
    if (e == cudaSuccess) e = kick_solve_field_push(k, cs);
    if (e == cudaSuccess)
        e = capture_if(cs, bs, cg, hn, [&](cudaStream_t b) { return kick_next_deposit(k, b); });
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();  // clear a sticky capture error, if any
    return e;
}

}  // namespace

int32_t bt::set_noctx_error(int32_t code, const char *msg) { return fail(nullptr, code, msg); }

extern "C" {

int32_t bx_create(bx_ctx **out, const bx_options *opt) {
    if (!out || !opt) return fail(nullptr, BX_BAD_ARG, "NULL argument");
    *out = nullptr;
    int n = opt->n_grid;
    if (n < 8 || n > 256 || (n & (n - 1)) != 0)
        return fail(nullptr, BX_BAD_ARG, "n_grid must be a power of two in [8, 256]");
    if (opt->shape_order != 1) return fail(nullptr, BX_BAD_ARG, "shape_order must be 1 (CIC)");
    bx_ctx *ctx = new (std::nothrow) bx_ctx();
    if (!ctx) return fail(nullptr, BX_OUT_OF_MEMORY, "host allocation");
    ctx->n = n;
    ctx->prof = profiler_new();
    const size_t n3 = (size_t)n * n * n, q3 = (size_t)(n + 2) * (n + 2) * (n + 2);
    const size_t o3 = (size_t)(n + 1) * (n + 1) * (n + 1);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes);
    };
    A((void **)&ctx->acc_hi, n3 * 8);
    A((void **)&ctx->acc_lo, n3 * 8);
    A((void **)&ctx->rho, n3 * 8);
    A((void **)&ctx->phi, q3 * 8);
    A((void **)&ctx->efield, n3 * sizeof(Field4));
    A((void **)&ctx->fcorner, q3 * 16);
    A((void **)&ctx->gtable, o3 * 8);
    A((void **)&ctx->st, sizeof(TrackState));
    A((void **)&ctx->tmp_box, sizeof(Box));
    A((void **)&ctx->status, sizeof(int32_t));
    A((void **)&ctx->log, ctx->log_cap * sizeof(long long));
    A((void **)&ctx->efix, n3 * sizeof(EFix));
    A((void **)&ctx->emax, 3 * sizeof(unsigned long long));
    A((void **)&ctx->escale, 4 * sizeof(int));
    A((void **)&ctx->dev_ptrs, 12 * sizeof(double *));
    if (e == cudaSuccess) e = fft_plan_init(&ctx->plan, n);
    if (e == cudaSuccess) {
        TrackState h;
        init_state(&h);
        e = cudaMemcpy(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(int32_t));
    if (e != cudaSuccess) {
        std::string m = std::string("bx_create: ") + cudaGetErrorString(e);
        int32_t code = e == cudaErrorMemoryAllocation ? BX_OUT_OF_MEMORY : BX_CUDA;
        bx_destroy(ctx);
        return fail(nullptr, code, m);
    }
    *out = ctx;
    return BX_OK;
}

int32_t bx_destroy(bx_ctx *ctx) {
    if (!ctx) return BX_OK;
    cudaDeviceSynchronize();
    void *ptrs[] = {ctx->acc_hi, ctx->acc_lo, ctx->rho, ctx->phi, ctx->efield, ctx->fcorner,
                    ctx->gtable, ctx->st, ctx->tmp_box, ctx->status, ctx->log,
                    ctx->mom_partial, ctx->maps, ctx->efix, ctx->emax, ctx->escale,
                    ctx->dev_ptrs, ctx->keys, ctx->counts, ctx->offs, ctx->sums, ctx->id_scr,
                    ctx->scr[0], ctx->scr[1], ctx->scr[2], ctx->scr[3], ctx->scr[4], ctx->scr[5]};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    fft_plan_free(&ctx->plan);
    if (ctx->kick_exec) cudaGraphExecDestroy(ctx->kick_exec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->body_stream) cudaStreamDestroy(ctx->body_stream);
    profiler_free(ctx->prof);
    delete ctx;
    return BX_OK;
}

int32_t bx_reset(bx_ctx *ctx) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    TrackState h;
    init_state(&h);
    CK(cudaMemcpy(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice), "reset");
    ctx->kick = 0;
    return BX_OK;
}

int32_t bx_track(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat, int64_t first_kick,
                 int64_t nkicks, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_lattice(ctx, lat))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // slice schedule: (element, ds) per kick
    std::vector<int> sel;
    std::vector<double> sds;
    for (int i = 0; i < lat->count; ++i)
        for (int k = 0; k < lat->elements[i].nslice; ++k) {
            sel.push_back(i);
            sds.push_back(lat->elements[i].length / lat->elements[i].nslice);
        }
    const int64_t total = (int64_t)sel.size();
    if (nkicks < 0) nkicks = total - first_kick;
    if (first_kick < 0 || first_kick > total || nkicks < 0 || first_kick + nkicks > total)
        return fail(ctx, BX_BAD_ARG, "kick range outside the slice schedule");
    if (nkicks == 0) return BX_OK;
    const Ref r = make_ref(beam);
    // map table: H_first, H_{k+1} H_k for inner boundaries, H_last
    std::vector<MapCoef> tab;
    tab.reserve(nkicks + 1);
    Mat hk, hn, mm;
    element_map(lat->elements[sel[first_kick]], 0.5 * sds[first_kick], r, hk);
    tab.push_back(to_coef(hk));
    for (int64_t k = first_kick; k < first_kick + nkicks; ++k) {
        if (k + 1 < first_kick + nkicks) {
            element_map(lat->elements[sel[k + 1]], 0.5 * sds[k + 1], r, hn);
            mat_mul(hn, hk, mm);
            tab.push_back(to_coef(mm));
            memcpy(hk, hn, sizeof(Mat));
        } else {
            tab.push_back(to_coef(hk));
        }
    }
    // kick factors of kick k and the map class, in table entry 1 + k
    for (int64_t k = 0; k < nkicks; ++k) {
        const double ds = sds[first_kick + k];
        tab[1 + k].kick_t = r.sign * ds / (r.mass_eV * (r.bg * r.bg));
        tab[1 + k].kick_z = -r.sign * ds / (r.mass_eV * r.bg);
    }
    for (auto &m : tab) m.kind = (double)map_kind(m);
    if ((rc = ensure_maps(ctx, tab.size()))) return rc;
    CK(cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                       cudaMemcpyHostToDevice, s),
       "upload maps");
    if (beam->n == 0) {
        ctx->kick += nkicks;
        return BX_OK;
    }
    double *const *c = beam->coord;
    if (!lat->space_charge) {
        // maps only: H_first, merged pairs, H_last in one pass per particle
        CK(launch_push_maps(c, beam->n, ctx->maps, (int)tab.size(), s), "push");
        ctx->kick += nkicks;
        return BX_OK;
    }
    const double q_macro = r.sign * std::fabs(beam->bunch_charge_C) / (double)beam->n;
    const bool binning = beam->id != nullptr;
    if (binning && (rc = ensure_sort_scratch(ctx, beam->n))) return rc;
    // Device-driven kicks: the box rule kernel of each kick sets the gates
    // (Green's function rebuild, deposit of the current positions, re-binning,
    // deposit for a next kick) that the later kernels of the kick read, and the
    // per-kick map and kick factors come from the table at index 1 + k; no
    // host decision or synchronisation between kicks.
    CK(launch_call_init(ctx->st, (int)nkicks, q_macro, binning ? ctx->sort_interval : 0,
                        ctx->kick, s),
       "call init");
    if (binning) CK(sort_set_pointers(c, ctx->scr, ctx->dev_ptrs, s), "sort pointers");
    CK(launch_push_maps(c, beam->n, ctx->maps, 1, s), "push");
    CK(launch_minmax(c, beam->n, r.bg, ctx->st, ctx->status, s), "minmax");
    const KickArgs ka{ctx, c, beam->id, beam->n, r.bg, binning};
    bool use_graph = !ctx->graphs_off && !profiler_timing(ctx->prof);
    if (use_graph) {
        bool same = ctx->kick_exec && ctx->graph_n == beam->n && ctx->graph_id == beam->id &&
                    ctx->graph_bg == r.bg;
        for (int q = 0; q < 6 && same; ++q) same = ctx->graph_c[q] == c[q];
        if (!same) {
            if (ctx->kick_exec) cudaGraphExecDestroy(ctx->kick_exec);
            ctx->kick_exec = nullptr;
            // the captured kernels must not run before the prologue above
            CK(cudaStreamSynchronize(s), "sync");
            if (build_kick_graph(ka, &ctx->kick_exec) != cudaSuccess) {
                ctx->kick_exec = nullptr;
                ctx->graphs_off = true;
                use_graph = false;
            } else {
                for (int q = 0; q < 6; ++q) ctx->graph_c[q] = c[q];
                ctx->graph_id = beam->id;
                ctx->graph_n = beam->n;
                ctx->graph_bg = r.bg;
            }
        }
    }
    for (int64_t k = 0; k < nkicks; ++k) {
        if (use_graph) CK(cudaGraphLaunch(ctx->kick_exec, s), "kick graph");
        else CK(kick_plain(ka, s), "kick");
    }
    ctx->kick += nkicks;
    ctx->green_valid = false;  // the device may have rebuilt the spectrum for another h
    return BX_OK;
}

int32_t bx_deposit(bx_ctx *ctx, const bx_beam *beam, bx_grid *grid, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_grid(ctx, grid, true, false))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const Ref r = make_ref(beam);
    double *const *c = beam->coord;
    const Box *box;
    Box hb;
    if (grid->use_box) {
        for (int d = 0; d < 3; ++d)
            if (!(grid->hi[d] > grid->lo[d]) || !std::isfinite(grid->lo[d]) ||
                !std::isfinite(grid->hi[d]))
                return fail(ctx, BX_BAD_ARG, "grid box needs finite lo < hi");
        Box b = explicit_box(grid->lo, grid->hi, ctx->n);
        hb = b;
        CK(cudaMemcpyAsync(ctx->tmp_box, &b, sizeof(b), cudaMemcpyHostToDevice, s), "box");
        for (int d = 0; d < 3; ++d) grid->h[d] = b.h[d];
        box = ctx->tmp_box;
    } else {
        if (beam->n == 0) return fail(ctx, BX_BAD_ARG, "box rule needs particles");
        CK(launch_minmax(c, beam->n, r.bg, ctx->st, ctx->status, s), "minmax");
        CK(cudaMemcpyAsync(&ctx->st->kick, &ctx->kick, sizeof(long long), cudaMemcpyHostToDevice, s),
           "kick counter");
        CK(launch_box_rule(ctx->st, ctx->n, beam->n, ctx->log, ctx->log_cap, false, s), "box rule");
        TrackState h;
        if ((rc = read_state(ctx, &h, s))) return rc;
        for (int d = 0; d < 3; ++d) {
            if (!std::isfinite(h.box.lo[d]) || !std::isfinite(h.box.hi[d]))
                return fail(ctx, BX_NONFINITE, "non-finite particle coordinates");
            grid->lo[d] = h.box.lo[d];
            grid->hi[d] = h.box.hi[d];
            grid->h[d] = h.box.h[d];
        }
        box = &ctx->st->box;
        hb = h.box;
    }
    const double q_macro =
        beam->n > 0 ? r.sign * std::fabs(beam->bunch_charge_C) / (double)beam->n : 0.0;
    CK(launch_deposit(c, beam->n, r.bg, box, hb, ctx->n, ctx->acc_hi, ctx->acc_lo, ctx->status, s),
       "deposit");
    CK(launch_acc_to_rho(ctx->acc_hi, ctx->acc_lo, ctx->n, q_macro, box, grid->rho, s), "rho");
    return BX_OK;
}

int32_t bx_solve(bx_ctx *ctx, bx_grid *grid, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_grid(ctx, grid, true, true);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d)
        if (!(grid->h[d] > 0.0) || !std::isfinite(grid->h[d]))
            return fail(ctx, BX_BAD_ARG, "grid h must be finite and > 0");
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = ensure_green(ctx, grid->h, s))) return rc;
    CK(solve_rho_to_phi(&ctx->plan, grid->rho, grid->phi, s), "solve");
    return BX_OK;
}

int32_t bx_gather_kick(bx_ctx *ctx, bx_beam *beam, const bx_grid *grid, double ds, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_grid(ctx, grid, false, true))) return rc;
    if (!(ds > 0.0) || !std::isfinite(ds)) return fail(ctx, BX_BAD_ARG, "ds must be > 0");
    for (int d = 0; d < 3; ++d)
        if (!(grid->h[d] > 0.0) || !std::isfinite(grid->lo[d]))
            return fail(ctx, BX_BAD_ARG, "grid lo/h invalid");
    cudaStream_t s = (cudaStream_t)stream;
    const Ref r = make_ref(beam);
    Box b;
    for (int d = 0; d < 3; ++d) {
        b.lo[d] = grid->lo[d];
        b.hi[d] = grid->hi[d];
        b.h[d] = grid->h[d];
        b.inv_h[d] = 1.0 / grid->h[d];
    }
    CK(cudaMemcpyAsync(ctx->tmp_box, &b, sizeof(b), cudaMemcpyHostToDevice, s), "box");
    const double kt = r.sign * ds / (r.mass_eV * (r.bg * r.bg));
    const double kz = -r.sign * ds / (r.mass_eV * r.bg);
    CK(launch_field(grid->phi, ctx->n, ctx->tmp_box, kt, kt, kz, ctx->efield, ctx->emax,
                    ctx->efix, ctx->escale, s),
       "field");
    CK(launch_kick_push_deposit(beam->coord, beam->n, r.bg, ctx->tmp_box, b, ctx->n, ctx->efix,
                                ctx->escale, nullptr, false, nullptr, nullptr, nullptr,
                                ctx->status, s),
       "gather/kick");
    return BX_OK;
}

int32_t bx_moments(bx_ctx *ctx, const bx_beam *beam, double *out, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if (!out) return fail(ctx, BX_BAD_ARG, "out is NULL");
    if (beam->n == 0) return fail(ctx, BX_BAD_ARG, "moments of an empty beam");
    cudaStream_t s = (cudaStream_t)stream;
    int nb = moments_blocks(beam->n);
    if (nb * 21 > ctx->mom_partial_cap) {
        if (ctx->mom_partial) cudaFree(ctx->mom_partial);
        ctx->mom_partial = nullptr;
        CK(cudaMalloc(&ctx->mom_partial, (size_t)nb * 21 * sizeof(double)), "moments scratch");
        ctx->mom_partial_cap = nb * 21;
    }
    CK(launch_moments(beam->coord, beam->n, ctx->mom_partial, nb, out, s), "moments");
    return BX_OK;
}

int32_t bx_green_table(bx_ctx *ctx, const double h[3], double *out, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    if (!h || !out) return fail(ctx, BX_BAD_ARG, "NULL argument");
    for (int d = 0; d < 3; ++d)
        if (!(h[d] > 0.0) || !std::isfinite(h[d])) return fail(ctx, BX_BAD_ARG, "h must be > 0");
    cudaStream_t s = (cudaStream_t)stream;
    CK(launch_igf_table(ctx->n, h, ctx->fcorner, ctx->gtable, s), "green table");
    const size_t o3 = (size_t)(ctx->n + 1) * (ctx->n + 1) * (ctx->n + 1);
    CK(cudaMemcpyAsync(out, ctx->gtable, o3 * 8, cudaMemcpyDeviceToDevice, s), "copy");
    return BX_OK;
}

int32_t bx_regrid_log(bx_ctx *ctx, int64_t *out, int64_t cap, int64_t *count) {
    if (!ctx || !count) return fail(ctx, BX_BAD_ARG, "NULL argument");
    TrackState h;
    int32_t rc = read_state(ctx, &h, 0);
    if (rc) return rc;
    *count = h.nlog;
    int64_t k = h.nlog < cap ? h.nlog : cap;
    if (k > ctx->log_cap) k = ctx->log_cap;
    if (k > 0 && out) CK(cudaMemcpy(out, ctx->log, k * sizeof(long long), cudaMemcpyDeviceToHost), "log");
    return BX_OK;
}

int32_t bx_get_box(bx_ctx *ctx, double lo[3], double hi[3], double h[3]) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    TrackState st;
    int32_t rc = read_state(ctx, &st, 0);
    if (rc) return rc;
    if (!st.has_box) return fail(ctx, BX_BAD_ARG, "no box yet");
    for (int d = 0; d < 3; ++d) {
        if (lo) lo[d] = st.box.lo[d];
        if (hi) hi[d] = st.box.hi[d];
        if (h) h[d] = st.box.h[d];
    }
    return BX_OK;
}

int32_t bx_sync(bx_ctx *ctx, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s), "sync");
    int32_t st = 0;
    CK(cudaMemcpy(&st, ctx->status, sizeof(st), cudaMemcpyDeviceToHost), "status");
    CK(cudaMemset(ctx->status, 0, sizeof(st)), "status clear");
    if (st & ST_NONFINITE) return fail(ctx, BX_NONFINITE, "non-finite particle coordinates");
    if (st & ST_TIMEOUT) return fail(ctx, BX_DEVICE_TIMEOUT, "a device wait timed out");
    if (st & ST_OUTSIDE) return fail(ctx, BX_BAD_ARG, "a particle lies outside the given box");
    return BX_OK;
}

int32_t bx_profile(bx_ctx *ctx, int32_t timing) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    profiler_enable(ctx->prof, timing != 0);
    return BX_OK;
}

int32_t bx_profile_read(bx_ctx *ctx, double *ms, int64_t *launches, int32_t cap, int32_t *count) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    if (cap < 0 || (cap > 0 && !ms && !launches)) return fail(ctx, BX_BAD_ARG, "bad output arrays");
    static_assert(sizeof(long long) == sizeof(int64_t), "int64");
    CK(profiler_read(ctx->prof, ms, (long long *)launches, cap), "profile read");
    if (count) *count = K_COUNT;
    return BX_OK;
}

const char *bx_kernel_name(int32_t id) { return kernel_name(id); }

const char *bx_last_error(const bx_ctx *ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

}  // extern "C"
