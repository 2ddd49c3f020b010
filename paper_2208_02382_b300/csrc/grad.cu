// Differentiation of the tracking (C ABI): a forward pass that keeps
// checkpoints, a reverse sweep that recomputes each checkpoint segment and
// runs the adjoint kernels kick by kick in reverse, and the chain rule from
// the per-map adjoints to the quadrupole strengths.
//
// Paper anchors (arXiv:2208.02382): the Introduction and Outlook motivate
// coupling the simulation to machine-learning workflows (differentiable
// modelling); Listing 1 and Model Assumptions define what is differentiated
// (map(ds/2) -> space-charge kick over ds -> map(ds/2) per slice).  The paper
// gives no adjoint: the reverse steps are the transposes of the forward
// kernels (adjoint.cu).  Readings: the grid box is held fixed between regrids
// (derivative zero); the objectives are the final unnormalised rms
// emittances and rms sizes.
//
// Memory (device, owned by the context, sized on the first call for a given
// particle count, kick count, checkpoint interval and grid):
//   z0                 6 n            the initial bunch
//   checkpoints        ceil(K/C) (6 n + one TrackState)
//   segment ring       (C + 1) 6 n    states before each kick of a segment
//   field ring         C n^3 EFix     the fixed-point field of each kick
//   Green's store      up to K + 1 spectra (n+1)^3, one per build
//   box/slot history   K
//   re-binning maps    ceil(K/C) n int32 (destination of each particle at the
//                      re-binning that starts a segment)
//   adjoint            6 n, 3 n^3 int64 scatter, 2 (n+2)^3 grid, (K+1) 13 map adjoints
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>

#include "ctx.cuh"

namespace bt {

struct GradTape {
    int64_t np = 0, K = 0;
    int C = 0, nseg = 0, n = 0, ghat_cap = 0;
    long long n3 = 0, o3 = 0, q3 = 0;
    double *z0 = nullptr, *ckpt = nullptr, *ring = nullptr;
    TrackState *ckst = nullptr;
    EFix *efix_ring = nullptr;
    int *escale_ring = nullptr;
    Box *box_hist = nullptr, *box_replay = nullptr;
    int32_t *slot_hist = nullptr;
    double *ghat_store = nullptr;
    double *adj = nullptr;
    long long *kbar = nullptr;
    double *phibar = nullptr, *rb = nullptr;
    unsigned long long *amax = nullptr;
    int *sexp = nullptr;
    double *part = nullptr, *mbar = nullptr, *sums0 = nullptr, *mom = nullptr;
    int *perm = nullptr;     // per segment: destination slot of each particle at its re-binning
    bool binned = false;     // segments >= 1 start with a re-binning
    // host record of the run
    std::vector<bx_element> elements;
    std::vector<int> sel;
    std::vector<double> sds;
    Ref ref{};
    double q_macro = 0.0;
    double *coord[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool valid = false;
};

void grad_free(bx_ctx *ctx) {
    GradTape *g = ctx->grad;
    if (!g) return;
    void *ptrs[] = {g->z0, g->ckpt, g->ring, g->ckst, g->efix_ring, g->escale_ring, g->box_hist,
                    g->box_replay, g->slot_hist, g->ghat_store, g->adj, g->kbar, g->phibar,
                    g->rb, g->amax, g->sexp, g->part, g->mbar, g->sums0, g->mom, g->perm};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete g;
    ctx->grad = nullptr;
}

static P6 p6(double *base, int64_t n) {
    P6 r;
    for (int k = 0; k < 6; ++k) r.p[k] = base + (size_t)k * n;
    return r;
}

static P6 p6(double *const c[6]) {
    P6 r;
    for (int k = 0; k < 6; ++k) r.p[k] = c[k];
    return r;
}

static int32_t grad_alloc(bx_ctx *ctx, int64_t np, int64_t K, int C) {
    GradTape *g = ctx->grad;
    const int n = ctx->n;
    if (g && g->np == np && g->K == K && g->C == C && g->n == n) return BX_OK;
    cudaDeviceSynchronize();
    grad_free(ctx);
    g = new (std::nothrow) GradTape();
    if (!g) return fail(ctx, BX_OUT_OF_MEMORY, "host allocation");
    ctx->grad = g;
    g->np = np;
    g->K = K;
    g->C = C;
    g->n = n;
    g->nseg = (int)((K + C - 1) / C);
    g->n3 = (long long)n * n * n;
    g->o3 = (long long)(n + 1) * (n + 1) * (n + 1);
    g->q3 = (long long)(n + 2) * (n + 2) * (n + 2);
    g->ghat_cap = (int)(K + 1);
    const size_t st6 = (size_t)6 * np * sizeof(double);
    cudaError_t e = cudaSuccess;
    auto A = [&](void **p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc(p, bytes < 8 ? 8 : bytes);
    };
    A((void **)&g->z0, st6);
    A((void **)&g->ckpt, st6 * g->nseg);
    A((void **)&g->ckst, sizeof(TrackState) * g->nseg);
    A((void **)&g->ring, st6 * (C + 1));
    A((void **)&g->efix_ring, sizeof(EFix) * g->n3 * C);
    A((void **)&g->escale_ring, sizeof(int) * 4 * C);
    A((void **)&g->box_hist, sizeof(Box) * K);
    A((void **)&g->box_replay, sizeof(Box) * K);
    A((void **)&g->slot_hist, sizeof(int32_t) * K);
    A((void **)&g->ghat_store, sizeof(double) * g->o3 * g->ghat_cap);
    A((void **)&g->adj, st6);
    A((void **)&g->kbar, sizeof(long long) * 3 * g->n3);
    A((void **)&g->phibar, sizeof(double) * g->q3);
    A((void **)&g->rb, sizeof(double) * g->q3);
    A((void **)&g->amax, sizeof(unsigned long long) * 12);
    A((void **)&g->sexp, sizeof(int) * 4);
    A((void **)&g->part, sizeof(double) * 49 * adj_blocks(np));
    A((void **)&g->mbar, sizeof(double) * 13 * (K + 1));
    A((void **)&g->sums0, sizeof(double) * 49);
    A((void **)&g->mom, sizeof(double) * 27);
    A((void **)&g->perm, sizeof(int) * np * g->nseg);
    if (e != cudaSuccess) {
        grad_free(ctx);
        return cuda_fail(ctx, e, "differentiation tape");
    }
    return BX_OK;
}

// Sets one pointer field of the device TrackState.
template <class T>
static cudaError_t set_state_ptr(TrackState *st, T *TrackState::*field, T *value, cudaStream_t s) {
    T *v = value;
    return cudaMemcpyAsync(&(st->*field), &v, sizeof(v), cudaMemcpyHostToDevice, s);
}

// Kick pieces shared by the forward and the recompute.  `load` replaces the
// Green's function build by the stored spectrum.
static cudaError_t grad_green(bx_ctx *ctx, bool load, cudaStream_t s) {
    GradTape *g = ctx->grad;
    cudaError_t e = cudaSuccess;
    if (!load) {
        e = launch_igf_table(ctx->n, nullptr, ctx->fcorner, ctx->gtable, s, ctx->st);
        if (e == cudaSuccess)
            e = green_spectrum_from_table(&ctx->plan, ctx->gtable, s, &ctx->st->green_stale);
    }
    if (e == cudaSuccess)
        e = launch_ghat_store(ctx->st, g->ghat_store, ctx->plan.ghat, g->o3, g->ghat_cap,
                              load ? 1 : 0, ctx->status, s);
    // a loaded spectrum: its copy for the block-floating-point solve
    if (e == cudaSuccess && load) e = green_quantize(&ctx->plan, s, &ctx->st->green_stale);
    if (e == cudaSuccess) e = launch_green_commit(ctx->st, s);
    return e;
}

static cudaError_t grad_kick(bx_ctx *ctx, double *const cin[6], double *const cout[6],
                             EFix *efix, int *escale, bool load, bool force_deposit,
                             cudaStream_t s) {
    GradTape *g = ctx->grad;
    const int64_t np = g->np;
    const double bg = g->ref.bg;
    cudaError_t e = launch_box_rule(ctx->st, ctx->n, np, ctx->log, ctx->log_cap, true, s);
    if (e == cudaSuccess) e = grad_green(ctx, load, s);
    if (e == cudaSuccess && force_deposit) e = launch_set_deposit_gate(ctx->st, s);
    if (e == cudaSuccess)
        e = launch_track_deposit(cin, np, bg, &ctx->st->box, ctx->n, ctx->acc_hi, ctx->acc_lo,
                                 ctx->st, ctx->status, s);
    if (e == cudaSuccess)
        e = solve_acc_to_phi_fixed(&ctx->plan, ctx->acc_hi, ctx->acc_lo, 0.0, ctx->phi, s,
                                   &ctx->st->rho_scale);
    if (e == cudaSuccess)
        e = launch_field(ctx->phi, ctx->n, &ctx->st->box, 0.0, 0.0, 0.0, ctx->emax,
                         efix, escale, s, ctx->st, ctx->maps);
    if (e == cudaSuccess)
        e = launch_track_particles_oop(cin, cout, np, bg, &ctx->st->box, ctx->n, efix, escale,
                                       ctx->maps, ctx->acc_hi, ctx->acc_lo, ctx->st, ctx->status,
                                       s);
    return e;
}

// dH/dk of a quadrupole piece ds (zero for other elements): the x block is
// d/dk of the focusing block of k, the y block minus that of -k.
static void focus_block_dk(double ds, double k, double out[2][2]) {
    if (k > 0.0) {
        const double w = std::sqrt(k), c = std::cos(w * ds), s = std::sin(w * ds), dw = 0.5 / w;
        out[0][0] = -ds * s * dw;
        out[0][1] = (ds * c * w - s) / (w * w) * dw;
        out[1][0] = (-s - w * ds * c) * dw;
        out[1][1] = -ds * s * dw;
    } else if (k < 0.0) {
        const double w = std::sqrt(-k), c = std::cosh(w * ds), s = std::sinh(w * ds), dw = -0.5 / w;
        out[0][0] = ds * s * dw;
        out[0][1] = (ds * c * w - s) / (w * w) * dw;
        out[1][0] = (s + w * ds * c) * dw;
        out[1][1] = ds * s * dw;
    } else {
        out[0][0] = -ds * ds / 2.0;
        out[0][1] = -ds * ds * ds / 6.0;
        out[1][0] = -ds;
        out[1][1] = -ds * ds / 2.0;
    }
}

static const int kMbarRow[13] = {0, 0, 0, 1, 1, 1, 2, 2, 3, 3, 4, 4, 4};
static const int kMbarCol[13] = {0, 1, 5, 0, 1, 5, 2, 3, 2, 3, 0, 1, 5};

}  // namespace bt

using namespace bt;

extern "C" {

int32_t bx_twiss_beam(const double twiss[8], const double *const xi[6], int64_t n,
                      double *const out[6], void *stream) {
    if (!twiss || !xi || !out) return set_noctx_error(BX_BAD_ARG, "NULL argument");
    if (n < 0) return set_noctx_error(BX_BAD_ARG, "n < 0");
    for (int k = 0; k < 6 && n > 0; ++k)
        if (!xi[k] || !out[k]) return set_noctx_error(BX_BAD_ARG, "NULL coordinate pointer");
    const double bx = twiss[1], ex = twiss[2], by = twiss[4], ey = twiss[5];
    for (int k = 0; k < 8; ++k)
        if (!std::isfinite(twiss[k])) return set_noctx_error(BX_BAD_ARG, "Twiss parameters not finite");
    if (!(bx > 0.0) || !(by > 0.0) || !(ex >= 0.0) || !(ey >= 0.0))
        return set_noctx_error(BX_BAD_ARG, "beta must be > 0 and emittance >= 0");
    const double c[8] = {std::sqrt(ex * bx), std::sqrt(ex / bx), twiss[0],
                         std::sqrt(ey * by), std::sqrt(ey / by), twiss[3], twiss[6], twiss[7]};
    P6 pi, po;
    for (int k = 0; k < 6; ++k) {
        pi.p[k] = const_cast<double *>(xi[k]);
        po.p[k] = out[k];
    }
    cudaError_t e = launch_twiss_beam(pi, n, c, po, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    return BX_OK;
}

int32_t bx_distribution_beam(int32_t kind, const double params[9],
                             const double *const normals[6], const double *uniforms, int64_t n,
                             double *const out[6], void *stream) {
    if (!params || !normals || !out) return set_noctx_error(BX_BAD_ARG, "NULL argument");
    if (kind != 0 && kind != 1) return set_noctx_error(BX_BAD_ARG, "kind must be 0 or 1");
    if (n < 0) return set_noctx_error(BX_BAD_ARG, "n < 0");
    if (n > 0) {
        for (int k = 0; k < 6; ++k)
            if (!normals[k] || !out[k]) return set_noctx_error(BX_BAD_ARG, "NULL coordinate pointer");
        if (kind == 1 && !uniforms) return set_noctx_error(BX_BAD_ARG, "uniforms is NULL");
    }
    Coef9 c9;
    double *c = c9.c;
    for (int pl = 0; pl < 3; ++pl) {
        const double lam = params[pl], lamp = params[3 + pl], mu = params[6 + pl];
        if (!std::isfinite(lam) || !std::isfinite(lamp) || !(std::fabs(mu) < 1.0))
            return set_noctx_error(BX_BAD_ARG, "parameters must be finite with |mu| < 1");
        const double root = std::sqrt(1.0 - mu * mu);
        c[3 * pl] = lam / root;
        c[3 * pl + 1] = lamp;
        c[3 * pl + 2] = mu / root;
    }
    if (n == 0) return BX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    P6 pz, po;
    for (int k = 0; k < 6; ++k) {
        pz.p[k] = const_cast<double *>(normals[k]);
        po.p[k] = out[k];
    }
    const cudaError_t e = launch_distribution(kind, pz, uniforms, n, c9, po, s);
    if (e != cudaSuccess) return set_noctx_error(BX_CUDA, cudaGetErrorString(e));
    return BX_OK;
}

int32_t bx_twiss_grad(const double twiss[8], const double S[36], double out[6]) {
    if (!twiss || !S || !out) return set_noctx_error(BX_BAD_ARG, "NULL argument");
    // S[i*6 + j] = sum_p zbar0_i z0_j.  With u = sqrt(eps beta) xi_u and
    // pu = sqrt(eps/beta)(xi_pu - alpha xi_u): du/dbeta = u/(2 beta),
    // dpu/dbeta = -pu/(2 beta), du/deps = u/(2 eps), dpu/deps = pu/(2 eps),
    // dpu/dalpha = -u/beta.
    for (int pl = 0; pl < 2; ++pl) {
        const int u = 2 * pl, pu = u + 1;
        const double a = twiss[3 * pl], b = twiss[3 * pl + 1], e = twiss[3 * pl + 2];
        (void)a;
        const double suu = S[u * 6 + u], spp = S[pu * 6 + pu], spu = S[pu * 6 + u];
        out[3 * pl + 0] = -spu / b;
        out[3 * pl + 1] = (suu - spp) / (2.0 * b);
        out[3 * pl + 2] = e > 0.0 ? (suu + spp) / (2.0 * e) : 0.0;
    }
    return BX_OK;
}

int32_t bx_objectives(const double moments[27], double out[4]) {
    if (!moments || !out) return set_noctx_error(BX_BAD_ARG, "NULL argument");
    // row-major upper triangle after the six means: <xx> = 6, <x px> = 7,
    // <px px> = 12, <yy> = 17, <y py> = 18, <py py> = 21
    const double cxx = moments[6], cxp = moments[7], cpp = moments[12];
    const double cyy = moments[17], cyq = moments[18], cqq = moments[21];
    out[0] = std::sqrt(cxx * cpp - cxp * cxp);
    out[1] = std::sqrt(cyy * cqq - cyq * cyq);
    out[2] = std::sqrt(cxx);
    out[3] = std::sqrt(cyy);
    for (int k = 0; k < 4; ++k)
        if (!std::isfinite(out[k])) return set_noctx_error(BX_NONFINITE, "objective not finite");
    return BX_OK;
}

int32_t bx_family_grad(const double *dk_element, const int32_t *family, int32_t count,
                       int32_t nfamilies, double *dk_family) {
    if (!dk_element || !family || !dk_family || count < 0 || nfamilies < 0)
        return set_noctx_error(BX_BAD_ARG, "NULL argument or negative count");
    for (int32_t f = 0; f < nfamilies; ++f) dk_family[f] = 0.0;
    for (int32_t e = 0; e < count; ++e) {
        const int32_t f = family[e];
        if (f < -1 || f >= nfamilies) return set_noctx_error(BX_BAD_ARG, "family index out of range");
        if (f >= 0) dk_family[f] += dk_element[e];
    }
    return BX_OK;
}

int32_t bx_grad_forward(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat,
                        int32_t checkpoint_interval, const double *box_replay, void *stream) {
    if (!ctx) return set_noctx_error(BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_lattice(ctx, lat))) return rc;
    if (beam->n <= 0) return fail(ctx, BX_BAD_ARG, "differentiation needs particles");
    if (ctx_sharded(ctx)) return fail(ctx, BX_BAD_ARG, "differentiation of a sharded run is not supported");
    if (checkpoint_interval <= 0) return fail(ctx, BX_BAD_ARG, "checkpoint_interval must be >= 1");
    if (ctx->shape != 1)
        return fail(ctx, BX_BAD_ARG, "the reverse mode supports particle shape 1 (CIC) only");
    if (lattice_has_multipoles(lat))
        return fail(ctx, BX_BAD_ARG, "the reverse mode supports linear thin elements only (no multipoles)");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int> sel;
    std::vector<double> sds;
    slice_schedule(lat, sel, sds);
    const int64_t K = (int64_t)sel.size();
    if (K == 0) return fail(ctx, BX_BAD_ARG, "empty lattice");
    const int C = (int)std::min<int64_t>(checkpoint_interval, K);
    if ((rc = grad_alloc(ctx, beam->n, K, C))) return rc;
    GradTape *g = ctx->grad;
    g->valid = false;
    g->elements.assign(lat->elements, lat->elements + lat->count);
    g->sel = sel;
    g->sds = sds;
    g->ref = make_ref(beam);
    g->q_macro = lat->space_charge
                     ? g->ref.sign * std::fabs(beam->bunch_charge_C) / (double)beam->n
                     : 0.0;
    for (int k = 0; k < 6; ++k) g->coord[k] = beam->coord[k];
    std::vector<MapCoef> tab;
    build_map_table(lat, sel, sds, 0, K, g->ref, tab);
    if ((rc = ensure_maps(ctx, tab.size()))) return rc;
    CK(cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                       cudaMemcpyHostToDevice, s),
       "upload maps");
    if (box_replay) {
        std::vector<Box> bx(K);
        for (int64_t k = 0; k < K; ++k) {
            const double *r = box_replay + 12 * k;
            for (int d = 0; d < 3; ++d) {
                bx[k].lo[d] = r[d];
                bx[k].hi[d] = r[3 + d];
                bx[k].h[d] = r[6 + d];
                bx[k].inv_h[d] = r[9 + d];
                if (!(bx[k].h[d] > 0.0) || !std::isfinite(bx[k].lo[d]) || !std::isfinite(bx[k].inv_h[d]))
                    return fail(ctx, BX_BAD_ARG, "replayed box invalid");
            }
        }
        CK(cudaMemcpyAsync(g->box_replay, bx.data(), sizeof(Box) * K, cudaMemcpyHostToDevice, s),
           "upload boxes");
        CK(cudaStreamSynchronize(s), "sync");
    }
    // fresh state: no box, no Green's function, kick counter 0
    TrackState h;
    init_state(&h);
    CK(cudaMemcpyAsync(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice, s), "state");
    CK(cudaStreamSynchronize(s), "sync");
    ctx->kick = 0;
    ctx->green_valid = false;
    CK(launch_call_init(ctx->st, (int)K, g->q_macro, 0, 0, s, g->ref.bg), "call init");
    CK(set_state_ptr<Box>(ctx->st, &TrackState::box_hist, g->box_hist, s), "state");
    CK(set_state_ptr<int32_t>(ctx->st, &TrackState::slot_hist, g->slot_hist, s), "state");
    {
        const Box *rp = box_replay ? g->box_replay : nullptr;
        CK(cudaMemcpyAsync(&ctx->st->box_replay, &rp, sizeof(rp), cudaMemcpyHostToDevice, s),
           "state");
    }
    double *const *c = beam->coord;
    const size_t bytes = (size_t)beam->n * sizeof(double);
    if (beam->id) {
        // bin the initial bunch by grid brick (of a box around it), so the
        // deposits and the reverse scatter touch compact sets of cells (each
        // later segment starts with another re-binning)
        if ((rc = ensure_sort_scratch(ctx, beam->n))) return rc;
        CK(sort_set_pointers(c, ctx->scr, ctx->dev_ptrs, s), "sort pointers");
        CK(launch_minmax(c, beam->n, g->ref.bg, ctx->st, ctx->status, s), "minmax");
        CK(launch_box_rule(ctx->st, ctx->n, beam->n, ctx->log, ctx->log_cap, false, s), "box");
        CK(launch_sort(c, (long long *)beam->id, beam->n, g->ref.bg, &ctx->st->box, ctx->n,
                       sort_brick_edge(ctx->n, ctx->bin_edge), ctx->keys, ctx->counts,
                       ctx->offs, ctx->sums, ctx->scr, ctx->id_scr, ctx->dev_ptrs, s),
           "initial binning");
        CK(cudaMemcpyAsync(ctx->st, &h, sizeof(h), cudaMemcpyHostToDevice, s), "state");
        CK(launch_call_init(ctx->st, (int)K, g->q_macro, 0, 0, s, g->ref.bg), "call init");
        CK(set_state_ptr<Box>(ctx->st, &TrackState::box_hist, g->box_hist, s), "state");
        CK(set_state_ptr<int32_t>(ctx->st, &TrackState::slot_hist, g->slot_hist, s), "state");
        const Box *rp = box_replay ? g->box_replay : nullptr;
        CK(cudaMemcpyAsync(&ctx->st->box_replay, &rp, sizeof(rp), cudaMemcpyHostToDevice, s),
           "state");
        CK(cudaStreamSynchronize(s), "sync");
    }
    for (int k = 0; k < 6; ++k)
        CK(cudaMemcpyAsync(g->z0 + (size_t)k * beam->n, c[k], bytes, cudaMemcpyDeviceToDevice, s),
           "save z0");
    CK(launch_push_maps(c, beam->n, ctx->maps, 1, s, ctx->status, ctx->st, g->ref.bg), "push");
    g->binned = beam->id != nullptr;
    for (int64_t k = 0; k < K; ++k) {
        if (k % C == 0) {
            const int64_t sg = k / C;
            if (sg > 0 && g->binned)
                // re-bin (the order decays as the lattice turns phase space),
                // keeping where each particle went for the reverse pass
                CK(launch_sort(c, (long long *)beam->id, beam->n, g->ref.bg, &ctx->st->box, ctx->n,
                               sort_brick_edge(ctx->n, ctx->bin_edge), ctx->keys, ctx->counts,
                               ctx->offs, ctx->sums, ctx->scr, ctx->id_scr, ctx->dev_ptrs, s,
                               nullptr, g->perm + (size_t)sg * beam->n),
                   "re-binning");
            double *dst = g->ckpt + (size_t)sg * 6 * beam->n;
            for (int q = 0; q < 6; ++q)
                CK(cudaMemcpyAsync(dst + (size_t)q * beam->n, c[q], bytes, cudaMemcpyDeviceToDevice, s),
                   "checkpoint");
            CK(cudaMemcpyAsync(g->ckst + sg, ctx->st, sizeof(TrackState), cudaMemcpyDeviceToDevice, s),
               "checkpoint state");
        }
        CK(grad_kick(ctx, c, c, ctx->efix, ctx->escale, false, false, s), "kick");
    }
    ctx->kick = K;
    g->valid = true;
    return BX_OK;
}

int32_t bx_grad_backward(bx_ctx *ctx, const bx_beam *beam, const double weights[4],
                         double *dk_out, double *S_out, double *const zbar0[6], void *stream) {
    if (!ctx) return set_noctx_error(BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    GradTape *g = ctx->grad;
    if (!g || !g->valid) return fail(ctx, BX_BAD_ARG, "no differentiation forward pass recorded");
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if (!weights) return fail(ctx, BX_BAD_ARG, "weights is NULL");
    if (beam->n != g->np) return fail(ctx, BX_BAD_ARG, "beam differs from the forward pass");
    for (int k = 0; k < 6; ++k)
        if (beam->coord[k] != g->coord[k])
            return fail(ctx, BX_BAD_ARG, "beam arrays differ from the forward pass");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t np = g->np, K = g->K;
    const int C = g->C;
    // dL/dz of the final bunch
    if ((rc = ensure_moment_scratch(ctx, np))) return rc;
    CK(launch_moments(beam->coord, np, ctx->mom_partial, moments_blocks(np), g->mom, ctx->status, s), "moments");
    P6 adj = p6(g->adj, np);
    CK(launch_adj_seed(p6(beam->coord), np, g->mom, weights, adj, g->amax, s), "seed");
    unsigned long long *cur = g->amax, *nxt = g->amax + 6;
    const size_t st6 = (size_t)6 * np;
    for (int sg = g->nseg - 1; sg >= 0; --sg) {
        const int64_t k0 = (int64_t)sg * C, k1 = std::min<int64_t>(K, k0 + C);
        // recompute the segment from its checkpoint, keeping every state and field
        CK(cudaMemcpyAsync(g->ring, g->ckpt + (size_t)sg * st6, st6 * sizeof(double),
                           cudaMemcpyDeviceToDevice, s),
           "restore");
        CK(cudaMemcpyAsync(ctx->st, g->ckst + sg, sizeof(TrackState), cudaMemcpyDeviceToDevice, s),
           "restore state");
        // the spectrum in use at the segment's first kick (recorded slot); the
        // recompute then loads a stored spectrum wherever the forward built one
        CK(launch_ghat_fetch(g->slot_hist, k0, g->ghat_store, ctx->plan.ghat, g->o3, g->ghat_cap, s),
           "spectrum");
        CK(green_quantize(&ctx->plan, s), "spectrum");
        for (int64_t k = k0; k < k1; ++k) {
            const int64_t j = k - k0;
            P6 pin = p6(g->ring + (size_t)j * st6, np), pout = p6(g->ring + (size_t)(j + 1) * st6, np);
            CK(grad_kick(ctx, pin.p, pout.p, g->efix_ring + (size_t)j * g->n3, g->escale_ring + 4 * j,
                         true, j == 0, s),
               "recompute");
        }
        // reverse through the segment
        for (int64_t k = k1 - 1; k >= k0; --k) {
            const int64_t j = k - k0;
            AdjKick a{};
            a.P = p6(g->ring + (size_t)j * st6, np);
            a.A = adj;
            a.ef = g->efix_ring + (size_t)j * g->n3;
            a.escale = g->escale_ring + 4 * j;
            a.box = g->box_hist + k;
            a.map = ctx->maps + 1 + k;
            a.betagamma = g->ref.bg;
            a.q_macro = g->q_macro;
            a.nn = ctx->n;
            a.n = np;
            a.kick = k;
            a.amax_in = cur;
            a.amax_out = nxt;
            a.kbar = g->kbar;
            a.sexp = g->sexp;
            a.part = g->part;
            a.mbar = g->mbar + (size_t)13 * (1 + k);
            a.phibar = g->phibar;
            a.rb = g->rb;
            a.plan = &ctx->plan;
            a.slot_hist = g->slot_hist;
            a.ghat_store = g->ghat_store;
            a.ghat_count = g->o3;
            a.ghat_cap = g->ghat_cap;
            CK(launch_adj_kick(a, s), "adjoint kick");
            std::swap(cur, nxt);
        }
        if (sg > 0 && g->binned) {
            // the segment started with a re-binning: back to the order before it
            P6 tmp = p6(g->ring + st6, np);
            CK(launch_permute6(adj, g->perm + (size_t)sg * np, np, tmp, true, s), "un-binning");
            CK(cudaMemcpyAsync(g->adj, g->ring + st6, st6 * sizeof(double), cudaMemcpyDeviceToDevice, s),
               "un-binning");
        }
    }
    P6 out = adj;
    if (zbar0) out = p6(zbar0);
    CK(launch_adj_initial(adj, p6(g->z0, np), np, ctx->maps, out, g->part, g->sums0, s), "initial");
    if (zbar0 && g->binned)
        // dL/dz0 in the beam's (final) particle order: the segments' re-binnings
        // in forward order
        for (int sg = 1; sg < g->nseg; ++sg) {
            P6 tmp = p6(g->ring + st6, np);
            CK(launch_permute6(out, g->perm + (size_t)sg * np, np, tmp, false, s), "re-binning");
            for (int q = 0; q < 6; ++q)
                CK(cudaMemcpyAsync(out.p[q], tmp.p[q], (size_t)np * sizeof(double),
                                   cudaMemcpyDeviceToDevice, s),
                   "re-binning");
        }
    std::vector<double> mbar((size_t)13 * (K + 1)), sums(49);
    CK(cudaMemcpyAsync(mbar.data() + 13, g->mbar + 13, sizeof(double) * 13 * K,
                       cudaMemcpyDeviceToHost, s),
       "read map adjoints");
    CK(cudaMemcpyAsync(sums.data(), g->sums0, sizeof(double) * 49, cudaMemcpyDeviceToHost, s),
       "read sums");
    // the spectrum in the plan no longer matches the state's h
    const double zero3[3] = {0.0, 0.0, 0.0};
    CK(cudaMemcpyAsync(ctx->st->green_h, zero3, sizeof(zero3), cudaMemcpyHostToDevice, s), "state");
    CK(cudaStreamSynchronize(s), "sync");
    g->valid = false;
    for (int q = 0; q < 13; ++q) mbar[q] = sums[q];
    if (S_out)
        for (int q = 0; q < 36; ++q) S_out[q] = sums[13 + q];
    if (dk_out) {
        // chain rule through the merged maps to each half-slice map H_k, then
        // dL/dk of the quadrupoles from dH/dk in closed form
        const int ne = (int)g->elements.size();
        for (int e = 0; e < ne; ++e) dk_out[e] = 0.0;
        std::vector<std::array<double, 36>> hbar(K);
        for (auto &a : hbar) a.fill(0.0);
        std::vector<std::array<double, 36>> H(K);
        for (int64_t k = 0; k < K; ++k) {
            Mat m;
            element_map(g->elements[g->sel[k]], 0.5 * g->sds[k], g->ref, m);
            for (int i = 0; i < 6; ++i)
                for (int jj = 0; jj < 6; ++jj) H[k][6 * i + jj] = m[i][jj];
        }
        // thin elements between the slices (no parameters; carried through)
        std::vector<Mat6> pre;
        Mat6 post;
        const bx_lattice lat_rec{g->elements.data(), (int32_t)g->elements.size(), 1};
        thin_maps(&lat_rec, g->ref, pre, post);
        auto mul = [](const double *a, const double *b, double *out) {  // out = a b
            double t[36];
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    double s = 0.0;
                    for (int l = 0; l < 6; ++l) s += a[6 * i + l] * b[6 * l + j];
                    t[6 * i + j] = s;
                }
            memcpy(out, t, sizeof(t));
        };
        auto mul_bt = [](const double *a, const double *b, double *acc) {  // acc += a b^T
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    double s = 0.0;
                    for (int l = 0; l < 6; ++l) s += a[6 * i + l] * b[6 * j + l];
                    acc[6 * i + j] += s;
                }
        };
        auto mul_at = [](const double *a, const double *b, double *acc) {  // acc += a^T b
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) {
                    double s = 0.0;
                    for (int l = 0; l < 6; ++l) s += a[6 * l + i] * b[6 * l + j];
                    acc[6 * i + j] += s;
                }
        };
        // M_0 = H_0 T_pre(0); M_t = H_t T_pre(t) H_{t-1}; M_K = T_post H_{K-1}:
        // the adjoint of each half map is Mbar times the other factors
        for (int64_t t = 0; t <= K; ++t) {
            double mb[36] = {0};
            for (int q = 0; q < 13; ++q) mb[6 * kMbarRow[q] + kMbarCol[q]] = mbar[13 * t + q];
            if (t == 0) {
                mul_bt(mb, &pre[0].a[0][0], hbar[0].data());
            } else if (t == K) {
                mul_at(&post.a[0][0], mb, hbar[K - 1].data());
            } else {
                double right[36], left[36];
                mul(&pre[t].a[0][0], H[t - 1].data(), right);   // T_pre(t) H_{t-1}
                mul(H[t].data(), &pre[t].a[0][0], left);         // H_t T_pre(t)
                mul_bt(mb, right, hbar[t].data());
                mul_at(left, mb, hbar[t - 1].data());
            }
        }
        for (int64_t k = 0; k < K; ++k) {
            const bx_element &el = g->elements[g->sel[k]];
            if (el.type != BX_QUAD) continue;
            double bxk[2][2], byk[2][2];
            focus_block_dk(0.5 * g->sds[k], el.k, bxk);
            focus_block_dk(0.5 * g->sds[k], -el.k, byk);
            double d = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int jj = 0; jj < 2; ++jj) {
                    d += hbar[k][6 * i + jj] * bxk[i][jj];
                    d -= hbar[k][6 * (2 + i) + (2 + jj)] * byk[i][jj];
                }
            dk_out[g->sel[k]] += d;
        }
    }
    return BX_OK;
}

int32_t bx_grad_boxes(bx_ctx *ctx, double *out, int64_t cap, int64_t *count) {
    if (!ctx) return set_noctx_error(BX_BAD_ARG, "NULL context");
    GradTape *g = ctx->grad;
    if (!g || !count) return fail(ctx, BX_BAD_ARG, "no differentiation forward pass recorded");
    *count = g->K;
    const int64_t k = std::min<int64_t>(cap, g->K);
    if (k > 0 && out) {
        std::vector<Box> bx(k);
        CK(cudaMemcpy(bx.data(), g->box_hist, sizeof(Box) * k, cudaMemcpyDeviceToHost), "boxes");
        for (int64_t i = 0; i < k; ++i)
            for (int d = 0; d < 3; ++d) {
                out[12 * i + d] = bx[i].lo[d];
                out[12 * i + 3 + d] = bx[i].hi[d];
                out[12 * i + 6 + d] = bx[i].h[d];
                out[12 * i + 9 + d] = bx[i].inv_h[d];
            }
    }
    return BX_OK;
}

}  // extern "C"
