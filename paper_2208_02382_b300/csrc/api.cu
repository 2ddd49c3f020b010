// C ABI of libbeamtrack (declared in include/beamtrack.h): the context, the
// split-operator tracking loop (device-driven kicks, one CUDA graph per kick)
// and the single-step calls (deposit, solve, gather + kick, moments).
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

#include "ctx.cuh"

using namespace bt;


int32_t bt::set_noctx_error(int32_t code, const char *msg) { return fail(nullptr, code, msg); }

extern "C" {

int32_t bx_create(bx_ctx **out, const bx_options *opt) {
    if (!out || !opt) return fail(nullptr, BX_BAD_ARG, "NULL argument");
    *out = nullptr;
    int n = opt->n_grid;
    if (n < 8 || n > 256 || (n & (n - 1)) != 0)
        return fail(nullptr, BX_BAD_ARG, "n_grid must be a power of two in [8, 256]");
    if (opt->shape_order != 1 && opt->shape_order != 2)
        return fail(nullptr, BX_BAD_ARG, "shape_order must be 1 (CIC) or 2 (TSC)");
    if (opt->rebin_interval < -1) return fail(nullptr, BX_BAD_ARG, "rebin_interval must be >= -1");
    if (opt->bin_edge != 0 && !sort_brick_edge_valid(n, opt->bin_edge))
        return fail(nullptr, BX_BAD_ARG,
                    "bin_edge must be 0 or a power of two in [2, n/2] giving at most 16^3 bins");
    if (opt->cell_order != 0 && opt->cell_order != 1)
        return fail(nullptr, BX_BAD_ARG, "cell_order must be 0 or 1");
    bx_ctx *ctx = new (std::nothrow) bx_ctx();
    if (!ctx) return fail(nullptr, BX_OUT_OF_MEMORY, "host allocation");
    ctx->n = n;
    ctx->sort_interval = opt->rebin_interval == 0 ? 16 : opt->rebin_interval < 0 ? 0 : opt->rebin_interval;
    ctx->bin_edge = opt->bin_edge;
    ctx->cell_order = opt->cell_order != 0;
    ctx->shape = opt->shape_order;
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
    A((void **)&ctx->fcorner, igf_scratch_doubles(n) * sizeof(double));
    A((void **)&ctx->gtable, o3 * 8);
    A((void **)&ctx->st, sizeof(TrackState));
    A((void **)&ctx->tmp_box, sizeof(Box));
    A((void **)&ctx->status, sizeof(int32_t));
    A((void **)&ctx->log, ctx->log_cap * sizeof(long long));
    A((void **)&ctx->efix, n3 * sizeof(EFix));
    A((void **)&ctx->emax, 3 * sizeof(unsigned long long));
    A((void **)&ctx->escale, 4 * sizeof(int));
    A((void **)&ctx->dev_ptrs, 24 * sizeof(double *));
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
    grad_free(ctx);
    void *ptrs[] = {ctx->acc_hi, ctx->acc_lo, ctx->rho, ctx->phi, ctx->fcorner,
                    ctx->gtable, ctx->st, ctx->tmp_box, ctx->status, ctx->log,
                    ctx->mom_partial, ctx->maps, ctx->efix, ctx->emax, ctx->escale,
                    ctx->dev_ptrs, ctx->keys, ctx->counts, ctx->offs, ctx->sums, ctx->id_scr,
                    ctx->scr[0], ctx->scr[1], ctx->scr[2], ctx->scr[3], ctx->scr[4], ctx->scr[5],
                    ctx->cells};
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

}  // extern "C"

namespace {

// Moments at every slice end (Listing 1 set_slice_step_diagnostics): after
// kick k the bunch holds P_{k+1} = H_first(k+1) T_pre(k+1) S_k with S_k the
// state at the end of slice k (T_pre: thin elements in between), so the
// moments of S_k are those of P_{k+1} taken back through the inverse of that
// product; after the last kick of the call the bunch is at the slice end, or
// past the thin elements that end the lattice.
int32_t slice_diagnostics(bx_ctx *ctx, const bx_lattice *lat, const std::vector<int> &sel,
                          const std::vector<double> &sds, int64_t first, int64_t nkicks,
                          const Ref &r, std::vector<MapCoef> &inv) {
    (void)ctx;
    std::vector<Mat6> pre;
    Mat6 post;
    thin_maps(lat, r, pre, post);
    const int64_t total = (int64_t)sel.size();
    inv.assign(nkicks, MapCoef{});
    for (int64_t k = 0; k < nkicks; ++k) {
        Mat m, mi;
        const int64_t j = first + k;
        if (k + 1 < nkicks) {
            Mat h;
            element_map(lat->elements[sel[j + 1]], 0.5 * sds[j + 1], r, h);
            mat_mul(h, pre[j + 1].a, m);   // P_{k+1} = H_first T_pre S_k
        } else if (j + 1 == total) {
            memcpy(m, post.a, sizeof(Mat));
        } else {
            mat_identity(m);
        }
        mat_inverse(m, mi);
        inv[k] = to_coef(mi);
    }
    return BX_OK;
}

int32_t track_impl(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat, int64_t first_kick,
                   int64_t nkicks, double *diag, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    ProfScope prof_scope(ctx->prof);
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_lattice(ctx, lat))) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // slice schedule: (element, ds) per kick
    std::vector<int> sel;
    std::vector<double> sds;
    slice_schedule(lat, sel, sds);
    const int64_t total = (int64_t)sel.size();
    if (nkicks < 0) nkicks = total - first_kick;
    if (first_kick < 0 || first_kick > total || nkicks < 0 || first_kick + nkicks > total)
        return fail(ctx, BX_BAD_ARG, "kick range outside the slice schedule");
    if (nkicks == 0) return BX_OK;
    const bool sharded = ctx_sharded(ctx);
    if (sharded && diag)
        return fail(ctx, BX_BAD_ARG, "per-slice diagnostics of a sharded run are not supported");
    if (sharded && beam->n > ctx->shard.n_total)
        return fail(ctx, BX_BAD_ARG, "the rank holds more particles than the shard's n_total");
    if (diag && lattice_has_multipoles(lat))
        return fail(ctx, BX_BAD_ARG,
                    "per-slice diagnostics need a lattice without thin multipoles (their moments "
                    "do not carry back through a nonlinear kick)");
    const Ref r = make_ref(beam);
    // map table: H_first, H_{k+1} H_k for inner boundaries, H_last
    std::vector<MapCoef> tab;
    build_map_table(lat, sel, sds, first_kick, nkicks, r, tab);
    if ((rc = ensure_maps(ctx, tab.size()))) return rc;
    CK(cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                       cudaMemcpyHostToDevice, s),
       "upload maps");
    // (a rank of a sharded run with no particles still takes part in every
    // kick's collectives, with empty extents and no charge)
    if (beam->n == 0 && !(sharded && lat->space_charge)) {
        ctx->kick += nkicks;
        return BX_OK;
    }
    double *const *c = beam->coord;
    std::vector<MapCoef> inv;
    MapCoef *inv_dev = nullptr;
    if (diag) {
        slice_diagnostics(ctx, lat, sel, sds, first_kick, nkicks, r, inv);
        if ((rc = ensure_maps(ctx, tab.size() + inv.size()))) return rc;
        // (re-)upload the map table: the buffer may have grown
        CK(cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                           cudaMemcpyHostToDevice, s),
           "upload maps");
        inv_dev = ctx->maps + tab.size();
        CK(cudaMemcpyAsync(inv_dev, inv.data(), inv.size() * sizeof(MapCoef),
                           cudaMemcpyHostToDevice, s),
           "upload inverse maps");
        if ((rc = ensure_moment_scratch(ctx, beam->n))) return rc;
    }
    const int mom_nb = moments_blocks(beam->n);
    auto diag_after = [&](int64_t k) -> cudaError_t {
        cudaError_t e = launch_moments(c, beam->n, ctx->mom_partial, mom_nb, diag + 27 * k, ctx->status, s);
        if (e == cudaSuccess) e = launch_moments_transform(diag + 27 * k, inv_dev + k, s);
        return e;
    };
    if (!lat->space_charge) {
        if (!diag) {
            // maps only: H_first, merged pairs, H_last in one pass per particle
            CK(launch_push_maps(c, beam->n, ctx->maps, (int)(nkicks + 1), s, ctx->status), "push");
        } else {
            CK(launch_push_maps(c, beam->n, ctx->maps, 1, s, ctx->status), "push");
            for (int64_t k = 0; k < nkicks; ++k) {
                CK(launch_push_maps(c, beam->n, ctx->maps + 1 + k, 1, s, ctx->status), "push");
                CK(diag_after(k), "slice diagnostics");
            }
        }
        ctx->kick += nkicks;
        return BX_OK;
    }
    // macroparticle charge of the whole bunch (a shard's particles carry the
    // charge of the bunch's n_total)
    const double q_macro = r.sign * std::fabs(beam->bunch_charge_C) /
                           (double)(sharded ? ctx->shard.n_total : beam->n);
    const bool binning = beam->id != nullptr && beam->n > 0;
    if (binning && (rc = ensure_sort_scratch(ctx, beam->n))) return rc;
    if (ctx->shape == 1 && (rc = ensure_cells(ctx, beam->n))) return rc;
    // Device-driven kicks: the box rule kernel of each kick sets the gates
    // (Green's function rebuild, deposit of the current positions, re-binning,
    // deposit for a next kick) that the later kernels of the kick read, and the
    // per-kick map and kick factors come from the table at index 1 + k; no
    // host decision or synchronisation between kicks.
    CK(launch_call_init(ctx->st, (int)nkicks, q_macro, binning ? ctx->sort_interval : 0,
                        ctx->kick, s, r.bg, true),
       "call init");
    if (binning) CK(sort_set_pointers(c, ctx->scr, ctx->dev_ptrs, s), "sort pointers");
    CK(launch_track_prologue(c, beam->n, r.bg, &ctx->st->box, ctx->n, ctx->maps, ctx->acc_hi,
                             ctx->acc_lo, ctx->st, ctx->status, s, ctx->shape, shared_cells(ctx),
                             tab.data()),
       "prologue");
    const KickArgs ka{ctx, c, beam->id, beam->n, r.bg, binning};
    if (sharded) {
        for (int64_t k = 0; k < nkicks; ++k) {
            cudaError_t ce = cudaSuccess;
            rc = kick_sharded(ka, s, &ce);
            if (rc == BX_COLLECTIVE)
                return fail(ctx, BX_COLLECTIVE, "the shard's allreduce callback failed");
            if (rc) return cuda_fail(ctx, ce, "sharded kick");
        }
        ctx->kick += nkicks;
        ctx->green_valid = false;
        return BX_OK;
    }
    bool use_graph = !ctx->graphs_off && !profiler_timing(ctx->prof) && !diag;
    if (use_graph) {
        bool same = ctx->kick_exec && ctx->graph_n == beam->n && ctx->graph_id == beam->id &&
                    ctx->graph_bg == r.bg && ctx->graph_maps == ctx->maps &&
                    ctx->graph_sort_n == ctx->sort_n && ctx->graph_cells == ctx->cells;
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
                ctx->graph_maps = ctx->maps;
                ctx->graph_sort_n = ctx->sort_n;
                ctx->graph_cells = ctx->cells;
            }
        }
    }
    for (int64_t k = 0; k < nkicks; ++k) {
        if (use_graph) CK(cudaGraphLaunch(ctx->kick_exec, s), "kick graph");
        else CK(kick_plain(ka, s), "kick");
        if (diag) CK(diag_after(k), "slice diagnostics");
    }
    ctx->kick += nkicks;
    ctx->green_valid = false;  // the device may have rebuilt the spectrum for another h
    return BX_OK;
}

}  // namespace

extern "C" {

int32_t bx_track(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat, int64_t first_kick,
                 int64_t nkicks, void *stream) {
    return track_impl(ctx, beam, lat, first_kick, nkicks, nullptr, stream);
}

int32_t bx_track_diagnostics(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat,
                             int64_t first_kick, int64_t nkicks, double *moments_device,
                             void *stream) {
    if (!moments_device) return fail(ctx, BX_BAD_ARG, "moments_device is NULL");
    if (beam && beam->n == 0) return fail(ctx, BX_BAD_ARG, "diagnostics of an empty beam");
    return track_impl(ctx, beam, lat, first_kick, nkicks, moments_device, stream);
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
        Box b = explicit_box(grid->lo, grid->hi, ctx->n, r.bg);
        hb = b;
        CK(cudaMemcpyAsync(ctx->tmp_box, &b, sizeof(b), cudaMemcpyHostToDevice, s), "box");
        for (int d = 0; d < 3; ++d) grid->h[d] = b.h[d];
        box = ctx->tmp_box;
    } else {
        if (beam->n == 0) return fail(ctx, BX_BAD_ARG, "box rule needs particles");
        const double nbg = -r.bg;
        CK(cudaMemcpyAsync(&ctx->st->nbg, &nbg, sizeof(nbg), cudaMemcpyHostToDevice, s), "beta gamma");
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
    CK(launch_deposit(c, beam->n, r.bg, box, hb, ctx->n, ctx->acc_hi, ctx->acc_lo, ctx->status, s,
                      ctx->shape),
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
    box_finish(b, -r.bg);
    CK(cudaMemcpyAsync(ctx->tmp_box, &b, sizeof(b), cudaMemcpyHostToDevice, s), "box");
    const double kt = r.sign * ds / (r.mass_eV * (r.bg * r.bg));
    const double kz = -r.sign * ds / (r.mass_eV * r.bg);
    CK(launch_field(grid->phi, ctx->n, ctx->tmp_box, kt, kt, kz, ctx->emax,
                    ctx->efix, ctx->escale, s),
       "field");
    CK(launch_kick_push_deposit(beam->coord, beam->n, r.bg, ctx->tmp_box, b, ctx->n, ctx->efix,
                                ctx->escale, nullptr, false, nullptr, nullptr, nullptr,
                                ctx->status, s, ctx->shape),
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
    if ((rc = ensure_moment_scratch(ctx, beam->n))) return rc;
    CK(launch_moments(beam->coord, beam->n, ctx->mom_partial, moments_blocks(beam->n), out,
                      ctx->status, s),
       "moments");
    return BX_OK;
}

int32_t bx_selftest_wait_timeout(bx_ctx *ctx, double limit_ms, void *stream) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    if (!(limit_ms > 0.0 && limit_ms <= 10000.0))
        return fail(ctx, BX_BAD_ARG, "limit_ms must lie in (0, 10000]");
    CK(launch_wait_selftest(ctx->status, limit_ms, (cudaStream_t)stream), "wait self-test");
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

int32_t bx_set_shard(bx_ctx *ctx, const bx_shard *shard) {
    if (!ctx) return fail(nullptr, BX_BAD_ARG, "NULL context");
    if (!shard) {
        ctx->shard = bx_shard{};
        return BX_OK;
    }
    if (!shard->allreduce || shard->n_total <= 0)
        return fail(ctx, BX_BAD_ARG, "a shard needs an allreduce callback and n_total > 0");
    ctx->shard = *shard;
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
