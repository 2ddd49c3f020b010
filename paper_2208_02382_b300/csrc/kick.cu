// One device-driven kick as kernel pieces, and its CUDA graphs: the per-kick
// graph of bx_track and the one-launch graph of a batch of independent
// tracking problems (each a device-side WHILE loop over its kick body).
//
// Paper anchors (arXiv:2208.02382): Model Assumptions (map(ds/2) -> space-
// charge kick over ds -> map(ds/2) per slice) and Listing 1 (sim.evolve()
// over the lattice's slices).  The batch has no counterpart in the paper; it
// runs many lattice variants or bunches at once (e.g. a scan of quadrupole
// strengths), each exactly as bx_track would.
#include <cmath>
#include <new>

#include "ctx.cuh"

namespace bt {

// The deposit with its atomics spread over the block's particles when the
// context re-bins by cell (and the particles are re-binned at all).  Both
// forms give bitwise the same charge.
static bool spread_deposit(const bx_ctx *ctx, const KickArgs &k) {
    return ctx->cell_order && k.binning && ctx->shape == 1;
}

// The kernels of one device-driven kick, in pieces (so the graph builder can
// put the gated pieces into conditional bodies).
cudaError_t kick_green(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = launch_igf_table(ctx->n, nullptr, ctx->fcorner, ctx->gtable, s, ctx->st);
    if (e == cudaSuccess) e = green_spectrum_from_table(&ctx->plan, ctx->gtable, s, &ctx->st->green_stale);
    if (e == cudaSuccess) e = launch_green_commit(ctx->st, s);
    return e;
}

cudaError_t kick_sort(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_sort(k.c, (long long *)k.id, k.n, k.bg, &ctx->st->box, ctx->n,
                       sort_brick_edge(ctx->n, ctx->bin_edge), ctx->keys,
                       ctx->counts, ctx->offs, ctx->sums, ctx->scr, ctx->id_scr, ctx->dev_ptrs, s,
                       &ctx->st->sort_gate, nullptr, ctx->cell_order);
}

cudaError_t kick_deposit(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_track_deposit(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->acc_hi, ctx->acc_lo,
                                ctx->st, ctx->status, s, ctx->shape, shared_cells(ctx),
                                spread_deposit(ctx, k));
}

cudaError_t kick_solve_field_push(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = solve_acc_to_phi_fixed(&ctx->plan, ctx->acc_hi, ctx->acc_lo, 0.0, ctx->phi, s,
                                           &ctx->st->rho_scale);
    if (e == cudaSuccess)
        e = launch_field(ctx->phi, ctx->n, &ctx->st->box, 0.0, 0.0, 0.0, ctx->emax,
                         ctx->efix, ctx->escale, s, ctx->st, ctx->maps);
    if (e == cudaSuccess)
        e = launch_track_particles(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->efix, ctx->escale,
                                   ctx->maps, ctx->acc_hi, ctx->acc_lo, ctx->st, ctx->status, s, 1,
                                   ctx->shape, shared_cells(ctx));
    return e;
}

cudaError_t kick_next_deposit(const KickArgs &k, cudaStream_t s) {
    bx_ctx *ctx = k.ctx;
    return launch_track_particles(k.c, k.n, k.bg, &ctx->st->box, ctx->n, ctx->efix, ctx->escale,
                                  ctx->maps, ctx->acc_hi, ctx->acc_lo, ctx->st, ctx->status, s, 2,
                                  ctx->shape, shared_cells(ctx), spread_deposit(ctx, k));
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

int32_t kick_sharded(const KickArgs &k, cudaStream_t s, cudaError_t *err) {
    bx_ctx *ctx = k.ctx;
    const bx_shard &sh = ctx->shard;
    *err = cudaSuccess;
    // the rest-frame extent over all ranks: order-preserving keys, exact
    int64_t *mm = reinterpret_cast<int64_t *>(ctx->st->mm);
    if (sh.allreduce(mm, 3, BX_OP_MIN, s, sh.user) != 0) return BX_COLLECTIVE;
    if (sh.allreduce(mm + 3, 3, BX_OP_MAX, s, sh.user) != 0) return BX_COLLECTIVE;
    cudaError_t e = launch_box_rule(ctx->st, ctx->n, k.n, ctx->log, ctx->log_cap, true, s);
    if (e == cudaSuccess) e = kick_green(k, s);
    if (e == cudaSuccess && k.binning) e = kick_sort(k, s);
    if (e == cudaSuccess) e = kick_deposit(k, s);
    if (e != cudaSuccess) {
        *err = e;
        return BX_CUDA;
    }
    // the bunch's charge: integer sums, independent of the split
    const int64_t n3 = (int64_t)ctx->n * ctx->n * ctx->n;
    if (sh.allreduce(reinterpret_cast<int64_t *>(ctx->acc_hi), n3, BX_OP_SUM, s, sh.user) != 0 ||
        sh.allreduce(reinterpret_cast<int64_t *>(ctx->acc_lo), n3, BX_OP_SUM, s, sh.user) != 0)
        return BX_COLLECTIVE;
    e = kick_solve_field_push(k, s);
    if (e == cudaSuccess) e = kick_next_deposit(k, s);
    *err = e;
    return e == cudaSuccess ? BX_OK : BX_CUDA;
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

// The nodes of one kick, captured on `cs` into the graph being captured
// there: box rule (sets the conditions), IF(Green's function stale){rebuild},
// IF(re-bin due){sort}, IF(deposit needed){deposit}, solve + field +
// gather/kick/map, IF(next kick){deposit for it}.  The IF bodies are captured
// on `bs`.  With `loop`, the box rule also sets that handle to "a next kick
// follows" (the condition of an enclosing WHILE node).
cudaError_t capture_kick(const KickArgs &k, cudaStream_t cs, cudaStream_t bs,
                         const cudaGraphConditionalHandle *loop) {
    bx_ctx *ctx = k.ctx;
    cudaGraph_t cg = nullptr;
    cudaStreamCaptureStatus status;
    cudaError_t e = cudaStreamGetCaptureInfo(cs, &status, nullptr, &cg, nullptr, nullptr, nullptr);
    cudaGraphConditionalHandle hg = 0, hs = 0, hd = 0, hn = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hg, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hs, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hd, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hn, cg, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = launch_box_rule_graph(ctx->st, ctx->n, ctx->log, ctx->log_cap, hg, hs, hd, hn, cs,
                                  loop ? *loop : 0, loop != nullptr);
    if (e == cudaSuccess) e = capture_if(cs, bs, cg, hg, [&](cudaStream_t b) { return kick_green(k, b); });
    if (e == cudaSuccess && k.binning)
        e = capture_if(cs, bs, cg, hs, [&](cudaStream_t b) { return kick_sort(k, b); });
    if (e == cudaSuccess) e = capture_if(cs, bs, cg, hd, [&](cudaStream_t b) { return kick_deposit(k, b); });
    if (e == cudaSuccess) e = kick_solve_field_push(k, cs);
    if (e == cudaSuccess)
        e = capture_if(cs, bs, cg, hn, [&](cudaStream_t b) { return kick_next_deposit(k, b); });
    return e;
}

cudaError_t ensure_capture_streams(bx_ctx *ctx) {
    cudaError_t e = cudaSuccess;
    if (!ctx->cap_stream) e = cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->body_stream)
        e = cudaStreamCreateWithFlags(&ctx->body_stream, cudaStreamNonBlocking);
    return e;
}

// One kick as an instantiated CUDA graph (bx_track launches it once per kick).
cudaError_t build_kick_graph(const KickArgs &k, cudaGraphExec_t *exec) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = ensure_capture_streams(ctx);
    if (e != cudaSuccess) return e;
    cudaStream_t cs = ctx->cap_stream, bs = ctx->body_stream;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    e = capture_kick(k, cs, bs, nullptr);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();  // clear a sticky capture error, if any
    return e;
}

}  // namespace bt

// ------------------------------------------------------------------ batch

using namespace bt;

struct bx_batch {
    cudaGraphExec_t exec = nullptr;
    int32_t count = 0;
    int64_t launches_per_run = 0;     // kernels one launch runs (all kicks of all problems)
    cudaStream_t s[3] = {nullptr, nullptr, nullptr};
    std::string err;
};

namespace {

thread_local std::string g_batch_err;

int32_t batch_fail(bx_batch *b, int32_t code, const std::string &msg) {
    if (b) b->err = msg;
    g_batch_err = msg;
    return code;
}

// Adds problem `k` to `top` as an independent branch: state reset and the
// first half map, then WHILE(a kick remains){one kick}.
cudaError_t capture_branch(cudaGraph_t top, const KickArgs &k, int nkicks, double q_macro,
                           int sort_interval, cudaStream_t s0, cudaStream_t s1, cudaStream_t s2) {
    bx_ctx *ctx = k.ctx;
    cudaError_t e = cudaStreamBeginCaptureToGraph(s0, top, nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    e = launch_state_reset(ctx->st, nkicks, q_macro, sort_interval, s0, k.bg);
    if (e == cudaSuccess) e = launch_push_maps(k.c, k.n, ctx->maps, 1, s0, ctx->status, ctx->st, k.bg);
    cudaGraphConditionalHandle hw = 0;
    if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&hw, top, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
        cudaStreamCaptureStatus status;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        e = cudaStreamGetCaptureInfo(s0, &status, nullptr, nullptr, &deps, nullptr, &ndeps);
        cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
        p.conditional.handle = hw;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t node;
        if (e == cudaSuccess) e = cudaGraphAddNode(&node, top, deps, nullptr, ndeps, &p);
        if (e == cudaSuccess)
            e = cudaStreamUpdateCaptureDependencies(s0, &node, nullptr, 1,
                                                    cudaStreamSetCaptureDependencies);
        if (e == cudaSuccess) {
            cudaGraph_t body = p.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                cudaError_t eb = capture_kick(k, s1, s2, &hw);
                e = cudaStreamEndCapture(s1, &body);
                if (eb != cudaSuccess) e = eb;
            }
        }
    }
    cudaGraph_t g = top;
    cudaError_t e2 = cudaStreamEndCapture(s0, &g);
    return e != cudaSuccess ? e : e2;
}

}  // namespace

extern "C" {

int32_t bx_batch_create(bx_batch **out, int32_t count, bx_ctx *const *ctxs,
                        bx_beam *const *beams, const bx_lattice *const *lattices, void *stream) {
    if (!out || !ctxs || !beams || !lattices || count <= 0)
        return batch_fail(nullptr, BX_BAD_ARG, "NULL argument or count <= 0");
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    for (int32_t v = 0; v < count; ++v) {
        if (!ctxs[v]) return batch_fail(nullptr, BX_BAD_ARG, "NULL context");
        for (int32_t u = 0; u < v; ++u)
            if (ctxs[u] == ctxs[v])
                return batch_fail(nullptr, BX_BAD_ARG, "a context appears twice in the batch");
        bx_ctx *ctx = ctxs[v];
        if (ctx_sharded(ctx))
            return batch_fail(nullptr, BX_BAD_ARG, "problem " + std::to_string(v) + ": sharded context");
        int32_t rc = check_beam(ctx, beams[v]);
        if (!rc) rc = check_lattice(ctx, lattices[v]);
        if (rc) return batch_fail(nullptr, rc, "problem " + std::to_string(v) + ": " + ctx->err);
    }
    bx_batch *b = new (std::nothrow) bx_batch();
    if (!b) return batch_fail(nullptr, BX_OUT_OF_MEMORY, "host allocation");
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 3 && e == cudaSuccess; ++i)
        e = cudaStreamCreateWithFlags(&b->s[i], cudaStreamNonBlocking);
    cudaGraph_t top = nullptr;
    if (e == cudaSuccess) e = cudaGraphCreate(&top, 0);
    int64_t launches = 0;
    for (int32_t v = 0; v < count && e == cudaSuccess; ++v) {
        bx_ctx *ctx = ctxs[v];
        bx_beam *beam = beams[v];
        const bx_lattice *lat = lattices[v];
        std::vector<int> sel;
        std::vector<double> sds;
        slice_schedule(lat, sel, sds);
        const int64_t K = (int64_t)sel.size();
        if (K == 0 || beam->n == 0 || !lat->space_charge) {
            if (K > 0 && beam->n > 0) {
                // maps only: one kernel over the whole table
                std::vector<MapCoef> tab;
                const Ref r = make_ref(beam);
                build_map_table(lat, sel, sds, 0, K, r, tab);
                if (ensure_maps(ctx, tab.size())) { e = cudaErrorMemoryAllocation; break; }
                e = cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                                    cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
                if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(b->s[0], top, nullptr, nullptr, 0,
                                                                        cudaStreamCaptureModeRelaxed);
                if (e == cudaSuccess) {
                    cudaError_t e1 = launch_push_maps(beam->coord, beam->n, ctx->maps, (int)(K + 1), b->s[0], ctx->status);
                    cudaGraph_t g = top;
                    e = cudaStreamEndCapture(b->s[0], &g);
                    if (e1 != cudaSuccess) e = e1;
                }
                launches += 1;
            }
            continue;
        }
        const Ref r = make_ref(beam);
        std::vector<MapCoef> tab;
        build_map_table(lat, sel, sds, 0, K, r, tab);
        if (ensure_maps(ctx, tab.size()) != BX_OK) { e = cudaErrorMemoryAllocation; break; }
        e = cudaMemcpyAsync(ctx->maps, tab.data(), tab.size() * sizeof(MapCoef),
                            cudaMemcpyHostToDevice, st);
        const bool binning = beam->id != nullptr;
        if (e == cudaSuccess && binning && ensure_sort_scratch(ctx, beam->n) != BX_OK)
            e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess && ctx->shape == 1 && ensure_cells(ctx, beam->n) != BX_OK)
            e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess && binning) e = sort_set_pointers(beam->coord, ctx->scr, ctx->dev_ptrs, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) break;
        const double q_macro = r.sign * std::fabs(beam->bunch_charge_C) / (double)beam->n;
        const KickArgs ka{ctx, beam->coord, beam->id, beam->n, r.bg, binning};
        e = capture_branch(top, ka, (int)K, q_macro, binning ? ctx->sort_interval : 0, b->s[0],
                           b->s[1], b->s[2]);
        launches += 3 + K * 16;
        ctx->green_valid = false;
        ctx->kick = K;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, top, 0);
    if (top) cudaGraphDestroy(top);
    cudaGetLastError();
    if (e != cudaSuccess) {
        std::string m = std::string("bx_batch_create: ") + cudaGetErrorString(e);
        bx_batch_destroy(b);
        return batch_fail(nullptr, e == cudaErrorMemoryAllocation ? BX_OUT_OF_MEMORY : BX_CUDA, m);
    }
    b->count = count;
    b->launches_per_run = launches;
    *out = b;
    return BX_OK;
}

int32_t bx_batch_launch(bx_batch *b, void *stream) {
    if (!b || !b->exec) return batch_fail(b, BX_BAD_ARG, "NULL batch");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return batch_fail(b, BX_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return BX_OK;
}

int32_t bx_batch_destroy(bx_batch *b) {
    if (!b) return BX_OK;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto &s : b->s)
        if (s) cudaStreamDestroy(s);
    delete b;
    return BX_OK;
}

const char *bx_batch_last_error(const bx_batch *b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

}  // extern "C"
