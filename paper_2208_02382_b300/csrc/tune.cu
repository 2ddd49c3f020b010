// Binning parameters and their autotuner.  The re-binning interval and the
// bin edge of the counting sort (sort.cu) only change the speed of the
// deposit (how compact each block's cells are) against the cost of sorting;
// the autotuner times the candidates on the caller's own problem.  The paper
// has no counterpart (its deposition is ABLASTR's); see bx_autotune_binning
// in include/beamtrack.h.
#include <algorithm>
#include <cmath>
#include <vector>

#include "ctx.cuh"

using namespace bt;

extern "C" {

int32_t bx_set_binning(bx_ctx *ctx, int32_t rebin_interval, int32_t bin_edge,
                       int32_t cell_order) {
    if (!ctx) return set_noctx_error(BX_BAD_ARG, "NULL context");
    if (rebin_interval < -1) return fail(ctx, BX_BAD_ARG, "rebin_interval must be >= -1");
    if (bin_edge != 0 && !sort_brick_edge_valid(ctx->n, bin_edge))
        return fail(ctx, BX_BAD_ARG,
                    "bin_edge must be 0 or a power of two in [2, n/2] giving at most 16^3 bins");
    if (cell_order != 0 && cell_order != 1) return fail(ctx, BX_BAD_ARG, "cell_order must be 0 or 1");
    const int interval = rebin_interval == 0 ? 16 : rebin_interval < 0 ? 0 : rebin_interval;
    if (interval != ctx->sort_interval || bin_edge != ctx->bin_edge ||
        (cell_order != 0) != ctx->cell_order) {
        ctx->sort_interval = interval;
        ctx->bin_edge = bin_edge;
        ctx->cell_order = cell_order != 0;
        // the per-kick graph holds the sort's launch parameters
        if (ctx->kick_exec) {
            cudaDeviceSynchronize();
            cudaGraphExecDestroy(ctx->kick_exec);
            ctx->kick_exec = nullptr;
        }
    }
    return BX_OK;
}

int32_t bx_autotune_binning(bx_ctx *ctx, bx_beam *beam, const bx_lattice *lat, int32_t kicks,
                            int32_t chosen[3], double *ms, int32_t cap, int32_t *count,
                            void *stream) {
    if (!ctx) return set_noctx_error(BX_BAD_ARG, "NULL context");
    int32_t rc = check_beam(ctx, beam);
    if (rc) return rc;
    if ((rc = check_lattice(ctx, lat))) return rc;
    if (!chosen) return fail(ctx, BX_BAD_ARG, "chosen is NULL");
    if (ctx_sharded(ctx)) return fail(ctx, BX_BAD_ARG, "tune a sharded context on one rank first");
    if (!beam->id || beam->n <= 0) return fail(ctx, BX_BAD_ARG, "tuning needs particles with ids");
    if (kicks <= 0) return fail(ctx, BX_BAD_ARG, "kicks must be >= 1");
    cudaStream_t s = (cudaStream_t)stream;
    int64_t total = 0;
    for (int i = 0; i < lat->count; ++i) total += lat->elements[i].nslice;
    const int64_t nk = std::min<int64_t>(kicks, total);
    // candidates: never; every 8, 16, 32 or 64 kicks (intervals no longer
    // than the timed window, so that each candidate's window holds its sorts)
    // with each valid edge of 4, 8, 16, in bin order and in cell order (the
    // cell-order deposit is CIC only)
    struct Cand {
        int iv, be, co;
    };
    std::vector<Cand> cand;
    cand.push_back({-1, 0, 0});
    for (int co = 0; co < (ctx->shape == 1 ? 2 : 1); ++co)
        for (int iv : {8, 16, 32, 64})
            if (iv <= nk)
                for (int be : {4, 8, 16})
                    if (sort_brick_edge_valid(ctx->n, be)) cand.push_back({iv, be, co});
    if (count) *count = (int32_t)cand.size();
    // save the bunch
    const int64_t n = beam->n;
    double *save = nullptr;
    CK(cudaMalloc(&save, (size_t)7 * n * sizeof(double)), "tuning scratch");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        e = cudaMemcpyAsync(save + (size_t)k * n, beam->coord[k], n * sizeof(double),
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(save + (size_t)6 * n, beam->id, n * sizeof(int64_t),
                            cudaMemcpyDeviceToDevice, s);
    auto restore = [&]() {
        cudaError_t r = cudaSuccess;
        for (int k = 0; k < 6 && r == cudaSuccess; ++k)
            r = cudaMemcpyAsync(beam->coord[k], save + (size_t)k * n, n * sizeof(double),
                                cudaMemcpyDeviceToDevice, s);
        if (r == cudaSuccess)
            r = cudaMemcpyAsync(beam->id, save + (size_t)6 * n, n * sizeof(int64_t),
                                cudaMemcpyDeviceToDevice, s);
        return r;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = -1;
    float best_ms = 0.0f;
    const int old_iv = ctx->sort_interval == 0 ? -1 : ctx->sort_interval, old_be = ctx->bin_edge;
    const int old_co = ctx->cell_order ? 1 : 0;
    for (size_t c = 0; c < cand.size() && e == cudaSuccess && rc == BX_OK; ++c) {
        if ((rc = bx_set_binning(ctx, cand[c].iv, cand[c].be, cand[c].co))) break;
        // one untimed pass builds the kick graph for these parameters
        for (int rep = 0; rep < 2 && rc == BX_OK && e == cudaSuccess; ++rep) {
            e = restore();
            if (e != cudaSuccess) break;
            if ((rc = bx_reset(ctx))) break;
            e = cudaEventRecord(e0, s);
            if (e != cudaSuccess) break;
            if ((rc = bx_track(ctx, beam, lat, 0, nk, stream))) break;
            e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float t = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
            if (e == cudaSuccess && rep == 1) {
                if (ms && (int32_t)c < cap) ms[c] = t;
                if (best < 0 || t < best_ms) {
                    best = (int)c;
                    best_ms = t;
                }
            }
        }
    }
    cudaError_t e2 = restore();
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(save);
    if (rc == BX_OK && e == cudaSuccess && best >= 0) {
        rc = bx_set_binning(ctx, cand[best].iv, cand[best].be, cand[best].co);
        chosen[0] = cand[best].iv;
        chosen[1] = cand[best].be;
        chosen[2] = cand[best].co;
    } else {
        bx_set_binning(ctx, old_iv, old_be, old_co);
    }
    if (rc == BX_OK) rc = bx_reset(ctx);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune");
    return BX_OK;
}

}  // extern "C"
