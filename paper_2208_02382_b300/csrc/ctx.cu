// Host helpers of the C ABI: error text, argument checks, the reference
// particle, the linear element maps and the per-call map table, and the lazily
// sized device scratch of the context.
//
// Paper anchors (arXiv:2208.02382): Listing 1 (set_energy_MeV, Drift/Quad
// with nslice, the lattice walked slice by slice) and Model Assumptions
// (linear symplectic maps, split-operator step).
#include <cmath>
#include <cstring>

#include "ctx.cuh"

namespace bt {

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
// Thin dipole edge (K. L. Brown, SLAC-75): edge angle psi = angle, bend
// curvature h = k: px += h tan(psi) x, py -= h tan(psi) y (ds ignored).
// Constant focusing: u'' = -k u in x, u'' = -k2 u in y, t-row as the drift.
void element_map(const bx_element &e, double ds, const Ref &r, Mat m) {
    mat_identity(m);
    if (e.type == BX_DIPEDGE) {
        const double f = e.k * std::tan(e.angle);
        m[1][0] = f;
        m[3][2] = -f;
        return;
    }
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
    if (e.type == BX_QUAD || e.type == BX_CONSTF) {
        double bx[2][2], by[2][2];
        focus_block(ds, e.k, bx);
        focus_block(ds, e.type == BX_QUAD ? -e.k : e.k2, by);
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

bool element_is_thin(const bx_element &e) { return e.type == BX_DIPEDGE || e.type == BX_MULTIPOLE; }

bool lattice_has_multipoles(const bx_lattice *lat) {
    for (int i = 0; i < lat->count; ++i)
        if (lat->elements[i].type == BX_MULTIPOLE) return true;
    return false;
}

// Gauss-Jordan inverse with partial pivoting (the maps are well conditioned).
void mat_inverse(const Mat a, Mat out) {
    double w[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) w[i][j] = j < 6 ? a[i][j] : (j - 6 == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int p = c;
        for (int i = c + 1; i < 6; ++i)
            if (std::fabs(w[i][c]) > std::fabs(w[p][c])) p = i;
        if (p != c)
            for (int j = 0; j < 12; ++j) std::swap(w[p][j], w[c][j]);
        const double d = w[c][c];
        for (int j = 0; j < 12; ++j) w[c][j] /= d;
        for (int i = 0; i < 6; ++i)
            if (i != c) {
                const double f = w[i][c];
                for (int j = 0; j < 12; ++j) w[i][j] -= f * w[c][j];
            }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) out[i][j] = w[i][6 + j];
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
        if (e.type != BX_DRIFT && e.type != BX_QUAD && e.type != BX_SBEND &&
            e.type != BX_DIPEDGE && e.type != BX_CONSTF && e.type != BX_MULTIPOLE)
            return fail(ctx, BX_BAD_ARG, "unknown element type");
        if (!std::isfinite(e.k) || !std::isfinite(e.angle) || !std::isfinite(e.k2))
            return fail(ctx, BX_BAD_ARG, "element k/angle/k2 not finite");
        if (element_is_thin(e)) {
            if (e.nslice != 0) return fail(ctx, BX_BAD_ARG, "thin element needs nslice = 0");
            if (e.type == BX_DIPEDGE && !(std::fabs(e.angle) < 1.5))
                return fail(ctx, BX_BAD_ARG, "edge angle out of range");
            if (e.type == BX_MULTIPOLE && (e.order < 1 || e.order > BX_MULTIPOLE_MAX_ORDER))
                return fail(ctx, BX_BAD_ARG, "multipole order must be in 1..BX_MULTIPOLE_MAX_ORDER");
            continue;
        }
        if (!(e.length > 0.0) || !std::isfinite(e.length))
            return fail(ctx, BX_BAD_ARG, "element length must be > 0");
        if (e.nslice <= 0) return fail(ctx, BX_BAD_ARG, "element nslice must be >= 1");
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

Box explicit_box(const double lo[3], const double hi[3], int n, double betagamma) {
    Box b;
    for (int d = 0; d < 3; ++d) {
        b.lo[d] = lo[d];
        b.hi[d] = hi[d];
        b.h[d] = (hi[d] - lo[d]) / (double)(n - 1);
        b.inv_h[d] = 1.0 / b.h[d];
    }
    box_finish(b, -betagamma);
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

// The cell codes of n particles (deposit -> gather), allocated on the first
// call for a larger n.
int32_t ensure_cells(bx_ctx *ctx, int64_t n) {
    if (n <= ctx->cells_n) return BX_OK;
    cudaDeviceSynchronize();
    if (ctx->cells) cudaFree(ctx->cells);
    ctx->cells = nullptr;
    ctx->cells_n = 0;
    CK(cudaMalloc(&ctx->cells, (size_t)3 * n * sizeof(unsigned long long)), "cell codes");
    CK(cudaMemset(ctx->cells, 0, (size_t)3 * n * sizeof(unsigned long long)), "cell codes");
    ctx->cells_n = n;
    return BX_OK;
}

// Binning scratch for n particles, allocated on the first call for a larger n.
int32_t ensure_sort_scratch(bx_ctx *ctx, int64_t n) {
    const int nb = sort_bins(ctx->n, sort_brick_edge(ctx->n, ctx->bin_edge), ctx->cell_order);
    if (n <= ctx->sort_n && nb == ctx->sort_nb) return BX_OK;
    if (n < ctx->sort_n) n = ctx->sort_n;
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
    const long long len = (long long)nb * sort_chunks(n);
    CK(cudaMalloc(&ctx->keys, n * sizeof(int)), "sort keys");
    CK(cudaMalloc(&ctx->counts, len * sizeof(long long)), "sort counts");
    CK(cudaMalloc(&ctx->offs, len * sizeof(long long)), "sort offsets");
    CK(cudaMalloc(&ctx->sums, (len / 2048 + 2) * sizeof(long long)), "sort sums");
    CK(cudaMalloc(&ctx->id_scr, n * sizeof(long long)), "sort ids");
    for (int k = 0; k < 6; ++k) CK(cudaMalloc(&ctx->scr[k], n * sizeof(double)), "sort arrays");
    ctx->sort_n = n;
    ctx->sort_nb = nb;
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


void slice_schedule(const bx_lattice *lat, std::vector<int> &sel, std::vector<double> &sds) {
    sel.clear();
    sds.clear();
    for (int i = 0; i < lat->count; ++i)
        for (int k = 0; k < (element_is_thin(lat->elements[i]) ? 0 : lat->elements[i].nslice); ++k) {
            sel.push_back(i);
            sds.push_back(lat->elements[i].length / lat->elements[i].nslice);
        }
}

void thin_maps(const bx_lattice *lat, const Ref &r, std::vector<Mat6> &pre, Mat6 &post) {
    pre.clear();
    Mat t;
    mat_identity(t);
    for (int i = 0; i < lat->count; ++i) {
        const bx_element &e = lat->elements[i];
        if (element_is_thin(e)) {
            if (e.type == BX_MULTIPOLE) continue;  // nonlinear: thin_multipoles
            Mat m;
            element_map(e, 0.0, r, m);
            mat_mul(m, t, t);
            continue;
        }
        for (int k = 0; k < e.nslice; ++k) {
            Mat6 p;
            memcpy(p.a, t, sizeof(Mat));
            pre.push_back(p);
            mat_identity(t);
        }
    }
    memcpy(post.a, t, sizeof(Mat));
}

void thin_multipoles(const bx_lattice *lat, std::vector<MpPoly> &pre, MpPoly &post) {
    pre.clear();
    MpPoly q;
    for (int i = 0; i < lat->count; ++i) {
        const bx_element &e = lat->elements[i];
        if (e.type == BX_MULTIPOLE) {
            // kick polynomial term (kn + i ks) z^(m-1) / (m-1)!
            const int j = e.order - 1;
            double f = 1.0;
            for (int a = 2; a <= j; ++a) f *= (double)a;
            q.cr[j] += e.k / f;
            q.ci[j] += e.k2 / f;
            if (j + 1 > q.nc) q.nc = j + 1;
            continue;
        }
        if (element_is_thin(e)) continue;
        for (int k = 0; k < e.nslice; ++k) {
            pre.push_back(q);
            q = MpPoly();
        }
    }
    post = q;
}

// Appends a MAP_SPLIT record for entry `idx` (before, multipoles, after).
static void add_split(std::vector<MapCoef> &tab, std::vector<SplitRec> &recs, size_t idx,
                      const Mat before, const Mat after, const MpPoly &q) {
    SplitRec rec;
    memset(&rec, 0, sizeof(rec));
    rec.before = to_coef(before);
    rec.after = to_coef(after);
    rec.before.kind = rec.after.kind = (double)MAP_GENERAL;
    rec.nc = (double)q.nc;
    for (int j = 0; j < MP_MAX; ++j) {
        rec.cr[j] = q.cr[j];
        rec.ci[j] = q.ci[j];
    }
    tab[idx].kind = (double)MAP_SPLIT;
    tab[idx].aux = (double)recs.size();  // record number for now; offset below
    recs.push_back(rec);
}

void build_map_table(const bx_lattice *lat, const std::vector<int> &sel,
                     const std::vector<double> &sds, int64_t first, int64_t nkicks, const Ref &r,
                     std::vector<MapCoef> &tab) {
    tab.clear();
    tab.reserve(nkicks + 1);
    std::vector<Mat6> pre;
    Mat6 post;
    thin_maps(lat, r, pre, post);
    std::vector<MpPoly> mp;
    MpPoly mp_post;
    thin_multipoles(lat, mp, mp_post);
    std::vector<SplitRec> recs;
    const int64_t total = (int64_t)sel.size();
    Mat eye;
    mat_identity(eye);
    // entry 0: H_first(first) T_pre(first); entry 1 + k: H_first(k+1) T_pre(k+1)
    // H_second(k); the last: T_post (at the end of the lattice) H_second(last).
    // Thin multipoles at a boundary sit between H_second (or nothing, ahead of
    // the first slice) and T_pre H_first (or T_post).
    Mat hk, hn, mm, after;
    element_map(lat->elements[sel[first]], 0.5 * sds[first], r, hk);
    mat_mul(hk, pre[first].a, mm);
    tab.push_back(to_coef(mm));
    if (mp[first].nc) add_split(tab, recs, 0, eye, mm, mp[first]);
    for (int64_t k = first; k < first + nkicks; ++k) {
        if (k + 1 < first + nkicks) {
            element_map(lat->elements[sel[k + 1]], 0.5 * sds[k + 1], r, hn);
            mat_mul(pre[k + 1].a, hk, mm);
            mat_mul(hn, mm, mm);
            tab.push_back(to_coef(mm));
            if (mp[k + 1].nc) {
                mat_mul(hn, pre[k + 1].a, after);
                add_split(tab, recs, tab.size() - 1, hk, after, mp[k + 1]);
            }
            memcpy(hk, hn, sizeof(Mat));
        } else {
            if (k + 1 == total) mat_mul(post.a, hk, mm);
            else memcpy(mm, hk, sizeof(Mat));
            tab.push_back(to_coef(mm));
            if (k + 1 == total && mp_post.nc) add_split(tab, recs, tab.size() - 1, hk, post.a, mp_post);
        }
    }
    // kick factors of kick k and the map class, in table entry 1 + k
    for (int64_t k = 0; k < nkicks; ++k) {
        const double ds = sds[first + k];
        tab[1 + k].kick_t = r.sign * ds / (r.mass_eV * (r.bg * r.bg));
        tab[1 + k].kick_z = -r.sign * ds / (r.mass_eV * r.bg);
    }
    for (auto &m : tab)
        if ((int)m.kind != MAP_SPLIT) m.kind = (double)map_kind(m);
    // the records after the entries; aux = offset from the entry to its record
    const size_t nent = tab.size();
    for (size_t i = 0; i < nent; ++i)
        if ((int)tab[i].kind == MAP_SPLIT) {
            const size_t rec_at = nent + (size_t)tab[i].aux * SPLIT_UNITS;
            tab[i].aux = (double)(rec_at - i);
        }
    tab.resize(nent + recs.size() * SPLIT_UNITS);
    for (size_t q = 0; q < recs.size(); ++q)
        memcpy((void *)&tab[nent + q * SPLIT_UNITS], &recs[q], sizeof(SplitRec));
}

int32_t ensure_moment_scratch(bx_ctx *ctx, int64_t n) {
    const int need = (int)moments_scratch_doubles(moments_blocks(n));
    if (need > ctx->mom_partial_cap) {
        if (ctx->mom_partial) cudaFree(ctx->mom_partial);
        ctx->mom_partial = nullptr;
        CK(cudaMalloc(&ctx->mom_partial, (size_t)need * sizeof(double)), "moments scratch");
        ctx->mom_partial_cap = need;
    }
    return BX_OK;
}

}  // namespace bt
