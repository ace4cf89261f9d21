// C-ABI entry points (include/fda_bem.h).  Each call validates its
// arguments, runs on the handle's stream and converts failures into a
// status code plus a message; no exception leaves this file.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <vector>

#include "fda_internal.cuh"

void fda_alloc_densities(fda_handle *h, int want32);
void fda_far_convert_f32(fda_handle *h);

static std::atomic<long long> g_launches{0};

void fda_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void fda_count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long fda_launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void fda_cone_symmetry(int nc, std::vector<int> &rep, std::vector<int> &g);

extern "C" int fda_cone_symmetry_table(int nc, int *rep, int *g)
{
    if (nc < 1 || nc > 64 || !rep || !g) return FDA_ERR_ARG;
    try {
        std::vector<int> r, m;
        fda_cone_symmetry(nc, r, m);
        std::copy(r.begin(), r.end(), rep);
        std::copy(m.begin(), m.end(), g);
    } catch (...) {
        return FDA_ERR_NUMERIC;
    }
    return FDA_OK;
}

extern "C" long long fda_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int fda_debug_sync()
{
    static int v = -1;
    if (v < 0) {
        const char *e = getenv("FDA_DEBUG_SYNC");
        v = (e && e[0] == '1') ? 1 : 0;
    }
    return v;
}

namespace {

template <typename F>
fda_status guarded(fda_handle *h, F &&f)
{
    try {
        f();
        return FDA_OK;
    } catch (const fda_error &e) {
        if (h) h->err = e.msg;
        return e.st;
    } catch (const std::bad_alloc &) {
        if (h) h->err = "host allocation failed";
        return FDA_ERR_OOM;
    } catch (...) {
        if (h) h->err = "unexpected internal error";
        return FDA_ERR_CUDA;
    }
}

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t handle_bytes(const fda_handle *h)
{
    size_t s = 0;
    const dbuf *bufs[] = {&h->perm, &h->iperm, &h->verts9, &h->cent, &h->nrm, &h->area, &h->h2, &h->qpt, &h->qw,
                          &h->keys, &h->box_begin, &h->box_end, &h->box_key, &h->box_coord, &h->box_parent,
                          &h->box_child0, &h->box_child1, &h->box_leaf, &h->box_level, &h->leaf_box,
                          &h->leaf_of_box, &h->il_ptr, &h->il_src, &h->il_op, &h->il_cone, &h->nr_ptr,
                          &h->nr_begin, &h->nr_end, &h->nf_colptr, &h->nf_cols, &h->nf_off, &h->leaf_op_off,
                          &h->op64.St, &h->op64.Tt, &h->op64.near, &h->op32.St, &h->op32.Tt, &h->op32.near,
                          &h->op64.St1, &h->op64.near1, &h->op32.St1, &h->op32.near1,
                          &h->xs, &h->ys, &h->xs32, &h->tt32c, &h->tt_c_off, &h->sai_M, &h->sai_M32, &h->pc_M};
    for (const dbuf *b : bufs) s += b->bytes;
    for (int l = 0; l < FDA_MAX_LEVELS; ++l) {
        s += h->eq_up[l].bytes + h->chk_up[l].bytes + h->rot[l].bytes + h->Uup[l].bytes + h->Vup[l].bytes +
             h->sig[l].bytes;
        s += h->op64.Kt[l].bytes + h->op64.Mt[l].bytes + h->op64.Lt[l].bytes;
        s += h->op32.Kt[l].bytes + h->op32.Mt[l].bytes + h->op32.Lt[l].bytes;
        s += h->q64[l].bytes + h->p64[l].bytes + h->q32[l].bytes + h->p32[l].bytes;
    }
    return s;
}

}  // namespace

extern "C" {

void fda_default_config(fda_config *c)
{
    if (!c) return;
    memset(c, 0, sizeof(*c));
    c->eps = 1e-4;
    c->p_lf = 8;
    c->p_hf = 10;
    c->hf_nr = 5;
    c->hf_na = 300;
    c->leaf_max = 64;
    c->hf_wavelengths = 1.0;
    c->rho_min = 2.2;
    c->precision = FDA_PLAIN_FP64;
    c->mode = FDA_MODE_FDA;
    c->restart = 100;
    c->maxit = 1000;
    c->precond = 0;
    c->alpha_sign = -1.0;
    c->max_rhs = 1;
    c->tensor_cores = 1;
    c->cuda_stream = nullptr;
    c->graphs = 1;
    c->autotune = 1;
    c->autotune_cache = nullptr;
    c->lowrank = 1;
}

fda_status fda_create(const fda_config *cfg, fda_handle **out)
{
    if (!out) return FDA_ERR_ARG;
    *out = nullptr;
    fda_config c;
    if (cfg) c = *cfg; else fda_default_config(&c);
    if (!(c.eps >= 1e-7 && c.eps <= 0.1) || c.leaf_max < 1 || c.leaf_max > 64 || c.p_lf < 3 || c.p_lf > 16 ||
        c.p_hf < 3 || c.p_hf > 16 || c.hf_nr < 1 || c.hf_na < 8 || !(c.hf_wavelengths > 0) || !(c.rho_min >= 2.0) ||
        (c.precision != FDA_PLAIN_FP64 && c.precision != FDA_CHOSEN_FP32) ||
        (c.mode != FDA_MODE_FDA && c.mode != FDA_MODE_DENSE) || c.restart < 1 || c.restart > 255 || c.maxit < 1 || c.precond < 0 ||
        c.precond > 1 || (c.graphs != 0 && c.graphs != 1) || (c.autotune != 0 && c.autotune != 1) || (c.alpha_sign != 1.0 && c.alpha_sign != -1.0) || c.max_rhs < 1 || c.max_rhs > 256 ||
        c.tensor_cores < 0 || c.tensor_cores > 1 || c.lowrank < 0 || c.lowrank > 1)
        return FDA_ERR_ARG;
    fda_handle *h = new (std::nothrow) fda_handle();
    if (!h) return FDA_ERR_OOM;
    h->cfg = c;
    if (c.autotune_cache) h->autotune_cache = c.autotune_cache;
    h->cfg.autotune_cache = nullptr;  // the handle keeps its own copy
    h->stream = (cudaStream_t)c.cuda_stream;
    fda_status st = guarded(h, [&] {
        for (int i = 0; i < 8; ++i) FDA_CUDA(cudaEventCreate(&h->ev[i]));
    });
    if (st != FDA_OK) {
        delete h;
        return st;
    }
    *out = h;
    return FDA_OK;
}

fda_status fda_build_tree(fda_handle *h, const double *verts, int64_t nv, const int32_t *tris, int64_t nt, double k)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 0) {
        h->err = "fda_build_tree called twice on one handle";
        return FDA_ERR_STATE;
    }
    if (!verts || !tris || nv < 3 || nt < 1 || nt > (int64_t)INT32_MAX / 2 || !(k > 0) || !std::isfinite(k) ||
        (h->cfg.mode == FDA_MODE_DENSE && nt > 65535)) {
        h->err = "invalid mesh or wavenumber";
        return FDA_ERR_ARG;
    }
    return guarded(h, [&] {
        double t0 = now_s();
        h->k = k;
        fda_geometry_build(h, verts, nv, tris, nt);
        fda_tree_build(h);
        h->tree_s = now_s() - t0;
        h->state = 1;
    });
}

fda_status fda_precompute_translations(fda_handle *h)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 1) {
        h->err = "fda_precompute_translations needs fda_build_tree first (and runs once)";
        return FDA_ERR_STATE;
    }
    return guarded(h, [&] {
        double t0 = now_s();
        fda_near_build(h);
        h->near_s = now_s() - t0;
        fda_precond_build(h);
        fda_far_precompute(h);
        int want32 = h->cfg.precision == FDA_CHOSEN_FP32;
        if (want32) {
            fda_near_convert_f32(h);
            fda_far_convert_f32(h);
            h->have32 = 1;
        }
        fda_alloc_densities(h, want32);
        if (h->lev_lo >= 0) fda_build_batches(h);
        if (want32 && h->cfg.tensor_cores && h->lev_lo >= 0) {
            fda_pack_tc(h);
            if (h->cfg.autotune) fda_autotune_tc(h);
        }
        h->xs.alloc(sizeof(c64d) * h->N * h->cfg.max_rhs);
        h->ys.alloc(sizeof(c64d) * h->N * h->cfg.max_rhs);
        FDA_CUDA(cudaStreamSynchronize(h->stream));
        h->precompute_s = now_s() - t0;
        h->state = 2;
    });
}

fda_status fda_apply(fda_handle *h, const fda_c128 *x, fda_c128 *y, int nrhs, int64_t ld)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_apply before fda_precompute_translations";
        return FDA_ERR_STATE;
    }
    if (!x || !y || nrhs < 1 || ld < h->N) {
        h->err = "invalid apply arguments";
        return FDA_ERR_ARG;
    }
    return guarded(h, [&] {
        const int mr = std::max(1, h->cfg.max_rhs);
        for (int m0 = 0; m0 < nrhs; m0 += mr) {
            int nm = std::min(mr, nrhs - m0);
            fda_gather_cols(h, reinterpret_cast<const c64d *>(x) + (int64_t)m0 * ld, ld, h->xs.as<c64d>(), nm,
                            h->stream);
            fda_apply_staged(h, h->cfg.precision, nm);
            fda_scatter_cols(h, h->ys.as<c64d>(), reinterpret_cast<c64d *>(y) + (int64_t)m0 * ld, ld, nm,
                             h->stream);
        }
    });
}

fda_status fda_apply_host(fda_handle *h, const fda_c128 *x, fda_c128 *y, int nrhs, int64_t ld)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_apply_host before fda_precompute_translations";
        return FDA_ERR_STATE;
    }
    if (!x || !y || nrhs < 1 || ld < h->N) {
        h->err = "invalid apply arguments";
        return FDA_ERR_ARG;
    }
    return guarded(h, [&] {
        if (!h->io_x.p) {
            h->io_x.alloc(sizeof(c64d) * h->N);
            h->io_y.alloc(sizeof(c64d) * h->N);
        }
        dbuf &dx = h->io_x, &dy = h->io_y;
        for (int m = 0; m < nrhs; ++m) {
            FDA_CUDA(cudaMemcpyAsync(dx.p, x + (int64_t)m * ld, sizeof(c64d) * h->N, cudaMemcpyHostToDevice,
                                     h->stream));
            fda_gather_to_sorted(h, dx.as<c64d>(), h->xs.as<c64d>());
            fda_apply_staged(h, h->cfg.precision, 1);
            fda_scatter_from_sorted(h, h->ys.as<c64d>(), dy.as<c64d>());
            FDA_CUDA(cudaMemcpyAsync(y + (int64_t)m * ld, dy.p, sizeof(c64d) * h->N, cudaMemcpyDeviceToHost,
                                     h->stream));
        }
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    });
}

fda_status fda_rhs_neumann(fda_handle *h, const fda_c128 *q, fda_c128 *b, int nrhs, int64_t ld)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_rhs_neumann before fda_precompute_translations";
        return FDA_ERR_STATE;
    }
    if (!q || !b || nrhs < 1 || ld < h->N) {
        h->err = "invalid fda_rhs_neumann arguments";
        return FDA_ERR_ARG;
    }
    return guarded(h, [&] {
        fda_rhs_layers_prepare(h);
        const int mr = std::max(1, h->cfg.max_rhs);
        for (int m0 = 0; m0 < nrhs; m0 += mr) {
            int nm = std::min(mr, nrhs - m0);
            fda_gather_cols(h, reinterpret_cast<const c64d *>(q) + (int64_t)m0 * ld, ld, h->xs.as<c64d>(), nm,
                            h->stream);
            fda_apply_sorted(h, h->xs.as<c64d>(), h->ys.as<c64d>(), h->cfg.precision, nm, 1);
            fda_scatter_cols(h, h->ys.as<c64d>(), reinterpret_cast<c64d *>(b) + (int64_t)m0 * ld, ld, nm,
                             h->stream);
        }
    });
}

fda_status fda_rhs_plane_wave(fda_handle *h, const double *dirs, int nrhs, fda_c128 *b)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_rhs_plane_wave before fda_build_tree";
        return FDA_ERR_STATE;
    }
    if (!dirs || !b || nrhs < 1) {
        h->err = "invalid right-hand-side arguments";
        return FDA_ERR_ARG;
    }
    for (int m = 0; m < nrhs; ++m) {
        double n2 = dirs[3 * m] * dirs[3 * m] + dirs[3 * m + 1] * dirs[3 * m + 1] + dirs[3 * m + 2] * dirs[3 * m + 2];
        if (!(fabs(n2 - 1.0) < 1e-6)) {
            h->err = "incidence directions must be unit vectors";
            return FDA_ERR_ARG;
        }
    }
    return guarded(h, [&] {
        dbuf dd, bs;
        dd.alloc(sizeof(double) * 3 * nrhs);
        bs.alloc(sizeof(c64d) * h->N * nrhs);
        FDA_CUDA(cudaMemcpyAsync(dd.p, dirs, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, h->stream));
        fda_rhs_sorted(h, dd.as<double>(), nrhs, bs.as<c64d>());
        for (int m = 0; m < nrhs; ++m)
            fda_scatter_from_sorted(h, bs.as<c64d>() + (int64_t)m * h->N, reinterpret_cast<c64d *>(b) + (int64_t)m * h->N);
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    });
}

fda_status fda_rhs_point_source(fda_handle *h, const double *src, int nrhs, fda_c128 *b)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_rhs_point_source before fda_build_tree";
        return FDA_ERR_STATE;
    }
    if (!src || !b || nrhs < 1) {
        h->err = "invalid right-hand-side arguments";
        return FDA_ERR_ARG;
    }
    for (int i = 0; i < 3 * nrhs; ++i)
        if (!std::isfinite(src[i])) {
            h->err = "non-finite source position";
            return FDA_ERR_ARG;
        }
    return guarded(h, [&] {
        dbuf ds;
        ds.alloc(sizeof(double) * 3 * nrhs);
        FDA_CUDA(cudaMemcpyAsync(ds.p, src, sizeof(double) * 3 * nrhs, cudaMemcpyHostToDevice, h->stream));
        fda_rhs_point(h, ds.as<double>(), nrhs, reinterpret_cast<c64d *>(b));
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    });
}

namespace {
fda_status field_call(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *tgt, int64_t ntgt,
                      int far, fda_c128 *out, const char *name)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = std::string(name) + " before fda_precompute_translations";
        return FDA_ERR_STATE;
    }
    if (!u || !tgt || !out || ntgt < 1) {
        h->err = std::string("invalid ") + name + " arguments";
        return FDA_ERR_ARG;
    }
    for (int64_t i = 0; i < ntgt; ++i) {
        const double *t = tgt + 3 * i;
        if (!std::isfinite(t[0]) || !std::isfinite(t[1]) || !std::isfinite(t[2]) ||
            ((far == 1 || far == 2) && !(fabs(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] - 1.0) < 1e-6))) {
            h->err = (far == 1 || far == 2) ? "far-field directions must be unit vectors" : "non-finite field point";
            return FDA_ERR_ARG;
        }
    }
    return guarded(h, [&] {
        dbuf dt;
        dt.alloc(sizeof(double) * 3 * ntgt);
        FDA_CUDA(cudaMemcpyAsync(dt.p, tgt, sizeof(double) * 3 * ntgt, cudaMemcpyHostToDevice, h->stream));
        if (far == 2)
            fda_far_field_upward(h, reinterpret_cast<const c64d *>(u), reinterpret_cast<const c64d *>(q),
                                 dt.as<double>(), (int)ntgt, reinterpret_cast<c64d *>(out));
        else if (far == 3)
            fda_field_fast(h, reinterpret_cast<const c64d *>(u), reinterpret_cast<const c64d *>(q), dt.as<double>(),
                           ntgt, reinterpret_cast<c64d *>(out));
        else
            fda_field(h, reinterpret_cast<const c64d *>(u), reinterpret_cast<const c64d *>(q), dt.as<double>(),
                      ntgt, far, reinterpret_cast<c64d *>(out));
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    });
}
}  // namespace

fda_status fda_far_field(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *dirs, int ndir,
                         fda_c128 *F)
{
    return field_call(h, u, q, dirs, ndir, 1, F, "fda_far_field");
}

fda_status fda_far_field_fast(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *dirs, int ndir,
                              fda_c128 *F)
{
    return field_call(h, u, q, dirs, ndir, 2, F, "fda_far_field_fast");
}

fda_status fda_scattered_field(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *pts, int64_t npts,
                               fda_c128 *out)
{
    return field_call(h, u, q, pts, npts, 0, out, "fda_scattered_field");
}

fda_status fda_scattered_field_fast(fda_handle *h, const fda_c128 *u, const fda_c128 *q, const double *pts,
                                    int64_t npts, fda_c128 *out)
{
    return field_call(h, u, q, pts, npts, 3, out, "fda_scattered_field_fast");
}

fda_status fda_rhs_plane_wave_noalloc(fda_handle *h, const double *dirs, int nrhs, fda_c128 *b)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_rhs_plane_wave_noalloc before fda_build_tree";
        return FDA_ERR_STATE;
    }
    if (!dirs || !b || nrhs < 1) {
        h->err = "invalid right-hand-side arguments";
        return FDA_ERR_ARG;
    }
    if (nrhs > FDA_NOALLOC_MAX_DIRS) {
        h->err = "fda_rhs_plane_wave_noalloc takes at most FDA_NOALLOC_MAX_DIRS (256) directions per call";
        return FDA_ERR_ARG;
    }
    for (int m = 0; m < nrhs; ++m) {
        double n2 = dirs[3 * m] * dirs[3 * m] + dirs[3 * m + 1] * dirs[3 * m + 1] + dirs[3 * m + 2] * dirs[3 * m + 2];
        if (!(fabs(n2 - 1.0) < 1e-6)) {
            h->err = "incidence directions must be unit vectors";
            return FDA_ERR_ARG;
        }
    }
    return guarded(h, [&] { fda_rhs_noalloc(h, dirs, nrhs, reinterpret_cast<c64d *>(b)); });
}

fda_status fda_solve(fda_handle *h, const fda_c128 *b, fda_c128 *x, int nrhs, double tol, fda_info *info)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_solve before fda_precompute_translations";
        return FDA_ERR_STATE;
    }
    if (!b || !x || nrhs < 1 || !(tol > 0) || !(tol < 1)) {
        h->err = "invalid solve arguments";
        return FDA_ERR_ARG;
    }
    fda_status last = FDA_OK;
    fda_status st = guarded(h, [&] {
        for (int m = 0; m < nrhs; ++m) {
            fda_status s = fda_solve_impl(h, reinterpret_cast<const c64d *>(b) + (int64_t)m * h->N,
                                          reinterpret_cast<c64d *>(x) + (int64_t)m * h->N, tol, info);
            if (s != FDA_OK) last = s;
        }
        if (fda_tc_error(h)) fda_fail(FDA_ERR_TIMEOUT, "a tensor-core translation gave up waiting on its copies");
    });
    return st != FDA_OK ? st : last;
}

fda_status fda_get_stats(fda_handle *h, fda_stats *out)
{
    if (!h || !out) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_get_stats before fda_build_tree";
        return FDA_ERR_STATE;
    }
    memset(out, 0, sizeof(*out));
    return guarded(h, [&] {
        out->n_elements = h->N;
        out->n_boxes = h->nbox_total;
        out->n_leaves = h->nleaf;
        out->n_levels = h->nlev;
        out->nnz_near = h->nnz_near;
        out->n_m2l = h->n_il_total;
        int64_t ops = 0;
        for (int l = 0; l < 32; ++l) {
            out->level_regime[l] = l < h->nlev ? h->lev[l].hf : -1;
            out->level_rank[l] = l < h->nlev ? h->lev[l].T : 0;
            out->level_boxes[l] = l < h->nlev ? h->lev[l].nbox : 0;
            out->level_cones[l] = l < h->nlev ? h->lev[l].ncones : 0;
            out->level_m2l_pairs[l] = l < h->nlev ? h->lev[l].n_il : 0;
            out->level_m2l_ops[l] = l < h->nlev ? h->lev[l].n_ops : 0;
            if (l < h->nlev) ops += h->lev[l].n_ops;
        }
        out->n_m2l_ops = ops;
        out->graph_replays = h->graph_replays;
        out->graph_fallback = h->graphs_broken;
        out->autotune_cached = h->autotune_cached;
        out->autotune_timed = h->autotune_timed;
        for (int l = 0; l < h->nlev && l < 32; ++l) {
            const level_info &L = h->lev[l];
            const std::vector<int> &rk = h->op_rank[l];
            const std::vector<int> &bk = h->op_bucket[l];
            double rsum = 0.0;
            int rcnt = 0, rmax = 0, nlr = 0;
            for (size_t o = 0; o < rk.size(); ++o) {
                if (rk[o] >= 0) {
                    rsum += rk[o];
                    ++rcnt;
                }
                if (o < bk.size() && bk[o] >= 0) {
                    ++nlr;
                    rmax = std::max(rmax, rk[o]);
                }
            }
            out->level_lr_ops[l] = nlr;
            out->level_lr_rank_max[l] = rmax;
            out->level_lr_rank_mean[l] = rcnt ? (float)(rsum / rcnt) : 0.0f;
            int64_t lrp = 0;
            for (const lr_bucket &B : h->lr[l]) lrp += B.npairs;
            out->level_lr_pairs[l] = lrp;
            out->level_lr_tc[l] = h->lr_tc[l] | (h->lr_tc_many[l] << 1);
            {
                auto code = [](const tr_batch &B) { return B.nc_tuned ? B.nc_tuned * 100 + B.r_tuned * 10 + B.st_tuned : 0; };
                const tr_batch &F = !h->lr[l].empty() && !h->lr_tc[l] ? h->b_m2l_all[l] : h->b_m2l[l];
                out->level_tc_shape[l][0] = l + 1 < h->nlev ? code(h->b_m2m[l]) : 0;
                out->level_tc_shape[l][1] = code(F);
                out->level_tc_shape[l][2] = l + 1 < h->nlev ? code(h->b_l2l[l]) : 0;
            }
            // algorithmic work of the level's M2L pass, one right-hand side, in
            // the form the current precision applies
            const double T = L.T;
            if (T == 0 || L.n_il == 0) continue;
            const bool tcpath = h->cfg.precision == FDA_CHOSEN_FP32 && h->have_tc && h->cfg.tensor_cores;
            const bool lrform = !h->lr[l].empty() && (!tcpath || h->lr_tc[l]);
            const tr_batch &F = (lrform || h->lr[l].empty()) ? h->b_m2l[l] : h->b_m2l_all[l];
            double fl = 0.0, by = 0.0;
            for (int o = 0; o + 1 < (int)F.op_start.size(); ++o) {
                const int np = F.op_start[o + 1] - F.op_start[o];
                if (np == 0) continue;
                fl += 8.0 * T * T * np;
                by += 8.0 * T * T;
            }
            if (lrform)
                for (const lr_bucket &B : h->lr[l]) {
                    for (size_t i = 0; i < B.ops.size(); ++i) {
                        const double r = rk[B.ops[i]];
                        const int np = B.b1.op_start[i + 1] - B.b1.op_start[i];
                        fl += 8.0 * 2.0 * r * T * np;
                        by += 8.0 * 2.0 * r * T + 2.0 * 8.0 * r * np;
                    }
                }
            by += 3.0 * 8.0 * L.nbox * L.ncones * T;
            out->level_m2l_flops[l] = fl;
            out->level_m2l_bytes[l] = by;
        }
        int rb = h->cfg.precision == FDA_CHOSEN_FP32 ? 8 : 16;
        out->bytes_near = h->nnz_near * rb;
        // far-field flop count (real flops, 8 per complex multiply-add)
        if (h->state == 2 && h->lev_lo >= 0) {
            std::vector<int32_t> leaf(h->nbox_total), c0(h->nbox_total), c1(h->nbox_total), beg(h->nbox_total),
                end(h->nbox_total);
            std::vector<int64_t> ilp(h->nbox_total + 1);
            FDA_CUDA(cudaMemcpy(leaf.data(), h->box_leaf.p, 4 * leaf.size(), cudaMemcpyDeviceToHost));
            FDA_CUDA(cudaMemcpy(c0.data(), h->box_child0.p, 4 * c0.size(), cudaMemcpyDeviceToHost));
            FDA_CUDA(cudaMemcpy(c1.data(), h->box_child1.p, 4 * c1.size(), cudaMemcpyDeviceToHost));
            FDA_CUDA(cudaMemcpy(beg.data(), h->box_begin.p, 4 * beg.size(), cudaMemcpyDeviceToHost));
            FDA_CUDA(cudaMemcpy(end.data(), h->box_end.p, 4 * end.size(), cudaMemcpyDeviceToHost));
            FDA_CUDA(cudaMemcpy(ilp.data(), h->il_ptr.p, 8 * ilp.size(), cudaMemcpyDeviceToHost));
            double fl = 0, by = 0;
            int cb = h->cfg.precision == FDA_CHOSEN_FP32 ? 8 : 16;
            for (int l = h->lev_lo; l < h->nlev; ++l) {
                const level_info &L = h->lev[l];
                double T = L.T;
                for (int b = L.box0; b < L.box0 + L.nbox; ++b) {
                    double nB = end[b] - beg[b];
                    if (leaf[b]) {
                        fl += 2 * 8.0 * T * nB;  // S2M + L2T
                        by += 2.0 * cb * 64 * T;
                    } else if (l + 1 < h->nlev) {
                        fl += 8.0 * T * h->lev[l + 1].T * (c1[b] - c0[b]) * L.ncones;  // M2M
                    }
                    if (l > h->lev_lo) fl += 8.0 * T * h->lev[l - 1].T * h->lev[l - 1].ncones;  // L2L (upper bound)
                    fl += 8.0 * T * T * (double)(ilp[b + 1] - ilp[b]);                         // M2L
                }
                by += (double)cb * L.n_ops * T * T;                 // distinct K~
                by += 2.0 * 2.0 * cb * L.nbox * L.ncones * T;       // q~ and p~ written and read
            }
            out->flops_far = (int64_t)fl;
            out->bytes_far = (int64_t)by;
        }
        out->device_bytes = (int64_t)handle_bytes(h);
        for (int l = 0; l < FDA_MAX_LEVELS; ++l)
            out->device_bytes += (int64_t)(h->tc_m2l[l].A.bytes + h->tc_m2m[l].A.bytes + h->tc_l2l[l].A.bytes +
                                           h->qs[l].bytes + h->ps[l].bytes);
        if (fda_tc_error(h)) fda_fail(FDA_ERR_TIMEOUT, "a tensor-core translation gave up waiting on its copies");
        out->tree_s = h->tree_s;
        out->near_s = h->near_s;
        out->precompute_s = h->precompute_s;
    });
}

fda_status fda_set_precision(fda_handle *h, int precision)
{
    if (!h) return FDA_ERR_ARG;
    if (precision != FDA_PLAIN_FP64 && precision != FDA_CHOSEN_FP32) {
        h->err = "unknown precision";
        return FDA_ERR_ARG;
    }
    if (precision == FDA_CHOSEN_FP32 && !h->have32) {
        h->err = "FP32 operators were not built (create the handle with precision = FDA_CHOSEN_FP32)";
        return FDA_ERR_STATE;
    }
    h->cfg.precision = precision;
    return FDA_OK;
}

fda_status fda_set_tensor_cores(fda_handle *h, int on)
{
    if (!h) return FDA_ERR_ARG;
    if (on != 0 && on != 1) {
        h->err = "tensor_cores must be 0 or 1";
        return FDA_ERR_ARG;
    }
    if (on && !h->have_tc) {
        h->err = "tensor-core operators were not built (chosen precision with tensor_cores = 1)";
        return FDA_ERR_STATE;
    }
    h->cfg.tensor_cores = on;
    return FDA_OK;
}

fda_status fda_tree_sizes(fda_handle *h, int64_t *sizes)
{
    if (!h || !sizes) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_tree_sizes before fda_build_tree";
        return FDA_ERR_STATE;
    }
    sizes[0] = h->nbox_total;
    sizes[1] = h->nleaf;
    sizes[2] = h->n_il_total;
    sizes[3] = h->ncols_total;
    return FDA_OK;
}

fda_status fda_get_tree(fda_handle *h, int32_t *box_level, int32_t *box_coord, int32_t *box_leaf,
                        int32_t *box_parent, int32_t *box_begin, int32_t *box_end, int32_t *perm, int64_t *il_ptr,
                        int32_t *il_src, int32_t *leaf_box, int64_t *nf_colptr, int32_t *nf_cols)
{
    if (!h) return FDA_ERR_ARG;
    if (h->state < 1) {
        h->err = "fda_get_tree before fda_build_tree";
        return FDA_ERR_STATE;
    }
    return guarded(h, [&] {
        const size_t nb = (size_t)h->nbox_total, nl = (size_t)h->nleaf;
        auto cp = [&](void *dst, const dbuf &src, size_t bytes) {
            if (dst && bytes) FDA_CUDA(cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToHost, h->stream));
        };
        cp(box_level, h->box_level, 4 * nb);
        cp(box_coord, h->box_coord, 12 * nb);
        cp(box_leaf, h->box_leaf, 4 * nb);
        cp(box_parent, h->box_parent, 4 * nb);
        cp(box_begin, h->box_begin, 4 * nb);
        cp(box_end, h->box_end, 4 * nb);
        cp(perm, h->perm, 4 * (size_t)h->N);
        cp(il_ptr, h->il_ptr, 8 * (nb + 1));
        cp(il_src, h->il_src, 4 * (size_t)h->n_il_total);
        cp(leaf_box, h->leaf_box, 4 * nl);
        cp(nf_colptr, h->nf_colptr, 8 * (nl + 1));
        cp(nf_cols, h->nf_cols, 4 * (size_t)h->ncols_total);
        FDA_CUDA(cudaStreamSynchronize(h->stream));
    });
}

fda_status fda_set_tc_tiles(fda_handle *h, int columns, int row_tiles, int stages)
{
    if (!h) return FDA_ERR_ARG;
    static const int shapes[15][3] = {{32, 1, 2}, {32, 1, 4}, {64, 1, 2}, {64, 1, 4}, {32, 2, 4},
                                      {64, 2, 3}, {64, 2, 4}, {32, 3, 3}, {32, 3, 4}, {128, 1, 3},
                                      {128, 1, 4}, {128, 2, 2}, {128, 2, 3}, {64, 3, 3}, {64, 4, 2}};
    bool known = columns == 0 && row_tiles == 0 && stages == 0;
    for (const auto &c : shapes) known |= c[0] == columns && c[1] == row_tiles && c[2] == stages;
    if (!known) {
        h->err = "unknown tensor-core tile shape (columns, row tiles, stages)";
        return FDA_ERR_ARG;
    }
    return guarded(h, [&] {
        // captured graphs hold the previous shape's launches
        fda_graphs_release(h);
        h->tc_force[0] = columns;
        h->tc_force[1] = row_tiles;
        h->tc_force[2] = stages;
    });
}

fda_status fda_set_precond(fda_handle *h, int precond)
{
    if (!h) return FDA_ERR_ARG;
    if (precond < 0 || precond > 2) {
        h->err = "unknown preconditioner";
        return FDA_ERR_ARG;
    }
    if (precond == 1 && !h->pc_M.p) {
        h->err = "block-diagonal preconditioner was not built (create the handle with precond = 1)";
        return FDA_ERR_STATE;
    }
    if (precond == 2 && !h->sai_M.p && !h->sai_M32.p) {
        h->err = "learned preconditioner not set (call fda_sai_set or fda_sai_set_pattern first)";
        return FDA_ERR_STATE;
    }
    h->cfg.precond = precond;
    return FDA_OK;
}

fda_status fda_set_timing(fda_handle *h, int enable)
{
    if (!h) return FDA_ERR_ARG;
    h->timing = enable ? 1 : 0;
    return FDA_OK;
}

fda_status fda_get_pass_times(fda_handle *h, float out[6])
{
    if (!h || !out) return FDA_ERR_ARG;
    if (!h->timing) {
        h->err = "pass timing is off (fda_set_timing)";
        return FDA_ERR_STATE;
    }
    for (int i = 0; i < 6; ++i) out[i] = h->pass_ms[i];
    return FDA_OK;
}

const char *fda_last_error(const fda_handle *h)
{
    if (!h) return "null handle";
    return h->err.c_str();
}

void fda_destroy(fda_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream); else cudaDeviceSynchronize();
    for (int i = 0; i < 8; ++i)
        if (h->ev[i]) cudaEventDestroy(h->ev[i]);
    fda_graphs_release(h);
    delete h;
}

}  // extern "C"

// ---- learned SAI preconditioner

extern "C" int fda_sai_num_params(void) { return fda_sai_nparams(); }

extern "C" size_t fda_struct_size(int which)
{
    switch (which) {
    case 0: return sizeof(fda_config);
    case 1: return sizeof(fda_info);
    case 2: return sizeof(fda_stats);
    case 3: return sizeof(fda_sai_config);
    case 4: return sizeof(fda_sai_report);
    case 5: return sizeof(fda_batch_stats);
    default: return 0;
    }
}

extern "C" fda_status fda_sai_default_config(fda_sai_config *c)
{
    if (!c) return FDA_ERR_ARG;
    c->epochs = 400;
    c->lr = 3e-3;
    c->seed = 1;
    c->pattern = 0;
    c->sample_leaves = 256;
    return FDA_OK;
}

extern "C" fda_status fda_sai_init_weights(unsigned long long seed, float *weights)
{
    if (!weights) return FDA_ERR_ARG;
    fda_sai_init(seed, weights);
    return FDA_OK;
}

extern "C" fda_status fda_sai_train(fda_handle *const *handles, int nhandles, const fda_sai_config *cfg,
                                    float *weights, fda_sai_report *rep)
{
    if (!handles || nhandles < 1 || !cfg || !weights || cfg->epochs < 0 || !(cfg->lr > 0) ||
        (cfg->pattern != 0 && cfg->pattern != 1) || (cfg->pattern == 1 && cfg->sample_leaves < 1))
        return FDA_ERR_ARG;
    for (int q = 0; q < nhandles; ++q) {
        if (!handles[q]) return FDA_ERR_ARG;
        if (handles[q]->state != 2) {
            handles[q]->err = "fda_sai_train needs fda_precompute_translations first";
            return FDA_ERR_STATE;
        }
    }
    return guarded(handles[0], [&] {
        double l0 = 0, l1 = 0, ts = 0;
        if (cfg->pattern == 1)
            fda_sai_train_near_impl(handles, nhandles, cfg->epochs, cfg->lr, cfg->sample_leaves, cfg->seed, weights,
                                    &l0, &l1, &ts);
        else
            fda_sai_train_impl(handles, nhandles, cfg->epochs, cfg->lr, weights, &l0, &l1, &ts);
        if (rep) {
            rep->loss_init = l0;
            rep->loss_final = l1;
            rep->train_s = ts;
        }
    });
}

extern "C" fda_status fda_sai_set(fda_handle *h, const float *weights, double *loss)
{
    if (!h || !weights) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_sai_set needs fda_precompute_translations first";
        return FDA_ERR_STATE;
    }
    return guarded(h, [&] {
        double l = fda_sai_set_impl(h, weights);
        if (loss) *loss = l;
    });
}

extern "C" fda_status fda_sai_set_pattern(fda_handle *h, const float *weights, int pattern, double *loss)
{
    if (!h || !weights || (pattern != 0 && pattern != 1)) return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_sai_set_pattern needs fda_precompute_translations first";
        return FDA_ERR_STATE;
    }
    return guarded(h, [&] {
        const double l = pattern == 1 ? fda_sai_set_near_impl(h, weights, loss != nullptr)
                                      : fda_sai_set_impl(h, weights);
        if (loss) *loss = l;
    });
}

extern "C" fda_status fda_sai_loss_grad_near(fda_handle *h, const double *weights, int nleaves,
                                             const int32_t *leaves, int precision, double *loss, double *grad)
{
    if (!h || !weights || nleaves < 1 || !leaves || !loss || !grad ||
        (precision != FDA_PLAIN_FP64 && precision != FDA_CHOSEN_FP32))
        return FDA_ERR_ARG;
    if (h->state != 2) {
        h->err = "fda_sai_loss_grad_near needs fda_precompute_translations first";
        return FDA_ERR_STATE;
    }
    for (int b = 0; b < nleaves; ++b)
        if (leaves[b] < 0 || leaves[b] >= h->nleaf) {
            h->err = "leaf index out of range";
            return FDA_ERR_ARG;
        }
    return guarded(h, [&] {
        fda_sai_loss_grad_near_impl(h, weights, nleaves, leaves, precision == FDA_CHOSEN_FP32, loss, grad);
    });
}

extern "C" fda_status fda_sai_loss_grad(int64_t n, const double *centroids, const double *normals,
                                        const double *areas, double k, int nblocks, const int64_t *block_ptr,
                                        const int32_t *block_elems, const fda_c128 *blocks, const double *weights,
                                        int precision, double *loss, double *grad)
{
    if (n < 1 || !centroids || !normals || !areas || !(k > 0) || nblocks < 1 || !block_ptr || !block_elems ||
        !blocks || !weights || !loss || !grad || block_ptr[0] != 0 ||
        (precision != FDA_PLAIN_FP64 && precision != FDA_CHOSEN_FP32))
        return FDA_ERR_ARG;
    for (int b = 0; b < nblocks; ++b)
        if (block_ptr[b + 1] <= block_ptr[b]) return FDA_ERR_ARG;
    try {
        fda_sai_loss_grad_impl(n, centroids, normals, areas, k, nblocks, block_ptr, block_elems,
                               reinterpret_cast<const c64d *>(blocks), weights, precision == FDA_CHOSEN_FP32, loss,
                               grad);
    } catch (const fda_error &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        return FDA_ERR_OOM;
    } catch (...) {
        return FDA_ERR_CUDA;
    }
    return FDA_OK;
}
