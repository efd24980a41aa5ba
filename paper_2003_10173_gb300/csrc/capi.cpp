// C ABI of the library: argument validation, error translation, handle life cycle.
#include <cmath>
#include <cstring>
#include <new>

#include "handle.h"

namespace h2 {
h2_tree_s* make_tree(const double* coords, int64_t N, int dim, int leaf, int adm, double eta);
int build_handle(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o,
                 h2_handle_s* h);
int build_batched(int count, const h2_op_fn* ops, void* const* ctxs, const h2_tree_t* trees, double tol,
                  const h2_build_opts& o, h2_handle_t* outs);
int update_handle(h2_handle_s* A, const double* B, int64_t ldb, int r, const double* M, double tol,
                  const h2_build_opts& o, h2_handle_s* h);
void colored_plan_counts(const h2_tree_s* tree, int q, int* out);
h2_batch_s* batch_create(int count, const h2_handle_t* hs);
void batch_matvec(h2_batch_s* b, const void* const* X, const int64_t* ldx, void* const* Y, const int64_t* ldy,
                  int64_t nrhs, int mode, cudaStream_t s);
int batch_tuned(h2_batch_s* b, int64_t nrhs, int mode);
h2_rankmodel_s* rm_create(uint64_t seed, int bf16);
void rm_free(h2_rankmodel_s* m);
void rm_get(h2_rankmodel_s* m, float* p, float* am, float* av, int64_t* step);
void rm_set(h2_rankmodel_s* m, const float* p, const float* am, const float* av, int64_t step);
void rm_features(const h2_tree_s* t, double kT, double dens, double tol, double* out);
void rm_train(h2_rankmodel_s* m, const float* X, const float* T, int64_t n, const int32_t* idx, int steps, int batch,
              float lr, float* loss_out, cudaStream_t s);
void rm_loss_grad(h2_rankmodel_s* m, const float* X, const float* T, int64_t n, float* loss, float* grad);
void rm_predict(h2_rankmodel_s* m, const float* X, int64_t n, float* Y, cudaStream_t s);
void rm_q_levels(h2_rankmodel_s* m, const h2_tree_s* t, double kT, double dens, double tol, int pad, int q_max,
                 int32_t* q, float* y_host);
void rm_save(h2_rankmodel_s* m, const char* path);
void invert(h2_handle_s* A, const h2_invert_opts& io, const h2_build_opts& bo, h2_handle_s** Xout, h2_invert_stats* st);
h2_rankmodel_s* rm_load(const char* path);

// Device permutation, matvec plan, reduced-precision copies and statistics of a built handle.
void finish_handle(h2_handle_s* h, const h2_build_opts& o, cudaStream_t s) {
    std::vector<int32_t> perm(h->N);
    for (int64_t i = 0; i < h->N; ++i) perm[i] = (int32_t)h->tree->perm[i];
    h->d_perm.reserve(h->N);
    H2_CUDA(cudaMemcpyAsync(h->d_perm.p, perm.data(), h->N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    H2_CUDA(cudaStreamSynchronize(s));
    build_plan(h, s);
    make_copies(h, o.keep_fp32, o.keep_bf16, s);
    H2_CUDA(cudaStreamSynchronize(s));
    h->stats.far_lower = 0;
    for (auto& f : h->far_lower) h->stats.far_lower += (int64_t)f.size();
    h->stats.near_lower = (int64_t)h->near_lower.size();
    h->stats.entries_D = h->entries_D;
    h->stats.entries_S = h->entries_S;
    h->stats.entries_U = h->entries_U;
    h->stats.entries_E = h->entries_E;
}
}  // namespace h2

namespace {

thread_local std::string g_last_error;

template <class F>
int guard(F&& f) {
    try {
        g_last_error.clear();
        return f();
    } catch (const h2::Error& e) {
        g_last_error = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return H2_ERR_OOM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return H2_ERR_INVALID_ARG;
    } catch (...) {
        g_last_error = "unknown error";
        return H2_ERR_INVALID_ARG;
    }
}

void require(bool ok, const char* msg) {
    if (!ok) h2::fail(H2_ERR_INVALID_ARG, msg);
}

h2_build_opts checked_opts(double tol, const h2_build_opts* opts) {
    require(tol > 0.0 && std::isfinite(tol), "h2_build: tol must be positive");
    h2_build_opts o;
    h2_build_opts_default(&o);
    if (opts) o = *opts;
    require(o.kmax >= 1, "h2_build: kmax must be >= 1");
    require(o.q0 >= 1 && o.q_max >= 1, "h2_build: probe counts must be >= 1");
    require(o.b_inc >= 1 && o.b_inc <= 16, "h2_build: b_inc must be in 1..16");
    require(o.q_test >= 1 && o.q_test <= 16, "h2_build: q_test must be in 1..16");
    require(o.q_level_stride >= 0, "h2_build: q_level_stride must be >= 0");
    require(o.global_rank >= 0, "h2_build: global_rank must be >= 0");
    require(o.batch_workers >= 0 && o.batch_workers <= 256, "h2_build: batch_workers must be in 0..256");
    require(o.sampling == H2_SAMPLING_WEAK || o.sampling == H2_SAMPLING_COLORED, "h2_build: unknown sampling");
    require(o.certified == 0 || o.certified == 1, "h2_build: certified must be 0 or 1");
    require(o.sampling != H2_SAMPLING_COLORED || (o.q0 <= 16 && o.global_rank == 0),
            "h2_build: coloured sampling needs q0 <= 16 and global_rank 0");
    require(o.norm_maxit >= 1 && o.norm_rtol > 0.0, "h2_build: bad power-iteration settings");
    require(!(o.norm_est < 0.0) && std::isfinite(o.norm_est), "h2_build: bad norm_est");
    return o;
}

}  // namespace

extern "C" {

int h2_build_opts_default(h2_build_opts* o) {
    if (!o) return H2_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->kmax = 32;
    o->q0 = 32;
    o->b_inc = 16;
    o->q_max = 256;
    o->adaptive = 1;
    o->seed = 7;
    o->norm_est = 0.0;
    o->norm_maxit = 50;
    o->norm_rtol = 1e-3;
    o->keep_fp32 = 0;
    o->keep_bf16 = 0;
    o->stream = nullptr;
    o->q_level = nullptr;
    o->q_level_stride = 0;
    o->q_test = 8;
    o->global_rank = 0;
    return H2_OK;
}

int h2_tree_create(const double* coords_host, int64_t n, int dim, int leaf_size, int adm, double eta,
                   h2_tree_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_tree_create: out is NULL");
        *out = nullptr;
        *out = h2::make_tree(coords_host, n, dim, leaf_size, adm, eta);
        return H2_OK;
    });
}

void h2_tree_free(h2_tree_t tree) { delete tree; }

int h2_tree_info(h2_tree_t t, int* levels, int64_t* n, int64_t* n_far, int64_t* n_near) {
    return guard([&] {
        require(t != nullptr, "h2_tree_info: NULL tree");
        if (levels) *levels = t->L;
        if (n) *n = t->N;
        if (n_far) {
            int64_t c = 0;
            for (auto& f : t->far) c += (int64_t)f.size();
            *n_far = c;
        }
        if (n_near) *n_near = (int64_t)t->near.size();
        return H2_OK;
    });
}

int h2_tree_perm(h2_tree_t t, int64_t* perm_host) {
    return guard([&] {
        require(t && perm_host, "h2_tree_perm: NULL argument");
        std::memcpy(perm_host, t->perm.data(), t->perm.size() * sizeof(int64_t));
        return H2_OK;
    });
}

int h2_tree_boxes(h2_tree_t t, int level, int64_t* starts, int64_t* sizes) {
    return guard([&] {
        require(t && starts && sizes, "h2_tree_boxes: NULL argument");
        require(level >= 0 && level <= t->L, "h2_tree_boxes: level out of range");
        std::memcpy(starts, t->start[level].data(), t->start[level].size() * sizeof(int64_t));
        std::memcpy(sizes, t->size[level].data(), t->size[level].size() * sizeof(int64_t));
        return H2_OK;
    });
}

int h2_tree_far(h2_tree_t t, int level, int64_t* count, int32_t* pairs) {
    return guard([&] {
        require(t && count, "h2_tree_far: NULL argument");
        require(level >= 0 && level <= t->L, "h2_tree_far: level out of range");
        const auto& f = t->far[level];
        *count = (int64_t)f.size();
        if (pairs)
            for (size_t i = 0; i < f.size(); ++i) {
                pairs[2 * i] = f[i].first;
                pairs[2 * i + 1] = f[i].second;
            }
        return H2_OK;
    });
}

int h2_tree_near(h2_tree_t t, int64_t* count, int32_t* pairs) {
    return guard([&] {
        require(t && count, "h2_tree_near: NULL argument");
        *count = (int64_t)t->near.size();
        if (pairs)
            for (size_t i = 0; i < t->near.size(); ++i) {
                pairs[2 * i] = t->near[i].first;
                pairs[2 * i + 1] = t->near[i].second;
            }
        return H2_OK;
    });
}

int h2_build(h2_op_fn op, void* ctx, h2_tree_t tree, double tol, const h2_build_opts* opts, h2_handle_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_build: out is NULL");
        *out = nullptr;
        require(op != nullptr && tree != nullptr, "h2_build: NULL operator or tree");
        h2_build_opts o = checked_opts(tol, opts);
        auto* h = new h2_handle_s();
        try {
            const cudaStream_t s = (cudaStream_t)o.stream;
            h2::AllocScope scope(s);
            const int st = h2::build_handle(op, ctx, tree, tol, o, h);
            h2::finish_handle(h, o, s);
            *out = h;
            return st;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int h2_build_batched(int count, const h2_op_fn* ops, void* const* ctxs, const h2_tree_t* trees, double tol,
                     const h2_build_opts* opts, h2_handle_t* outs) {
    return guard([&] {
        require(count >= 0 && (count == 0 || (ops && trees && outs)), "h2_build_batched: NULL arrays");
        for (int i = 0; i < count; ++i) require(ops[i] && trees[i], "h2_build_batched: NULL operator or tree");
        h2_build_opts o = checked_opts(tol, opts);
        if (count == 0) return (int)H2_OK;
        return h2::build_batched(count, ops, ctxs, trees, tol, o, outs);
    });
}

int h2_batch_create(int count, const h2_handle_t* hs, h2_batch_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_batch_create: out is NULL");
        *out = nullptr;
        require(count >= 1 && hs, "h2_batch_create: need at least one handle");
        for (int i = 0; i < count; ++i) require(hs[i] != nullptr, "h2_batch_create: NULL handle");
        *out = h2::batch_create(count, hs);
        return H2_OK;
    });
}

int h2_batch_matvec(h2_batch_t b, const void* const* X, const int64_t* ldx, void* const* Y, const int64_t* ldy,
                    int64_t nrhs, int mode, h2_stream_t stream) {
    return guard([&] {
        require(b != nullptr, "h2_batch_matvec: NULL batch");
        require(nrhs >= 0 && nrhs <= 2000000, "h2_batch_matvec: nrhs out of range");
        if (nrhs == 0) return H2_OK;
        require(X && Y && ldx && ldy, "h2_batch_matvec: NULL arrays");
        require(mode >= H2_FP64 && mode <= H2_TF32X3, "h2_batch_matvec: unknown mode");
        h2::batch_matvec(b, X, ldx, Y, ldy, nrhs, mode, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_batch_tuned(h2_batch_t b, int64_t nrhs, int mode, int* rhs_tile) {
    return guard([&] {
        require(b && rhs_tile, "h2_batch_tuned: NULL argument");
        *rhs_tile = h2::batch_tuned(b, nrhs, mode);
        return H2_OK;
    });
}

void h2_batch_free(h2_batch_t b) {
    if (b) {
        cudaDeviceSynchronize();
        delete b;
    }
}

int h2_matvec_batched(int count, const h2_handle_t* hs, const void* const* X, const int64_t* ldx, void* const* Y,
                      const int64_t* ldy, int64_t nrhs, int mode, h2_stream_t stream) {
    h2_batch_t b = nullptr;
    int st = h2_batch_create(count, hs, &b);
    if (st != H2_OK) return st;
    st = h2_batch_matvec(b, X, ldx, Y, ldy, nrhs, mode, stream);
    h2_batch_free(b);
    return st;
}

int h2_rankmodel_create(uint64_t seed, int bf16, h2_rankmodel_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_rankmodel_create: out is NULL");
        *out = nullptr;
        *out = h2::rm_create(seed, bf16);
        return H2_OK;
    });
}

void h2_rankmodel_free(h2_rankmodel_t m) {
    if (m) {
        cudaDeviceSynchronize();
        h2::rm_free(m);
    }
}

int h2_rankmodel_get(h2_rankmodel_t m, float* p, float* am, float* av, int64_t* step) {
    return guard([&] {
        require(m != nullptr, "h2_rankmodel_get: NULL model");
        h2::rm_get(m, p, am, av, step);
        return H2_OK;
    });
}

int h2_rankmodel_set(h2_rankmodel_t m, const float* p, const float* am, const float* av, int64_t step) {
    return guard([&] {
        require(m != nullptr, "h2_rankmodel_set: NULL model");
        h2::rm_set(m, p, am, av, step);
        return H2_OK;
    });
}

int h2_colored_plan(h2_tree_t tree, int q, int* counts) {
    return guard([&] {
        require(tree && counts, "h2_colored_plan: NULL argument");
        require(q >= 1 && q <= 16, "h2_colored_plan: q must be in 1..16");
        h2::colored_plan_counts(tree, q, counts);
        return H2_OK;
    });
}

int h2_lowrank_update(h2_handle_t A, const double* B, int64_t ldb, int r, const double* M, double tol,
                      const h2_build_opts* opts, h2_handle_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_lowrank_update: out is NULL");
        *out = nullptr;
        require(A != nullptr, "h2_lowrank_update: NULL handle");
        require(r >= 0 && r <= 144, "h2_lowrank_update: r must be in 0..144");
        require(r == 0 || (B != nullptr && ldb >= A->N && ldb <= INT32_MAX), "h2_lowrank_update: bad B or ldb");
        if (M)
            for (int64_t i = 0; i < (int64_t)r * r; ++i)
                require(std::isfinite(M[i]), "h2_lowrank_update: M must be finite");
        h2_build_opts o = checked_opts(tol, opts);
        auto* h = new h2_handle_s();
        try {
            h2::AllocScope scope((cudaStream_t)o.stream);
            const int st = h2::update_handle(A, B, ldb, r, M, tol, o, h);
            *out = h;
            return st;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int h2_invert_opts_default(h2_invert_opts* o) {
    if (!o) return H2_ERR_INVALID_ARG;
    std::memset(o, 0, sizeof(*o));
    o->order = 2;
    o->eps = 1e-6;
    o->eps_loose = 1e-6;
    o->theta = 0.1;
    o->max_iter = 50;
    o->shift = 0.0;
    o->res_maxit = 50;
    o->res_rtol = 1e-2;
    o->seed = 9;
    return H2_OK;
}

int h2_invert(h2_handle_t A, const h2_invert_opts* opts, const h2_build_opts* build_opts, h2_handle_t* X_out,
              h2_invert_stats* stats) {
    return guard([&] {
        require(X_out != nullptr, "h2_invert: X_out is NULL");
        *X_out = nullptr;
        require(A != nullptr, "h2_invert: NULL handle");
        h2_invert_opts io;
        h2_invert_opts_default(&io);
        if (opts) io = *opts;
        require(io.unroll > 0 || (io.order >= 2 && io.order <= 64), "h2_invert: order must be in 2..64");
        require(io.eps > 0.0 && std::isfinite(io.eps), "h2_invert: eps must be positive");
        require(io.eps_loose >= io.eps && std::isfinite(io.eps_loose), "h2_invert: need eps_loose >= eps");
        require(io.theta > 0.0 && std::isfinite(io.theta), "h2_invert: theta must be positive");
        require(io.max_iter >= 0 && io.max_iter <= H2_MAX_INVERT_ITERS, "h2_invert: max_iter out of range");
        require(std::isfinite(io.shift), "h2_invert: shift must be finite");
        require(io.res_maxit >= 1 && io.res_rtol > 0.0, "h2_invert: bad power-iteration settings");
        require(io.unroll >= 0 && io.unroll <= 6, "h2_invert: unroll must be in 0..6");
        require(!io.x0 || (io.x0->N == A->N && io.x0->tree->L == A->tree->L),
                "h2_invert: x0 must be a handle on A's tree");
        if (io.unroll > 0) {
            io.order = 1 << io.unroll;
            io.max_iter = 1;
        }
        h2_build_opts bo = checked_opts(io.eps, build_opts);
        h2_invert_stats local;
        h2_handle_s* X = nullptr;
        h2::invert(A, io, bo, &X, stats ? stats : &local);
        *X_out = X;
        return (stats ? stats : &local)->converged ? (int)H2_OK : (int)H2_WARN_TOL_NOT_MET;
    });
}

int h2_rankmodel_save(h2_rankmodel_t m, const char* path) {
    return guard([&] {
        require(m && path, "h2_rankmodel_save: NULL argument");
        h2::rm_save(m, path);
        return H2_OK;
    });
}

int h2_rankmodel_load(const char* path, h2_rankmodel_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_rankmodel_load: out is NULL");
        *out = nullptr;
        require(path != nullptr, "h2_rankmodel_load: NULL path");
        *out = h2::rm_load(path);
        return H2_OK;
    });
}

int h2_rankmodel_features(h2_tree_t tree, double kappa_T, double density, double tol, double* out) {
    return guard([&] {
        require(tree && out, "h2_rankmodel_features: NULL argument");
        require(kappa_T > 0.0 && std::isfinite(kappa_T), "h2_rankmodel_features: kappa_T must be positive");
        require(tol > 0.0 && std::isfinite(tol), "h2_rankmodel_features: tol must be positive");
        require(std::isfinite(density), "h2_rankmodel_features: density must be finite");
        h2::rm_features(tree, kappa_T, density, tol, out);
        return H2_OK;
    });
}

int h2_rankmodel_loss_grad(h2_rankmodel_t m, const float* X, const float* t, int64_t n, float* loss, float* grad) {
    return guard([&] {
        require(m != nullptr, "h2_rankmodel_loss_grad: NULL model");
        h2::rm_loss_grad(m, X, t, n, loss, grad);
        return H2_OK;
    });
}

int h2_rankmodel_train(h2_rankmodel_t m, const float* X, const float* t, int64_t n, const int32_t* idx, int steps,
                       int batch, float lr, float* loss_out, h2_stream_t stream) {
    return guard([&] {
        require(m != nullptr, "h2_rankmodel_train: NULL model");
        h2::rm_train(m, X, t, n, idx, steps, batch, lr, loss_out, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_rankmodel_predict(h2_rankmodel_t m, const float* X, int64_t n, float* y, h2_stream_t stream) {
    return guard([&] {
        require(m != nullptr, "h2_rankmodel_predict: NULL model");
        h2::rm_predict(m, X, n, y, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_rankmodel_q_levels(h2_rankmodel_t m, h2_tree_t tree, double kappa_T, double density, double tol, int pad,
                          int q_max, int32_t* q, float* y) {
    return guard([&] {
        require(m && tree && q, "h2_rankmodel_q_levels: NULL argument");
        require(kappa_T > 0.0 && std::isfinite(kappa_T) && tol > 0.0 && std::isfinite(tol) && std::isfinite(density),
                "h2_rankmodel_q_levels: bad kappa_T, density or tol");
        require(pad >= 0 && q_max >= 8, "h2_rankmodel_q_levels: need pad >= 0 and q_max >= 8");
        h2::rm_q_levels(m, tree, kappa_T, density, tol, pad, q_max, q, y);
        return H2_OK;
    });
}

int h2_rankmodel_targets(h2_handle_t h, int32_t* levels, float* targets, int* count) {
    return guard([&] {
        require(h && count, "h2_rankmodel_targets: NULL handle or count");
        int n = 0;
        for (int l = 1; l <= h->stats.levels; ++l) {
            if (h->stats.range_passed[l] < 0) continue;   // identity range: nothing was learned here
            if (levels) levels[n] = l;
            if (targets) targets[n] = (float)std::log2(1.0 + (double)h->stats.range_need[l]);
            ++n;
        }
        *count = n;
        return H2_OK;
    });
}

int h2_import(h2_tree_t tree, const int32_t* ranks, const double* U, const double* E, const double* S,
              const double* D, int keep_fp32, int keep_bf16, h2_handle_t* out) {
    return guard([&] {
        require(out != nullptr, "h2_import: out is NULL");
        *out = nullptr;
        require(tree && ranks, "h2_import: NULL tree or ranks");
        const int L = tree->L;
        auto* h = new h2_handle_s();
        try {
            h->tree = std::make_shared<h2_tree_s>(*tree);
            h->L = L;
            h->N = tree->N;
            h->koff.assign(L + 2, 0);
            for (int l = 0; l <= L + 1; ++l) h->koff[l] = ((int64_t)1 << l) - 1;
            h->k.assign((size_t)h->koff[L + 1], 0);
            for (size_t i = 0; i < h->k.size(); ++i) {
                require(ranks[i] >= 0 && ranks[i] <= 96, "h2_import: rank out of range");
                h->k[i] = ranks[i];
            }
            for (int t = 0; t < (1 << L); ++t)
                require(h->k[h->koff[L] + t] <= tree->size[L][t], "h2_import: leaf rank above leaf size");
            for (int l = 0; l < L; ++l)
                for (int p = 0; p < (1 << l); ++p)
                    require(h->k[h->koff[l] + p] <= h->k[h->koff[l + 1] + 2 * p] + h->k[h->koff[l + 1] + 2 * p + 1],
                            "h2_import: rank above the children's ranks");
            require(tree->leaf_max <= 96, "h2_import: leaf size above 96");
            h2::layout_factors(h);
            std::vector<double> fac((size_t)std::max<int64_t>(h->fac_entries, 1), 0.0);
            // leaf bases
            if (h->entries_U) {
                require(U != nullptr, "h2_import: NULL U");
                std::memcpy(fac.data(), U, h->entries_U * sizeof(double));
            }
            // transfer matrices: E_c (k_c x k_p, per child, levels 1..L) -> stacked [E_c1; E_c2]
            {
                int64_t eo = 0;
                for (int l = 1; l <= L; ++l)
                    for (int c = 0; c < (1 << l); ++c) {
                        const int p = c >> 1;
                        const int kc = h->k[h->koff[l] + c], kp = h->k[h->koff[l - 1] + p];
                        const int k1 = h->k[h->koff[l] + 2 * p], k2 = h->k[h->koff[l] + 2 * p + 1];
                        const int64_t base = h->uh_off[h->koff[l - 1] + p] + ((c & 1) ? k1 : 0);
                        if (kc && kp) require(E != nullptr, "h2_import: NULL E");
                        for (int j = 0; j < kp; ++j)
                            for (int i = 0; i < kc; ++i) fac[base + i + (int64_t)j * (k1 + k2)] = E[eo + i + (int64_t)j * kc];
                        eo += (int64_t)kc * kp;
                    }
            }
            if (h->entries_S) {
                require(S != nullptr, "h2_import: NULL S");
                std::memcpy(fac.data() + h->entries_U + h->entries_E, S, h->entries_S * sizeof(double));
            }
            if (h->entries_D) {
                require(D != nullptr, "h2_import: NULL D");
                std::memcpy(fac.data() + h->entries_U + h->entries_E + h->entries_S, D, h->entries_D * sizeof(double));
            }
            H2_CUDA(cudaMemcpy(h->fac64.p, fac.data(), fac.size() * sizeof(double), cudaMemcpyHostToDevice));
            std::vector<int32_t> perm(h->N);
            for (int64_t i = 0; i < h->N; ++i) perm[i] = (int32_t)tree->perm[i];
            h->d_perm.reserve(h->N);
            H2_CUDA(cudaMemcpy(h->d_perm.p, perm.data(), h->N * sizeof(int32_t), cudaMemcpyHostToDevice));
            h2::build_plan(h, nullptr);
            h2::make_copies(h, keep_fp32, keep_bf16, nullptr);
            H2_CUDA(cudaDeviceSynchronize());
            std::memset(&h->stats, 0, sizeof(h->stats));
            h->stats.n = h->N;
            h->stats.levels = L;
            h->stats.leaf_max = tree->leaf_max;
            h->stats.tol_met = 1;
            for (int l = 0; l <= L && l < H2_MAX_LEVELS; ++l) {
                int mx = 0;
                for (int b = 0; b < (1 << l); ++b) mx = std::max(mx, h->k[h->koff[l] + b]);
                h->stats.max_rank[l] = mx;
            }
            h->stats.far_lower = 0;
            for (auto& f : h->far_lower) h->stats.far_lower += (int64_t)f.size();
            h->stats.near_lower = (int64_t)h->near_lower.size();
            h->stats.entries_D = h->entries_D;
            h->stats.entries_S = h->entries_S;
            h->stats.entries_U = h->entries_U;
            h->stats.entries_E = h->entries_E;
            *out = h;
            return H2_OK;
        } catch (...) {
            delete h;
            throw;
        }
    });
}

int h2_factor_sizes(h2_handle_t h, int64_t* n_ranks, int64_t* n_U, int64_t* n_E, int64_t* n_S, int64_t* n_D) {
    return guard([&] {
        require(h != nullptr, "h2_factor_sizes: NULL handle");
        if (n_ranks) *n_ranks = (int64_t)h->k.size();
        if (n_U) *n_U = h->entries_U;
        if (n_E) *n_E = h->entries_E;
        if (n_S) *n_S = h->entries_S;
        if (n_D) *n_D = h->entries_D;
        return H2_OK;
    });
}

int h2_export(h2_handle_t h, int32_t* ranks, double* U, double* E, double* S, double* D) {
    return guard([&] {
        require(h != nullptr, "h2_export: NULL handle");
        H2_CUDA(cudaDeviceSynchronize());
        std::vector<double> fac((size_t)std::max<int64_t>(h->fac_entries, 1));
        if (h->fac_entries)
            H2_CUDA(cudaMemcpy(fac.data(), h->fac64.p, h->fac_entries * sizeof(double), cudaMemcpyDeviceToHost));
        if (ranks)
            for (size_t i = 0; i < h->k.size(); ++i) ranks[i] = h->k[i];
        if (U && h->entries_U) std::memcpy(U, fac.data(), h->entries_U * sizeof(double));
        if (E) {
            int64_t eo = 0;
            const int L = h->L;
            for (int l = 1; l <= L; ++l)
                for (int c = 0; c < (1 << l); ++c) {
                    const int p = c >> 1;
                    const int kc = h->k[h->koff[l] + c], kp = h->k[h->koff[l - 1] + p];
                    const int k1 = h->k[h->koff[l] + 2 * p], k2 = h->k[h->koff[l] + 2 * p + 1];
                    const int64_t base = h->uh_off[h->koff[l - 1] + p] + ((c & 1) ? k1 : 0);
                    for (int j = 0; j < kp; ++j)
                        for (int i = 0; i < kc; ++i) E[eo + i + (int64_t)j * kc] = fac[base + i + (int64_t)j * (k1 + k2)];
                    eo += (int64_t)kc * kp;
                }
        }
        if (S && h->entries_S) std::memcpy(S, fac.data() + h->entries_U + h->entries_E, h->entries_S * sizeof(double));
        if (D && h->entries_D)
            std::memcpy(D, fac.data() + h->entries_U + h->entries_E + h->entries_S, h->entries_D * sizeof(double));
        return H2_OK;
    });
}

int h2_matvec(h2_handle_t h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs, int mode,
              h2_stream_t stream) {
    return guard([&] {
        require(h != nullptr, "h2_matvec: NULL handle");
        require(nrhs >= 0, "h2_matvec: nrhs < 0");
        if (nrhs == 0) return H2_OK;
        require(X != nullptr && Y != nullptr, "h2_matvec: NULL X or Y");
        require(ldx >= h->N && ldy >= h->N, "h2_matvec: leading dimension smaller than n");
        require(mode >= H2_FP64 && mode <= H2_FP32C, "h2_matvec: unknown mode");
        h2::run_matvec(h, X, ldx, Y, ldy, nrhs, mode, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_matvec_host(h2_handle_t h, const void* X_host, int64_t ldx, void* Y_host, int64_t ldy, int64_t nrhs, int mode,
                   h2_stream_t stream) {
    return guard([&] {
        require(h != nullptr, "h2_matvec_host: NULL handle");
        require(nrhs >= 0, "h2_matvec_host: nrhs < 0");
        if (nrhs == 0) return H2_OK;
        require(X_host != nullptr && Y_host != nullptr, "h2_matvec_host: NULL X or Y");
        require(ldx >= h->N && ldy >= h->N, "h2_matvec_host: leading dimension smaller than n");
        require(mode >= H2_FP64 && mode <= H2_FP32C, "h2_matvec_host: unknown mode");
        h2::run_matvec_host(h, X_host, ldx, Y_host, ldy, nrhs, mode, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_matvec_noalloc(h2_handle_t h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs, int mode,
                      h2_stream_t stream) {
    return guard([&] {
        require(h != nullptr, "h2_matvec_noalloc: NULL handle");
        require(nrhs >= 0, "h2_matvec_noalloc: nrhs < 0");
        if (nrhs == 0) return H2_OK;
        require(X != nullptr && Y != nullptr, "h2_matvec_noalloc: NULL X or Y");
        require(ldx >= h->N && ldy >= h->N, "h2_matvec_noalloc: leading dimension smaller than n");
        require(mode >= H2_FP64 && mode <= H2_FP32C, "h2_matvec_noalloc: unknown mode");
        h2::run_matvec_noalloc(h, X, ldx, Y, ldy, nrhs, mode, (cudaStream_t)stream);
        return H2_OK;
    });
}

int h2_profile(h2_handle_t h, int enable) {
    return guard([&] {
        require(h != nullptr, "h2_profile: NULL handle");
        h->prof = enable ? 1 : 0;
        return H2_OK;
    });
}

int h2_profile_read(h2_handle_t h, double* ms_out, int64_t* launches_out) {
    return guard([&] {
        require(h != nullptr, "h2_profile_read: NULL handle");
        h2::profile_read(h, ms_out, launches_out);
        return H2_OK;
    });
}

int h2_gemm_profile(int enable) {
    return guard([&] {
        h2::gemm_profile_enable(enable ? 1 : 0);
        return H2_OK;
    });
}

int h2_gemm_profile_read(double* ms_out, double* flops_out, int64_t* launches_out, double* bytes_out) {
    return guard([&] {
        h2::gemm_profile_read(ms_out, flops_out, launches_out, bytes_out);
        return H2_OK;
    });
}

int h2_stack_profile_read(int which, double* ms_out, double* flops_out, int64_t* launches_out) {
    return guard([&] {
        require(which == 0 || which == 1, "h2_stack_profile_read: which must be 0 or 1");
        h2::stack_profile_read(which, ms_out, flops_out, launches_out);
        return H2_OK;
    });
}

int h2_device_status(h2_handle_t h) {
    return guard([&] {
        require(h != nullptr, "h2_device_status: NULL handle");
        H2_CUDA(cudaDeviceSynchronize());
        if (h2::tc_device_error(h)) h2::fail(H2_ERR_DEVICE_CHECK, "a tensor-core kernel timed out on a bounded wait");
        return H2_OK;
    });
}

int h2_get_stats(h2_handle_t h, h2_stats* out) {
    return guard([&] {
        require(h && out, "h2_get_stats: NULL argument");
        *out = h->stats;
        return H2_OK;
    });
}

void h2_free(h2_handle_t h) {
    if (h) {
        cudaDeviceSynchronize();
        delete h;
    }
}

const char* h2_error_string(int status) {
    switch (status) {
        case H2_OK: return "H2_OK";
        case H2_ERR_INVALID_ARG: return "H2_ERR_INVALID_ARG";
        case H2_ERR_CUDA: return "H2_ERR_CUDA";
        case H2_ERR_OP_FAILED: return "H2_ERR_OP_FAILED";
        case H2_ERR_NAN: return "H2_ERR_NAN";
        case H2_ERR_OOM: return "H2_ERR_OOM";
        case H2_ERR_DEVICE_CHECK: return "H2_ERR_DEVICE_CHECK";
        case H2_WARN_TOL_NOT_MET: return "H2_WARN_TOL_NOT_MET";
        default: return "unknown status";
    }
}

const char* h2_last_error(void) { return g_last_error.c_str(); }

int64_t h2_launch_count(void) { return h2::g_launches.load(); }

int64_t h2_device_bytes(void) { return h2::dev_live_bytes(); }

int h2_set_device_limit(int64_t bytes) {
    h2::dev_alloc_limit(bytes);
    return H2_OK;
}

const char* h2_version(void) { return "h2hess 0.1 (sm_103a)"; }

}  // extern "C"
