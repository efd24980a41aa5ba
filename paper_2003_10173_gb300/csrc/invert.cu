// Iterative inversion of a built H^2 matrix from products (Appendix A): every iterate of the
// order-l hyperpower iteration X_{k+1} = X_k sum_{i<l} R_k^i, R_k = I - A X_k (l = 2: Newton-
// Schulz) is a new H^2 matrix constructed by peeling (Section 3.3) from a sampler that applies
// the iteration to the probe block with H^2 matvecs of A and X_k (Algorithms 2 and 4).  A may
// carry a diagonal shift (a regularised Hessian H + shift I).  X_0 = alpha I, alpha = 1/||A||_2,
// or a given iterate (warm start).  An unrolled step (k Newton-Schulz steps as one construction)
// is the order-2^k hyperpower step: prod_{j<k} (I + R^{2^j}) = sum_{i<2^k} R^i.
// Construction threshold of iterate k: max(eps / (||A|| ||X_k||), min(eps_loose, theta E^2)),
// E = ||A X_k - I||_2 by power iteration on (X A - I)(A X - I), started from the counter-based
// Gaussians of the error stream in original node order.
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>

#include "handle.h"

namespace h2 {

int build_handle(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o,
                 h2_handle_s* h);
void finish_handle(h2_handle_s* h, const h2_build_opts& o, cudaStream_t s);

namespace {

constexpr int NT = 256;
constexpr int STREAM_ERR = 3;       // residual start vector: Gaussians in original node order
constexpr int STREAM_INVERT = 4;    // ||A|| start vector

__global__ void iota_kernel(int32_t* p, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

unsigned grid_of(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + NT - 1) / NT, 152 * 16)); }

// r <- r - u - shift t;  y <- y + r   (n x c, leading dimension n)
__global__ void hp_update_kernel(double* __restrict__ r, const double* __restrict__ u, const double* __restrict__ t,
                                 double shift, double* __restrict__ y, int64_t total) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = r[e] - u[e] - shift * t[e];
        r[e] = v;
        y[e] += v;
    }
}

// out[i + j ldo] = alpha in[i + j ldi] + beta extra[i + j ldi]  (extra may be null; out may be in)
__global__ void hp_axpby_kernel(const double* in, int64_t ldi, double alpha, const double* extra, double beta,
                                double* out, int64_t ldo, int64_t n, int64_t c) {
    const int64_t total = n * c;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % n, j = e / n;
        double v = alpha * in[i + j * ldi];
        if (extra) v += beta * extra[i + j * ldi];
        out[i + j * ldo] = v;
    }
}

struct Sampler {
    h2_handle_s* A = nullptr;
    double shift = 0.0;
    h2_handle_s* X = nullptr;   // null: X = alpha I
    double alpha = 0.0;
    int order = 2;
    DevBuf<double> R, T, U, Y;
    std::string err;

    // out = X in (n x c), leading dimensions as given
    void apply_X(const double* in, int64_t ldi, double* out, int64_t ldo, int64_t n, int64_t c, cudaStream_t s) {
        if (X) {
            run_matvec(X, in, ldi, out, ldo, c, H2_FP64, s);
        } else {
            hp_axpby_kernel<<<grid_of(n * c), NT, 0, s>>>(in, ldi, alpha, nullptr, 0.0, out, ldo, n, c);
            after_launch("hp_scale");
        }
    }
    // out = (A + shift I) in  (contiguous n x c)
    void apply_A(const double* in, double* out, int64_t n, int64_t c, cudaStream_t s) {
        run_matvec(A, in, n, out, n, c, H2_FP64, s);
        if (shift != 0.0) {
            hp_axpby_kernel<<<grid_of(n * c), NT, 0, s>>>(out, n, 1.0, in, shift, out, n, n, c);
            after_launch("hp_shift");
        }
    }
};

// Y = X_{k+1} Omega: Y = R = Omega; order - 1 times R <- R - A X_k R, Y <- Y + R; Y <- X_k Y.
int sampler_apply(void* ctx, int64_t n, int64_t nrhs, const double* Om, int64_t ldo, double* Yout, int64_t ldy,
                  h2_stream_t stream) {
    auto* S = static_cast<Sampler*>(ctx);
    try {
        cudaStream_t s = (cudaStream_t)stream;
        const size_t need = (size_t)n * (size_t)nrhs;
        S->R.reserve(need);
        S->T.reserve(need);
        S->U.reserve(need);
        S->Y.reserve(need);
        H2_CUDA(cudaMemcpy2DAsync(S->R.p, n * sizeof(double), Om, ldo * sizeof(double), n * sizeof(double), nrhs,
                                  cudaMemcpyDeviceToDevice, s));
        H2_CUDA(cudaMemcpyAsync(S->Y.p, S->R.p, need * sizeof(double), cudaMemcpyDeviceToDevice, s));
        for (int i = 1; i < S->order; ++i) {
            S->apply_X(S->R.p, n, S->T.p, n, n, nrhs, s);              // T = X_k R
            run_matvec(S->A, S->T.p, n, S->U.p, n, nrhs, H2_FP64, s);  // U = H T
            hp_update_kernel<<<grid_of((int64_t)need), NT, 0, s>>>(S->R.p, S->U.p, S->T.p, S->shift, S->Y.p,
                                                                   (int64_t)need);
            after_launch("hp_update");
        }
        S->apply_X(S->Y.p, n, Yout, ldy, n, nrhs, s);
        return 0;
    } catch (const Error& e) {
        S->err = e.what();
        return 1;
    } catch (...) {
        S->err = "unknown failure";
        return 1;
    }
}

double host_norm(const double* d_x, int64_t n, DevBuf<double>& red, cudaStream_t s) {
    red.reserve(1);
    col_sqnorms(n, 1, d_x, n, red.p, s);
    double v = 0.0;
    H2_CUDA(cudaMemcpyAsync(&v, red.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
    return std::sqrt(v);
}

void scale_vec(double* x, int64_t n, double a, cudaStream_t s) {
    hp_axpby_kernel<<<grid_of(n), NT, 0, s>>>(x, n, a, nullptr, 0.0, x, n, n, 1);
    after_launch("hp_scale");
}

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

void invert(h2_handle_s* A, const h2_invert_opts& io, const h2_build_opts& bo, h2_handle_s** Xout,
            h2_invert_stats* st) {
    const double t0 = now_s();
    cudaStream_t s = (cudaStream_t)bo.stream;
    AllocScope scope(s);   // workspace and retired iterates are reused by the next construction
    const int64_t N = A->N;
    Sampler S;
    S.A = A;
    S.shift = io.shift;
    S.order = io.order;
    DevBuf<double> v(N), w(N), t(N), z(N), red(1);
    DevBuf<int32_t> ident(N);
    iota_kernel<<<grid_of(N), NT, 0, s>>>(ident.p, N);
    after_launch("iota");
    // ||A||_2 by power iteration
    gaussian_vector(N, A->d_perm.p, io.seed, STREAM_INVERT, v.p, s);
    double nv = host_norm(v.p, N, red, s);
    scale_vec(v.p, N, 1.0 / nv, s);
    double normA = 0.0, prev = 0.0;
    for (int it = 0; it < io.res_maxit; ++it) {
        S.apply_A(v.p, w.p, N, 1, s);
        normA = host_norm(w.p, N, red, s);
        if (!(normA > 0.0) || !std::isfinite(normA)) fail(H2_ERR_NAN, "h2_invert: ||A|| is zero or not finite");
        scale_vec(w.p, N, 1.0 / normA, s);
        std::swap(v.p, w.p);
        if (it > 0 && std::fabs(normA - prev) <= io.res_rtol * normA) break;
        prev = normA;
    }
    S.alpha = 1.0 / normA;
    double normX = S.alpha;
    if (io.x0) {   // warm start from a given iterate (read only; never freed here)
        S.X = io.x0;
        normX = io.x0->stats.norm_est > 0.0 ? io.x0->stats.norm_est : S.alpha;
    }
    // residual E = ||A X - I||_2 of the current iterate
    auto residual = [&]() {
        gaussian_vector(N, ident.p, io.seed, STREAM_ERR, v.p, s);
        scale_vec(v.p, N, 1.0 / host_norm(v.p, N, red, s), s);
        double E = 0.0, pe = 0.0;
        for (int it = 0; it < io.res_maxit; ++it) {
            S.apply_X(v.p, N, t.p, N, N, 1, s);
            S.apply_A(t.p, w.p, N, 1, s);
            hp_axpby_kernel<<<grid_of(N), NT, 0, s>>>(w.p, N, 1.0, v.p, -1.0, w.p, N, N, 1);   // w = A X v - v
            after_launch("hp_axpby");
            E = host_norm(w.p, N, red, s);
            S.apply_A(w.p, t.p, N, 1, s);
            S.apply_X(t.p, N, z.p, N, N, 1, s);
            hp_axpby_kernel<<<grid_of(N), NT, 0, s>>>(z.p, N, 1.0, w.p, -1.0, z.p, N, N, 1);   // z = X A w - w
            after_launch("hp_axpby");
            const double nz = host_norm(z.p, N, red, s);
            if (!std::isfinite(E) || !std::isfinite(nz)) fail(H2_ERR_NAN, "h2_invert: residual is not finite");
            if (nz == 0.0) break;
            scale_vec(z.p, N, 1.0 / nz, s);
            std::swap(v.p, z.p);
            if (it > 0 && std::fabs(E - pe) <= io.res_rtol * E) break;
            pe = E;
        }
        return E;
    };
    std::memset(st, 0, sizeof(*st));
    st->norm_A = normA;
    st->alpha = S.alpha;
    h2_handle_s* X = nullptr;
    int k = 0;
    try {
        for (;; ++k) {
            const double E = residual();
            st->err[k] = E;
            if (E <= io.eps) {
                st->converged = 1;
                break;
            }
            if (k == io.max_iter) break;
            if (k > 0 && E > 0.9 * st->err[k - 1] && std::pow(st->err[k - 1], io.order) < 0.5 * E) break;
            const double floor = io.eps / (normA * normX);
            // an unrolled step is the final construction: it is built to the floor that the target
            // residual allows, not to a threshold derived from the current residual
            const double eps_k = io.unroll > 0 ? floor : std::max(floor, std::min(io.eps_loose, io.theta * E * E));
            const double tb = now_s();
            auto* Xn = new h2_handle_s();
            try {
                build_handle(sampler_apply, &S, A->tree.get(), eps_k, bo, Xn);
                finish_handle(Xn, bo, s);
            } catch (...) {
                delete Xn;
                if (!S.err.empty()) fail(H2_ERR_OP_FAILED, "h2_invert: sampler failed: " + S.err);
                throw;
            }
            st->eps_k[k] = eps_k;
            st->samples[k] = Xn->stats.samples;
            st->t_build[k] = now_s() - tb;
            normX = Xn->stats.norm_est;
            delete X;
            X = Xn;
            S.X = X;
        }
    } catch (...) {
        delete X;
        throw;
    }
    st->iterations = k;
    if (!X) {
        // converged at X_0 = alpha I: construct it (one product per probe column)
        auto* Xn = new h2_handle_s();
        S.order = 1;
        try {
            build_handle(sampler_apply, &S, A->tree.get(), io.eps, bo, Xn);
            finish_handle(Xn, bo, s);
        } catch (...) {
            delete Xn;
            throw;
        }
        X = Xn;
    }
    st->final_err = st->err[k];
    st->t_total = now_s() - t0;
    *Xout = X;
}

}  // namespace h2
