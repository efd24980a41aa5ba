// Hessian operators shipped with the library (callbacks of type h2_op_fn).
//
// heat2d: misfit Hessian of initial-condition inversion for the heat equation
// on the unit square, H = F diag(mask) F / sigma^2 with F = exp(T kappa Lap_h)
// (5-point Dirichlet Laplacian on the n x n interior grid).  The 2-D Laplacian is
// the Kronecker sum of 1-D ones, so its exponential is a Kronecker product:
// F = F1 (x) F1 with F1 = exp(T kappa Lap_1) = S diag(exp(-T kappa mu)) S, S the
// orthonormal type-I sine transform and mu_a = (4/h^2) sin^2(a pi h / 2).  With the
// vector x read as the column-major n x n array X (X[j, i] = x[i n + j]),
//     F x  <->  F1 X F1.
// The factors exp(-T kappa mu_b) decay like exp(-T kappa pi^2 b^2): only the r modes with
// exp(-T kappa mu_b) >= 2^-60 exp(-T kappa mu_1) are representable next to the largest one in
// FP64, so F1 = S_r diag(e_r) S_r^T to rounding (dropped part below 2^-60 relative), and
//     F1 X F1 = (S_r diag(e_r)) ((S_r^T X) S_r) diag(e_r) S_r^T
// costs 8 r n^2 flops instead of 4 n^3 (four FP64 GEMMs).  When 2 r >= n the dense F1 (formed
// once on the device from S) is used instead.
//
// dense: Y = A X with a caller-owned dense matrix.
#include <cmath>

#include "common.h"

namespace h2 {

namespace {

constexpr int NT = 256;

__global__ void scale_by_kernel(double* __restrict__ x, const double* __restrict__ f, int64_t per, int64_t total,
                                double c) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        x[e] *= c * f[e % per];
}

__global__ void store_kernel(const double* __restrict__ src, int64_t N, int64_t nrhs, double c, double* __restrict__ Y,
                             int64_t ldy) {
    const int64_t total = N * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e % N, r = e / N;
        Y[i + r * ldy] = c * src[e];
    }
}

unsigned grid_for(int64_t total) {
    int64_t b = (total + NT - 1) / NT;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)(b < 1 ? 1 : b);
}

struct Heat2d {
    int n = 0;
    int r = 0;               // retained sine modes (r == n: dense F1)
    double inv_s2 = 0.0;
    DevBuf<double> F1, Sr, Sar, mask, W1, W2, W3;
    GemmBatch gb;
};

// B <- F B = F1 B_q F1 for every column q of B (N x c contiguous); W, T are scratch
// (W: N x c, T: r n c).
void apply_F(Heat2d& H, double* B, double* W, double* T, int64_t c, cudaStream_t s) {
    const int n = H.n;
    const int64_t n2 = (int64_t)n * n;
    if (H.r == n) {
        // W = F1 * B_view  (n x n*c), then B_q = W_q * F1
        H.gb.add(H.F1.p, n, 0, B, n, 0, W, n, n, (int)(n * c), n, 1.0, 0.0);
        H.gb.run(s);
        for (int64_t q = 0; q < c; ++q) H.gb.add(W + q * n2, n, 0, H.F1.p, n, 0, B + q * n2, n, n, n, n, 1.0, 0.0);
        H.gb.run(s);
        return;
    }
    const int r = H.r;
    // T = S_r^T B_view (r x n c);  W = (S_r diag(e)) T = F1 B_view
    H.gb.add(H.Sr.p, n, 1, B, n, 0, T, r, r, (int)(n * c), n, 1.0, 0.0);
    H.gb.run(s);
    H.gb.add(H.Sar.p, n, 0, T, r, 0, W, n, n, (int)(n * c), r, 1.0, 0.0);
    H.gb.run(s);
    // T_q = W_q (S_r diag(e))  (n x r);  B_q = T_q S_r^T = W_q F1
    for (int64_t q = 0; q < c; ++q) H.gb.add(W + q * n2, n, 0, H.Sar.p, n, 0, T + q * n * r, n, n, r, n, 1.0, 0.0);
    H.gb.run(s);
    for (int64_t q = 0; q < c; ++q) H.gb.add(T + q * n * r, n, 0, H.Sr.p, n, 1, B + q * n2, n, n, n, r, 1.0, 0.0);
    H.gb.run(s);
}

struct DenseOp {
    const double* A = nullptr;
    int64_t n = 0, lda = 0;
    GemmBatch gb;
};

// Factored symmetric operator Y = scale Z (Z^T X): a misfit Hessian A^-T O^T O A^-1 / sigma^2
// given Z = A^-T O^T (one adjoint solve per observation).
struct LowRankOp {
    const double* Z = nullptr;
    int64_t n = 0, r = 0, ldz = 0;
    double scale = 1.0;
    DevBuf<double> T;
    GemmBatch gb;
};

}  // namespace

}  // namespace h2

using namespace h2;

extern "C" {

int h2_heat2d_create(int n, double kappa, double T, double sigma, const double* mask_host, void** ctx_out) {
    if (!ctx_out) return H2_ERR_INVALID_ARG;
    *ctx_out = nullptr;
    if (n < 1 || n > 4096 || !(kappa >= 0.0) || !(T >= 0.0) || !(sigma > 0.0) || !mask_host) return H2_ERR_INVALID_ARG;
    Heat2d* H = nullptr;
    try {
        H = new Heat2d();
        H->n = n;
        H->inv_s2 = 1.0 / (sigma * sigma);
        const double h = 1.0 / (n + 1);
        // S and S diag(exp(-T kappa mu)) on the host (mu increases with the mode index b)
        std::vector<double> S((size_t)n * n), Sa((size_t)n * n);
        std::vector<double> e(n);
        for (int b = 0; b < n; ++b) {
            const double mu = (4.0 / (h * h)) * std::pow(std::sin(0.5 * M_PI * h * (b + 1)), 2);
            e[b] = std::exp(-T * kappa * mu);
            for (int a = 0; a < n; ++a) {
                S[a + (size_t)b * n] = std::sqrt(2.0 * h) * std::sin(M_PI * h * (double)(a + 1) * (b + 1));
                Sa[a + (size_t)b * n] = S[a + (size_t)b * n] * e[b];
            }
        }
        int r = 0;
        while (r < n && e[r] >= 0x1p-60 * e[0]) ++r;
        H->r = (2 * r >= n) ? n : std::max(r, 1);
        const int64_t N = (int64_t)n * n;
        H->mask.reserve(N);
        if (H->r == n) {
            // F1 = (S diag(e)) S by the library's GEMM
            DevBuf<double> dS(S.size()), dSa(Sa.size());
            H->F1.reserve(S.size());
            H2_CUDA(cudaMemcpy(dS.p, S.data(), S.size() * sizeof(double), cudaMemcpyHostToDevice));
            H2_CUDA(cudaMemcpy(dSa.p, Sa.data(), Sa.size() * sizeof(double), cudaMemcpyHostToDevice));
            H->gb.add(dSa.p, n, 0, dS.p, n, 0, H->F1.p, n, n, n, n, 1.0, 0.0);
            H->gb.run(nullptr);
            H2_CUDA(cudaDeviceSynchronize());
        } else {
            // the first r columns of S and S diag(e) (column-major, leading dimension n)
            H->Sr.reserve((size_t)n * H->r);
            H->Sar.reserve((size_t)n * H->r);
            H2_CUDA(cudaMemcpy(H->Sr.p, S.data(), (size_t)n * H->r * sizeof(double), cudaMemcpyHostToDevice));
            H2_CUDA(cudaMemcpy(H->Sar.p, Sa.data(), (size_t)n * H->r * sizeof(double), cudaMemcpyHostToDevice));
        }
        H2_CUDA(cudaMemcpy(H->mask.p, mask_host, N * sizeof(double), cudaMemcpyHostToDevice));
        *ctx_out = H;
        return H2_OK;
    } catch (const Error& e) {
        delete H;
        return e.status;
    } catch (...) {
        delete H;
        return H2_ERR_OOM;
    }
}

int h2_heat2d_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy,
                    h2_stream_t stream) {
    auto* H = static_cast<Heat2d*>(ctx);
    if (!H || n != (int64_t)H->n * H->n || nrhs < 0 || ldx < n || ldy < n) return H2_ERR_INVALID_ARG;
    if (nrhs == 0) return H2_OK;
    if (!X || !Y) return H2_ERR_INVALID_ARG;
    try {
        cudaStream_t s = (cudaStream_t)stream;
        H->W1.reserve((size_t)n * nrhs);
        H->W2.reserve((size_t)n * nrhs);
        if (H->r < H->n) H->W3.reserve((size_t)H->n * H->r * nrhs);
        H2_CUDA(cudaMemcpy2DAsync(H->W1.p, n * sizeof(double), X, ldx * sizeof(double), n * sizeof(double), nrhs,
                                  cudaMemcpyDeviceToDevice, s));
        apply_F(*H, H->W1.p, H->W2.p, H->W3.p, nrhs, s);
        scale_by_kernel<<<grid_for(n * nrhs), NT, 0, s>>>(H->W1.p, H->mask.p, n, n * nrhs, 1.0);
        after_launch("heat_mask");
        apply_F(*H, H->W1.p, H->W2.p, H->W3.p, nrhs, s);
        store_kernel<<<grid_for(n * nrhs), NT, 0, s>>>(H->W1.p, n, nrhs, H->inv_s2, Y, ldy);
        after_launch("heat_store");
        return H2_OK;
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        return H2_ERR_CUDA;
    }
}

void h2_heat2d_destroy(void* ctx) {
    if (ctx) {
        cudaDeviceSynchronize();
        delete static_cast<Heat2d*>(ctx);
    }
}

int h2_dense_op_create(const double* A, int64_t n, int64_t lda, void** ctx_out) {
    if (!ctx_out) return H2_ERR_INVALID_ARG;
    *ctx_out = nullptr;
    if (!A || n < 1 || lda < n || n >= (1 << 22)) return H2_ERR_INVALID_ARG;
    auto* D = new (std::nothrow) DenseOp();
    if (!D) return H2_ERR_OOM;
    D->A = A;
    D->n = n;
    D->lda = lda;
    *ctx_out = D;
    return H2_OK;
}

int h2_dense_op_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy,
                      h2_stream_t stream) {
    auto* D = static_cast<DenseOp*>(ctx);
    if (!D || n != D->n || nrhs < 0 || ldx < n || ldy < n) return H2_ERR_INVALID_ARG;
    if (nrhs == 0) return H2_OK;
    if (!X || !Y) return H2_ERR_INVALID_ARG;
    try {
        D->gb.add(D->A, (int)D->lda, 0, X, (int)ldx, 0, Y, (int)ldy, (int)n, (int)nrhs, (int)n, 1.0, 0.0);
        D->gb.run((cudaStream_t)stream);
        return H2_OK;
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        return H2_ERR_CUDA;
    }
}

void h2_dense_op_destroy(void* ctx) {
    if (ctx) {
        cudaDeviceSynchronize();
        delete static_cast<DenseOp*>(ctx);
    }
}

int h2_lowrank_op_create(const double* Z, int64_t n, int64_t r, int64_t ldz, double scale, void** ctx_out) {
    if (!ctx_out) return H2_ERR_INVALID_ARG;
    *ctx_out = nullptr;
    if (!Z || n < 1 || r < 1 || ldz < n || n >= (1 << 22) || r >= (1 << 22) || !std::isfinite(scale))
        return H2_ERR_INVALID_ARG;
    auto* D = new (std::nothrow) LowRankOp();
    if (!D) return H2_ERR_OOM;
    D->Z = Z;
    D->n = n;
    D->r = r;
    D->ldz = ldz;
    D->scale = scale;
    *ctx_out = D;
    return H2_OK;
}

int h2_lowrank_op_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y, int64_t ldy,
                        h2_stream_t stream) {
    auto* D = static_cast<LowRankOp*>(ctx);
    if (!D || n != D->n || nrhs < 0 || ldx < n || ldy < n) return H2_ERR_INVALID_ARG;
    if (nrhs == 0) return H2_OK;
    if (!X || !Y) return H2_ERR_INVALID_ARG;
    try {
        const cudaStream_t s = (cudaStream_t)stream;
        D->T.reserve((size_t)D->r * nrhs);
        D->gb.add(D->Z, (int)D->ldz, 1, X, (int)ldx, 0, D->T.p, (int)D->r, (int)D->r, (int)nrhs, (int)n, 1.0, 0.0);
        D->gb.run(s);
        D->gb.add(D->Z, (int)D->ldz, 0, D->T.p, (int)D->r, 0, Y, (int)ldy, (int)n, (int)nrhs, (int)D->r, D->scale, 0.0);
        D->gb.run(s);
        return H2_OK;
    } catch (const Error& e) {
        return e.status;
    } catch (...) {
        return H2_ERR_CUDA;
    }
}

void h2_lowrank_op_destroy(void* ctx) {
    if (ctx) {
        cudaDeviceSynchronize();
        delete static_cast<LowRankOp*>(ctx);
    }
}

}  // extern "C"
