// Batched FP64 factorisations of the construction phase.
//
// * panel_qr: Householder QR (LAPACK dlarfg convention) of many tall panels at
//   once, one CTA per panel, producing the explicit orthonormal factor.  Used
//   for the range of each sampled sibling block (Section 3.3: "a QR
//   factorisation of (A Omega)_1 gives the orthogonal column basis"), panel by
//   panel after block Gram-Schmidt projection against the columns found so far.
// * panel_colnorm_max: largest column norm of each panel (the a-posteriori
//   range test of the adaptive sampler).
// * jacobi_eig_trunc: cyclic two-sided Jacobi eigen-decomposition (Jacobi 1846;
//   parallel round-robin ordering of Brent and Luk 1985) of the small Gram
//   matrices of block rows, one CTA per matrix, keeping the leading
//   eigenvectors above a threshold: the truncation step of the recompression
//   (Section 3.2: "truncated to the target accuracy via an SVD").
#include <cfloat>

#include "common.h"

namespace h2 {

namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int MAXC = 16;

// Block-wide sum of V values per thread (V <= MAXC).  Result broadcast in out[0..V).
template <int V>
__device__ void block_sum(double (&v)[V], double* sh /* NW*V */, double* out /* V */) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < V; ++q) {
        double x = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[w * V + q] = x;
    }
    __syncthreads();
    if (threadIdx.x < V) {
        double x = 0.0;
        for (int ww = 0; ww < NW; ++ww) x += sh[ww * V + threadIdx.x];
        out[threadIdx.x] = x;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(NT) panel_qr_kernel(const int64_t* __restrict__ y_off,
                                                       const int64_t* __restrict__ q_off,
                                                       const int* __restrict__ mrows, int c,
                                                       double* __restrict__ Yall, int ldy,
                                                       double* __restrict__ Qall, int ldq) {
    const int m = mrows[blockIdx.x];
    double* Y = Yall + y_off[blockIdx.x];
    double* Q = Qall + q_off[blockIdx.x];
    __shared__ double sh[NW * MAXC];
    __shared__ double res[MAXC];
    __shared__ double tau[MAXC];
    const int nref = min(m, c);
    for (int j = 0; j < nref; ++j) {
        // norm of the part below the diagonal
        double p[1] = {0.0};
        for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
            const double y = Y[i + (int64_t)j * ldy];
            p[0] = fma(y, y, p[0]);
        }
        block_sum<1>(p, sh, res);
        const double xn2 = res[0];
        const double alpha = Y[j + (int64_t)j * ldy];
        double tj = 0.0, scale = 0.0, beta = alpha;
        if (xn2 > 0.0) {
            beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
            tj = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
        }
        __syncthreads();
        if (tj != 0.0)
            for (int i = j + 1 + threadIdx.x; i < m; i += NT) Y[i + (int64_t)j * ldy] *= scale;
        if (threadIdx.x == 0) {
            tau[j] = tj;
            Y[j + (int64_t)j * ldy] = beta;
        }
        __syncthreads();
        if (tj == 0.0) continue;
        // w_k = v^T Y[:, k] for k > j (v_j = 1)
        double w[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) w[k] = 0.0;
        for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
            const double v = Y[i + (int64_t)j * ldy];
#pragma unroll
            for (int k = 0; k < MAXC; ++k)
                if (k > j && k < c) w[k] = fma(v, Y[i + (int64_t)k * ldy], w[k]);
        }
        block_sum<MAXC>(w, sh, res);
        // res[k] += Y[j,k]
        if (threadIdx.x > j && threadIdx.x < c) res[threadIdx.x] += Y[j + (int64_t)threadIdx.x * ldy];
        __syncthreads();
        for (int k = j + 1; k < c; ++k) {
            const double f = tj * res[k];
            if (threadIdx.x == 0) Y[j + (int64_t)k * ldy] -= f;
            for (int i = j + 1 + threadIdx.x; i < m; i += NT)
                Y[i + (int64_t)k * ldy] = fma(-f, Y[i + (int64_t)j * ldy], Y[i + (int64_t)k * ldy]);
        }
        __syncthreads();
    }
    // explicit Q = H_0 ... H_{nref-1} [I; 0]
    for (int e = threadIdx.x; e < m * c; e += NT) {
        const int i = e % m, k = e / m;
        Q[i + (int64_t)k * ldq] = (i == k && k < nref) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int j = nref - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (tj == 0.0) continue;
        double w[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) w[k] = 0.0;
        for (int i = j + 1 + threadIdx.x; i < m; i += NT) {
            const double v = Y[i + (int64_t)j * ldy];
#pragma unroll
            for (int k = 0; k < MAXC; ++k)
                if (k >= j && k < c) w[k] = fma(v, Q[i + (int64_t)k * ldq], w[k]);
        }
        block_sum<MAXC>(w, sh, res);
        if (threadIdx.x >= j && threadIdx.x < c) res[threadIdx.x] += Q[j + (int64_t)threadIdx.x * ldq];
        __syncthreads();
        for (int k = j; k < c; ++k) {
            const double f = tj * res[k];
            if (threadIdx.x == 0) Q[j + (int64_t)k * ldq] -= f;
            for (int i = j + 1 + threadIdx.x; i < m; i += NT)
                Q[i + (int64_t)k * ldq] = fma(-f, Y[i + (int64_t)j * ldy], Q[i + (int64_t)k * ldq]);
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(NT) colnorm_max_kernel(const int64_t* __restrict__ y_off,
                                                          const int* __restrict__ mrows, int c,
                                                          const double* __restrict__ Yall, int ldy,
                                                          double* __restrict__ out) {
    const int m = mrows[blockIdx.x];
    const double* Y = Yall + y_off[blockIdx.x];
    __shared__ double sh[NW * MAXC];
    __shared__ double res[MAXC];
    double p[MAXC];
#pragma unroll
    for (int k = 0; k < MAXC; ++k) p[k] = 0.0;
    for (int i = threadIdx.x; i < m; i += NT)
#pragma unroll
        for (int k = 0; k < MAXC; ++k)
            if (k < c) {
                const double y = Y[i + (int64_t)k * ldy];
                p[k] = fma(y, y, p[k]);
            }
    block_sum<MAXC>(p, sh, res);
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int k = 0; k < c; ++k) mx = fmax(mx, sqrt(res[k]));
        out[blockIdx.x] = mx;
    }
}

// Jacobi eigen-decomposition of one symmetric matrix per CTA held in shared memory.
constexpr int EIG_MAXN = 96;

__global__ void __launch_bounds__(NT) jacobi_kernel(const int64_t* __restrict__ a_off,
                                                     const int* __restrict__ nn,
                                                     const double* __restrict__ Aall,
                                                     const int64_t* __restrict__ u_off,
                                                     double* __restrict__ Uall, int* __restrict__ kout,
                                                     double thr, int kmax, int* __restrict__ cap_flag) {
    extern __shared__ double smem[];
    const int n = nn[blockIdx.x];
    const int np = n + (n & 1);          // even order for the round-robin schedule
    const int ld = np + 1;
    double* A = smem;                     // np x np, ld
    double* V = smem + np * ld;           // np x np, ld
    __shared__ double cs[EIG_MAXN / 2], sn[EIG_MAXN / 2];
    __shared__ int pp[EIG_MAXN / 2], qq[EIG_MAXN / 2];
    __shared__ double red[NW * 2];
    __shared__ int rank[EIG_MAXN];
    __shared__ int kk;
    const double* Ag = Aall + a_off[blockIdx.x];
    for (int e = threadIdx.x; e < np * np; e += NT) {
        const int i = e % np, j = e / np;
        A[i + j * ld] = (i < n && j < n) ? Ag[i + (int64_t)j * n] : 0.0;
        V[i + j * ld] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (n == 0) {
        if (threadIdx.x == 0) kout[blockIdx.x] = 0;
        return;
    }
    const int half = np / 2;
    for (int sweep = 0; sweep < 30; ++sweep) {
        // convergence: off-diagonal mass relative to the whole matrix
        double off = 0.0, tot = 0.0;
        for (int e = threadIdx.x; e < np * np; e += NT) {
            const int i = e % np, j = e / np;
            const double a = A[i + j * ld];
            tot = fma(a, a, tot);
            if (i != j) off = fma(a, a, off);
        }
        double v2[2] = {off, tot};
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                double x = v2[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == 0) red[w * 2 + q] = x;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                double a = 0.0, b = 0.0;
                for (int ww = 0; ww < NW; ++ww) { a += red[ww * 2]; b += red[ww * 2 + 1]; }
                red[0] = a;
                red[1] = b;
            }
            __syncthreads();
        }
        const bool done = !(red[0] > 1e-30 * red[1]);
        __syncthreads();
        if (done) break;
        for (int r = 0; r < np - 1; ++r) {
            // rotation parameters of the round's disjoint pairs
            if (threadIdx.x < half) {
                const int k = threadIdx.x;
                int p, q;
                if (k == 0) { p = np - 1; q = r; }
                else { p = (r + k) % (np - 1); q = (r - k + (np - 1)) % (np - 1); }
                if (p > q) { const int t = p; p = q; q = t; }
                const double apq = A[p + q * ld];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double app = A[p + p * ld], aqq = A[q + q * ld];
                    const double theta = (aqq - app) / (2.0 * apq);
                    const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(fma(theta, theta, 1.0)));
                    c = 1.0 / sqrt(fma(t, t, 1.0));
                    s = t * c;
                }
                pp[k] = p; qq[k] = q; cs[k] = c; sn[k] = s;
            }
            __syncthreads();
            // A <- A J and V <- V J (columns p, q of every pair)
            for (int e = threadIdx.x; e < np * half; e += NT) {
                const int row = e % np, k = e / np;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[row + p * ld], aq = A[row + q * ld];
                A[row + p * ld] = c * ap - s * aq;
                A[row + q * ld] = s * ap + c * aq;
                const double vp = V[row + p * ld], vq = V[row + q * ld];
                V[row + p * ld] = c * vp - s * vq;
                V[row + q * ld] = s * vp + c * vq;
            }
            __syncthreads();
            // A <- J^T A (rows p, q of every pair)
            for (int e = threadIdx.x; e < np * half; e += NT) {
                const int col = e % np, k = e / np;
                const int p = pp[k], q = qq[k];
                const double c = cs[k], s = sn[k];
                const double ap = A[p + col * ld], aq = A[q + col * ld];
                A[p + col * ld] = c * ap - s * aq;
                A[q + col * ld] = s * ap + c * aq;
            }
            __syncthreads();
            if (threadIdx.x < half) {
                const int p = pp[threadIdx.x], q = qq[threadIdx.x];
                A[p + q * ld] = 0.0;
                A[q + p * ld] = 0.0;
            }
            __syncthreads();
        }
    }
    // order eigenvalues descending (ties by index), keep those above thr
    if (threadIdx.x < n) {
        const int i = threadIdx.x;
        const double li = A[i + i * ld];
        int rnk = 0;
        for (int j = 0; j < n; ++j) {
            const double lj = A[j + j * ld];
            if (lj > li || (lj == li && j < i)) ++rnk;
        }
        rank[i] = rnk;
    }
    if (threadIdx.x == 0) {
        int k = 0;
        for (int j = 0; j < n; ++j) k += (A[j + j * ld] > thr) ? 1 : 0;
        if (k > kmax) {
            atomicExch(cap_flag, 1);
            k = kmax;
        }
        kk = k;
        kout[blockIdx.x] = k;
    }
    __syncthreads();
    double* U = Uall + u_off[blockIdx.x];
    const int k = kk;
    for (int e = threadIdx.x; e < n * n; e += NT) {
        const int row = e % n, i = e / n;
        const int rnk = rank[i];
        if (rnk < k) U[row + (int64_t)rnk * n] = V[row + i * ld];
    }
}

}  // namespace

void panel_qr(int count, const int64_t* d_y_off, const int64_t* d_q_off, const int* d_m, int c,
              double* Y, int ldy, double* Q, int ldq, cudaStream_t s) {
    if (count <= 0) return;
    if (c < 1 || c > MAXC) fail(H2_ERR_INVALID_ARG, "panel_qr: panel width out of range");
    panel_qr_kernel<<<count, NT, 0, s>>>(d_y_off, d_q_off, d_m, c, Y, ldy, Q, ldq);
    after_launch("panel_qr");
}

void panel_colnorm_max(int count, const int64_t* d_y_off, const int* d_m, int c, const double* Y,
                       int ldy, double* out, cudaStream_t s) {
    if (count <= 0) return;
    if (c < 1 || c > MAXC) fail(H2_ERR_INVALID_ARG, "colnorm: panel width out of range");
    colnorm_max_kernel<<<count, NT, 0, s>>>(d_y_off, d_m, c, Y, ldy, out);
    after_launch("colnorm_max");
}

void jacobi_eig_trunc(int count, const int64_t* d_a_off, const int* d_n, const double* A,
                      const int64_t* d_u_off, double* U, int* d_k_out, double thr, int kmax,
                      int* d_cap_flag, cudaStream_t s) {
    if (count <= 0) return;
    const int np = EIG_MAXN;
    const size_t smem = 2 * (size_t)np * (np + 1) * sizeof(double);
    static bool attr_set = false;
    if (!attr_set) {
        H2_CUDA(cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_set = true;
    }
    jacobi_kernel<<<count, NT, smem, s>>>(d_a_off, d_n, A, d_u_off, U, d_k_out, thr, kmax, d_cap_flag);
    after_launch("jacobi_eig");
}

int eig_max_order() { return EIG_MAXN; }

}  // namespace h2
