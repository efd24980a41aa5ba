// Batched FP64 factorisations of the construction phase.
//
// * panel_qr: Householder QR (LAPACK dlarfg convention) of many tall panels at
//   once, one CTA per panel, producing the explicit orthonormal factor.  Used
//   for the range of each sampled sibling block (Section 3.3: "a QR
//   factorisation of (A Omega)_1 gives the orthogonal column basis"), panel by
//   panel after block Gram-Schmidt projection against the columns found so far.
// * panel_colnorm_max: largest column norm of each panel (the a-posteriori
//   range test of the adaptive sampler).
// * align_signs: the sign convention of the range bases (non-negative diagonal
//   of R in Y = QR).
#include <cfloat>

#include <mutex>

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

// ---------------------------------------------------------------------------
// Tall-skinny QR (TSQR) of panels in shared memory.
//
// Each panel (m rows x c <= 16 columns) is split into row chunks; every chunk is
// factorised by Householder QR in shared memory (stage 1), the stacked c x c R
// factors of a panel are factorised once more (stage 2), and each chunk's
// orthonormal factor is multiplied by its c x c block of the second factor
// (stage 3): Q = diag(Q_1..Q_k) Q_s.  Householder vectors follow dlarfg; the
// explicit factor is formed in place backwards as in dorg2r.
// ---------------------------------------------------------------------------

// Householder QR in place of the h x c matrix A (shared memory, leading dimension h),
// h >= c.  R in the upper triangle, reflectors below the diagonal, tau[0..c).
__device__ void house_qr_smem(double* A, int h, int c, double* tau, double* sh, double* res) {
    for (int j = 0; j < c; ++j) {
        double p[1] = {0.0};
        for (int i = j + 1 + threadIdx.x; i < h; i += NT) p[0] = fma(A[i + j * h], A[i + j * h], p[0]);
        block_sum<1>(p, sh, res);
        const double xn2 = res[0];
        const double alpha = A[j + j * h];
        double tj = 0.0, scale = 0.0, beta = alpha;
        if (xn2 > 0.0) {
            beta = -copysign(sqrt(fma(alpha, alpha, xn2)), alpha);
            tj = (beta - alpha) / beta;
            scale = 1.0 / (alpha - beta);
        }
        __syncthreads();
        if (tj != 0.0)
            for (int i = j + 1 + threadIdx.x; i < h; i += NT) A[i + j * h] *= scale;
        if (threadIdx.x == 0) {
            tau[j] = tj;
            A[j + j * h] = beta;
        }
        __syncthreads();
        if (tj == 0.0) continue;
        double w[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) w[k] = 0.0;
        for (int i = j + 1 + threadIdx.x; i < h; i += NT) {
            const double v = A[i + j * h];
#pragma unroll
            for (int k = 0; k < MAXC; ++k)
                if (k > j && k < c) w[k] = fma(v, A[i + k * h], w[k]);
        }
        block_sum<MAXC>(w, sh, res);
        if (threadIdx.x > j && threadIdx.x < c) res[threadIdx.x] += A[j + threadIdx.x * h];
        __syncthreads();
        for (int e = threadIdx.x; e < (h - j) * (c - j - 1); e += NT) {
            const int i = j + e % (h - j), k = j + 1 + e / (h - j);
            const double f = tj * res[k];
            const double v = (i == j) ? 1.0 : A[i + j * h];
            A[i + k * h] = fma(-f, v, A[i + k * h]);
        }
        __syncthreads();
    }
}

// Overwrites the reflectors of house_qr_smem with the explicit h x c orthonormal factor.
__device__ void house_orgqr_smem(double* A, int h, int c, const double* tau, double* sh, double* res) {
    for (int j = c - 1; j >= 0; --j) {
        const double tj = tau[j];
        if (j < c - 1) {
            // apply H_j to A[j:h, j+1:c] with v = [1; A[j+1:h, j]]
            double w[MAXC];
#pragma unroll
            for (int k = 0; k < MAXC; ++k) w[k] = 0.0;
            for (int i = j + 1 + threadIdx.x; i < h; i += NT) {
                const double v = A[i + j * h];
#pragma unroll
                for (int k = 0; k < MAXC; ++k)
                    if (k > j && k < c) w[k] = fma(v, A[i + k * h], w[k]);
            }
            block_sum<MAXC>(w, sh, res);
            if (threadIdx.x > j && threadIdx.x < c) res[threadIdx.x] += A[j + threadIdx.x * h];
            __syncthreads();
            for (int e = threadIdx.x; e < (h - j) * (c - j - 1); e += NT) {
                const int i = j + e % (h - j), k = j + 1 + e / (h - j);
                const double v = (i == j) ? 1.0 : A[i + j * h];
                A[i + k * h] = fma(-tj * res[k], v, A[i + k * h]);
            }
            __syncthreads();
        }
        for (int i = j + 1 + threadIdx.x; i < h; i += NT) A[i + j * h] *= -tj;
        for (int i = threadIdx.x; i < j; i += NT) A[i + j * h] = 0.0;
        if (threadIdx.x == 0) A[j + j * h] = 1.0 - tj;
        __syncthreads();
    }
}

// stage 1: one chunk per CTA.  d = {src offset in Y, dst offset in Q, rows, R offset (-1: single chunk)}
__global__ void __launch_bounds__(NT) tsqr_chunk_kernel(const TsqrChunk* __restrict__ chunks, int c,
                                                         const double* __restrict__ Y, int ldy,
                                                         double* __restrict__ Q, int ldq, double* __restrict__ Rbuf) {
    extern __shared__ double A[];
    __shared__ double sh[NW * MAXC];
    __shared__ double res[MAXC];
    __shared__ double tau[MAXC];
    const TsqrChunk d = chunks[blockIdx.x];
    const int h = d.rows;
    for (int e = threadIdx.x; e < h * c; e += NT) {
        const int i = e % h, k = e / h;
        A[i + k * h] = Y[d.y_off + i + (int64_t)k * ldy];
    }
    __syncthreads();
    house_qr_smem(A, h, c, tau, sh, res);
    if (d.r_off >= 0)
        for (int e = threadIdx.x; e < c * c; e += NT) {
            const int i = e % c, k = e / c;
            Rbuf[d.r_off + i + k * c] = (i <= k) ? A[i + k * h] : 0.0;
        }
    __syncthreads();
    house_orgqr_smem(A, h, c, tau, sh, res);
    for (int e = threadIdx.x; e < h * c; e += NT) {
        const int i = e % h, k = e / h;
        Q[d.q_off + i + (int64_t)k * ldq] = A[i + k * h];
    }
}

// stage 2: the stacked R factors of one panel per CTA -> Qs (nchunk*c x c, leading dimension nchunk*c);
// with roots[].w >= 0 the combined R factor also goes to Rout block w (the next level of the tree)
__global__ void __launch_bounds__(NT) tsqr_root_kernel(const int4* __restrict__ roots, int c,
                                                        const double* __restrict__ Rbuf, double* __restrict__ Qs,
                                                        double* __restrict__ Rout) {
    extern __shared__ double A[];
    __shared__ double sh[NW * MAXC];
    __shared__ double res[MAXC];
    __shared__ double tau[MAXC];
    const int4 r = roots[blockIdx.x];   // x: first R offset / (c*c) chunk index, y: nchunk, z: Qs offset (in c*c units)
    const int nch = r.y;
    const int h = nch * c;
    const double* R = Rbuf + (int64_t)r.x * c * c;
    for (int e = threadIdx.x; e < h * c; e += NT) {
        const int i = e % h, k = e / h;
        const int ch = i / c, ii = i % c;
        A[i + k * h] = R[(int64_t)ch * c * c + ii + k * c];
    }
    __syncthreads();
    house_qr_smem(A, h, c, tau, sh, res);
    if (r.w >= 0)
        for (int e = threadIdx.x; e < c * c; e += NT) {
            const int i = e % c, k = e / c;
            Rout[(int64_t)r.w * c * c + i + k * c] = (i <= k) ? A[i + k * h] : 0.0;
        }
    __syncthreads();
    house_orgqr_smem(A, h, c, tau, sh, res);
    double* out = Qs + (int64_t)r.z * c * c;
    for (int e = threadIdx.x; e < h * c; e += NT) out[e] = A[e];
}

// stage 3: Q_chunk <- Q_chunk * Qs[chunk block]  (in place, row by row)
__global__ void __launch_bounds__(NT) tsqr_apply_kernel(const TsqrChunk* __restrict__ chunks, int c,
                                                         double* __restrict__ Q, int ldq, const double* __restrict__ Qs) {
    __shared__ double B[MAXC * MAXC];
    const TsqrChunk d = chunks[blockIdx.x];
    // qs position: Qs block rows [kc*c, kc*c+c) of the panel's Qs with leading dimension ldqs
    const int64_t base = d.qs_off;
    const int ldqs = d.ldqs;
    // the whole MAXC x MAXC tile is written (zeros outside c x c): the product below runs over
    // all MAXC rows, and stale shared memory times a zero factor could be NaN
    for (int e = threadIdx.x; e < MAXC * MAXC; e += NT) {
        const int i = e % MAXC, k = e / MAXC;
        B[e] = (i < c && k < c) ? Qs[base + i + (int64_t)k * ldqs] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < d.rows; i += NT) {
        double q[MAXC], o[MAXC];
#pragma unroll
        for (int k = 0; k < MAXC; ++k) q[k] = (k < c) ? Q[d.q_off + i + (int64_t)k * ldq] : 0.0;
#pragma unroll
        for (int k = 0; k < MAXC; ++k) {
            double acc = 0.0;
#pragma unroll
            for (int j = 0; j < MAXC; ++j) acc = fma(q[j], B[j + k * MAXC], acc);
            o[k] = acc;
        }
#pragma unroll
        for (int k = 0; k < MAXC; ++k)
            if (k < c) Q[d.q_off + i + (int64_t)k * ldq] = o[k];
    }
}

}  // namespace

void tsqr_panels(int count, const int64_t* y_off, const int64_t* q_off, const int* m, int c, double* Y, int ldy,
                 double* Q, int ldq, TsqrWork& w, cudaStream_t s) {
    if (count <= 0) return;
    if (c < 1 || c > MAXC) fail(H2_ERR_INVALID_ARG, "tsqr: panel width out of range");
    // level 1: chunks of at most kTsqrMaxRows rows, one R each; groups of at most kTsqrMaxChunks
    // chunks combine their stacked R factors in one root.  A panel with more than one group
    // (taller than kTsqrMaxChunks * kTsqrMaxRows rows) adds level 2: a root over the groups' R
    // factors, applied to every chunk after its group's factor.
    std::vector<TsqrChunk> chunks, multi, multi2;
    std::vector<int4> roots, roots2;
    int64_t rcount = 0, qscount = 0, r2count = 0, qs2count = 0;
    int max_h = 0, max_root = 0;
    for (int p = 0; p < count; ++p) {
        if (m[p] <= c) fail(H2_ERR_INVALID_ARG, "tsqr: panel must have more rows than columns");
        int nch = std::max(1, std::min(kTsqrMaxChunks, m[p] / kTsqrChunk));
        if ((m[p] + nch - 1) / nch > kTsqrMaxRows) nch = (m[p] + kTsqrMaxRows - 1) / kTsqrMaxRows;   // two levels
        const int ngroups = (nch + kTsqrMaxChunks - 1) / kTsqrMaxChunks;
        if (ngroups > kTsqrMaxChunks) fail(H2_ERR_INVALID_ARG, "tsqr: panel too tall");
        const int64_t r2base = r2count, qs2base = qs2count;
        int row = 0, k = 0;
        for (int gi = 0; gi < ngroups; ++gi) {
            // chunks spread evenly over the groups (every group of a two-level panel has > 1 chunk)
            const int nchg = nch / ngroups + (gi < nch % ngroups ? 1 : 0);
            const int64_t r0 = rcount, qs0 = qscount;
            for (int kk = 0; kk < nchg; ++kk, ++k) {
                const int h = m[p] / nch + (k < m[p] % nch ? 1 : 0);
                TsqrChunk d{y_off[p] + row, q_off[p] + row, h, nch > 1 ? (r0 + kk) * c * c : -1,
                            (qs0 * c * c) + (int64_t)kk * c, nchg * c};
                chunks.push_back(d);
                if (nchg > 1) multi.push_back(d);
                if (ngroups > 1)
                    multi2.push_back(TsqrChunk{0, q_off[p] + row, h, -1, qs2base * c * c + (int64_t)gi * c, ngroups * c});
                max_h = std::max(max_h, h);
                row += h;
            }
            if (nchg > 1) {
                roots.push_back(make_int4((int)r0, nchg, (int)qs0, ngroups > 1 ? (int)(r2base + gi) : -1));
                max_root = std::max(max_root, nchg * c);
            } else if (ngroups > 1) {
                fail(H2_ERR_INVALID_ARG, "tsqr: single-chunk group in a two-level panel");
            }
            if (nchg > 1) {
                rcount += nchg;
                qscount += nchg;
            }
        }
        if (ngroups > 1) {
            roots2.push_back(make_int4((int)r2base, ngroups, (int)qs2base, -1));
            max_root = std::max(max_root, ngroups * c);
            r2count += ngroups;
            qs2count += ngroups;
        }
        if (max_h > kTsqrMaxRows) fail(H2_ERR_INVALID_ARG, "tsqr: panel too tall");
    }
    upload(w.d_chunks, chunks, s, w.st_chunks);
    w.Rbuf.reserve((size_t)std::max<int64_t>(rcount * c * c, 1));
    w.Qs.reserve((size_t)std::max<int64_t>(qscount * c * c, 1));
    const size_t smem1 = (size_t)max_h * c * sizeof(double);
    static std::once_flag attr;
    std::call_once(attr, [&] {
        const int mx = kTsqrMaxRows * MAXC * (int)sizeof(double);
        H2_CUDA(cudaFuncSetAttribute(tsqr_chunk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        H2_CUDA(cudaFuncSetAttribute(tsqr_root_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    });
    tsqr_chunk_kernel<<<(unsigned)chunks.size(), NT, smem1, s>>>(w.d_chunks.p, c, Y, ldy, Q, ldq, w.Rbuf.p);
    after_launch("tsqr_chunk");
    if (!roots.empty()) {
        if (!roots2.empty()) w.R2.reserve((size_t)(r2count * c * c));
        upload(w.d_roots, roots, s, w.st_roots);
        upload(w.d_multi, multi, s, w.st_multi);
        tsqr_root_kernel<<<(unsigned)roots.size(), NT, (size_t)max_root * c * sizeof(double), s>>>(
            w.d_roots.p, c, w.Rbuf.p, w.Qs.p, w.R2.p);
        after_launch("tsqr_root");
        tsqr_apply_kernel<<<(unsigned)multi.size(), NT, 0, s>>>(w.d_multi.p, c, Q, ldq, w.Qs.p);
        after_launch("tsqr_apply");
    }
    if (!roots2.empty()) {
        w.Qs2.reserve((size_t)(qs2count * c * c));
        upload(w.d_roots2, roots2, s, w.st_roots2);
        upload(w.d_multi2, multi2, s, w.st_multi2);
        tsqr_root_kernel<<<(unsigned)roots2.size(), NT, (size_t)max_root * c * sizeof(double), s>>>(
            w.d_roots2.p, c, w.R2.p, w.Qs2.p, nullptr);
        after_launch("tsqr_root");
        tsqr_apply_kernel<<<(unsigned)multi2.size(), NT, 0, s>>>(w.d_multi2.p, c, Q, ldq, w.Qs2.p);
        after_launch("tsqr_apply");
    }
}

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

namespace {

// Column j of Q is negated when q_j^T y_j < 0 (one CTA per column).
__global__ void __launch_bounds__(NT) align_signs_kernel(const SignItem* __restrict__ items, double* __restrict__ Q,
                                                         const double* __restrict__ Y) {
    __shared__ double sh[NW];
    __shared__ double res[1];
    const SignItem it = items[blockIdx.x];
    double p[1] = {0.0};
    for (int i = threadIdx.x; i < it.rows; i += NT) p[0] = fma(Q[it.q_off + i], Y[it.y_off + i], p[0]);
    block_sum<1>(p, sh, res);
    if (res[0] < 0.0)
        for (int i = threadIdx.x; i < it.rows; i += NT) Q[it.q_off + i] = -Q[it.q_off + i];
}

}  // namespace

void align_signs(int count, const SignItem* d_items, double* Q, const double* Y, cudaStream_t s) {
    if (count <= 0) return;
    align_signs_kernel<<<count, NT, 0, s>>>(d_items, Q, Y);
    after_launch("align_signs");
}



namespace {

constexpr int CHOL_NT = 1024;

// Right-looking Cholesky of the symmetric positive semidefinite n x n matrix A (column-major,
// lower triangle used and overwritten) into the lower-triangular C (zero above the diagonal).
// A pivot at or below n 2^-52 max(diag A) is rounding noise of a zero eigenvalue: its column
// of C stays zero and the elimination continues.  One CTA; every branch is uniform.
__global__ void __launch_bounds__(CHOL_NT) psd_cholesky_kernel(double* __restrict__ A, int n, double* __restrict__ C) {
    __shared__ double red[CHOL_NT / 32];
    __shared__ double s_drop;
    const int tid = threadIdx.x;
    double mx = 0.0;
    for (int i = tid; i < n; i += CHOL_NT) mx = fmax(mx, A[i + (int64_t)i * n]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((tid & 31) == 0) red[tid >> 5] = mx;
    for (int64_t e = tid; e < (int64_t)n * n; e += CHOL_NT) C[e] = 0.0;
    __syncthreads();
    if (tid == 0) {
        double m = 0.0;
        for (int w = 0; w < CHOL_NT / 32; ++w) m = fmax(m, red[w]);
        s_drop = (double)n * 0x1p-52 * m;
    }
    __syncthreads();
    const double drop = s_drop;
    for (int j = 0; j < n; ++j) {
        const double d = A[j + (int64_t)j * n];
        if (!(d > drop)) continue;   // the same value in every thread: uniform
        const double cjj = sqrt(d);
        for (int i = j + tid; i < n; i += CHOL_NT) C[i + (int64_t)j * n] = (i == j) ? cjj : A[i + (int64_t)j * n] / cjj;
        __syncthreads();
        const int m = n - j - 1;
        for (int64_t e = tid; e < (int64_t)m * m; e += CHOL_NT) {
            const int i = j + 1 + (int)(e % m), k = j + 1 + (int)(e / m);
            if (k <= i) A[i + (int64_t)k * n] -= C[i + (int64_t)j * n] * C[k + (int64_t)j * n];
        }
        __syncthreads();
    }
}

}  // namespace

void psd_cholesky(double* A, int n, double* C, cudaStream_t s) {
    if (n <= 0) return;
    psd_cholesky_kernel<<<1, CHOL_NT, 0, s>>>(A, n, C);
    after_launch("psd_cholesky");
}

}  // namespace h2
