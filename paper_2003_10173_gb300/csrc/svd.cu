// Batched R factors of stacked row blocks and truncated SVDs of block-row factors.
//
// The recompression of Section 3.2 needs, for every box, (i) the R factor of the
// column side of its far block row (the QR downsweep) and (ii) the leading left
// singular vectors of the weighted block-row factor W = [P_lp R_lp^T]_lp (the SVD
// upsweep).  Both are computed here without forming a Gram matrix, so that
// singular values are resolved to about eps * sigma_max instead of
// sqrt(eps) * sigma_max:
//
//  * stacked_r: Householder QR (LAPACK dlarfg convention) of a matrix given as a
//    stack of row blocks.  One CTA per matrix streams its rows through shared
//    memory in chunks under the running c x c triangle R (the incremental form of
//    a tall-skinny QR: every chunk is annihilated against R by c reflectors that
//    touch one row of R and the chunk).  Matrices taller than a few thousand rows
//    are first split over several CTAs whose R factors are stacked once more.
//  * stacked_svd_trunc: the same QR of W^T (W is m x sum(q), m <= 96), then the
//    one-sided Jacobi method (Hestenes 1958; round-robin ordering of Brent and
//    Luk 1985) on the columns of the m x m lower triangle R^T (W = R^T Q^T): at
//    convergence R^T V = U Sigma with orthogonal columns, whose normalised values
//    are the left singular vectors of W.  Rotating R^T rather than R converges
//    in about ten sweeps on the graded block rows (columns of R are not graded)
//    and needs no accumulated rotation matrix.  The vectors with singular value
//    above the threshold (at most kmax) are kept, sorted by descending value.
#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>

#include "common.h"

namespace h2 {

namespace {

constexpr int SQ_NT = 256;
constexpr int SQ_NW = SQ_NT / 32;
constexpr int QR_NT = 256;         // threads of the stacked QR kernel
constexpr int QR_NW = QR_NT / 32;
constexpr int SVD_MAXC = 96;
constexpr int kSplitRows = 4096;   // a single matrix taller than this is split over several CTAs
constexpr size_t kSmemCap = 200 * 1024;

constexpr int kSmemMaxC = 144;     // widest matrix of stacked_r (its working matrix in shared memory)

// rows of a chunk streamed under R: shared memory holds (c + chunk) x c doubles
__host__ __device__ inline int chunk_rows(int c) {
    return c <= 32 ? 224 : (c <= 48 ? 112 : (c <= 96 ? 64 : (c <= 128 ? 32 : 16)));
}
constexpr int kMaxChunk = 224;   // the largest chunk_rows
constexpr int kStackClasses = StackWork::kClasses;   // width classes of a stacked_r pass
// chunk height of the SVD kernel: fixed, so that its shared memory grows with c (one launch per level)
constexpr int kSvdChunk = 64;
// leading dimension of the working matrix [R; chunk]: odd, so that the columns of a warp's
// column pairs fall in different shared-memory banks
__host__ __device__ inline int work_ld(int c, int ch) { return (c + ch) | 1; }
__host__ __device__ inline int work_ld(int c) { return work_ld(c, chunk_rows(c)); }

// Reflector j (LAPACK dlarfg convention) from alpha = R[j, j] and x2 = ||y_j||^2: tau[j], the
// scale sc_j = 1 / (alpha - beta) of the chunk part (slot j & 1 of sc), and R[j, j] = beta.
__device__ inline void householder(double* A, int lda, int j, double x2, double* tau, double* sc) {
    const double alpha = A[j + (int64_t)j * lda];
    double tj = 0.0, scj = 0.0, beta = alpha;
    if (x2 > 0.0) {
        beta = -copysign(sqrt(fma(alpha, alpha, x2)), alpha);
        tj = (beta - alpha) / beta;
        scj = 1.0 / (alpha - beta);
    }
    tau[j] = tj;
    sc[j & 1] = scj;
    A[j + (int64_t)j * lda] = beta;
}

// R factor (upper c x c, rows 0..c-1 of A) of the stacked row blocks segs[b..e).  The rows
// stream through shared memory in chunks of up to chunk_rows(c) rows, taken in the order of
// their first possibly nonzero column f: level 0 holds every row of a dense segment and row 0 of
// each triangular one (RowSeg::tri), level f > 0 row f of each triangular segment.  A chunk
// whose rows all start at column f0 or later skips reflectors 0..f0-1 (they are the identity on
// it), and each reflector it applies meets rows that are nonzero in its column; a stack of
// triangles (the downsweep's R factors) so costs about half the reflector steps of a
// segment-by-segment order, each with full rows.  Entry state of A is irrelevant; every
// thread returns after a barrier with R complete.
template <int NT>
__device__ void stacked_qr(double* A, int lda, int c, int ch, const RowSeg* __restrict__ segs, int b, int e,
                           double* tau) {
    __shared__ const double* rp[kMaxChunk];
    __shared__ int rld[kMaxChunk];
    __shared__ int nact[kSmemMaxC + 1];   // chunk rows whose first nonzero column is <= j
    __shared__ int hs, j0s;
    __shared__ int wf, ws, wo, anytri;    // walk over the stack: level, segment, row offset
    __shared__ double scl[2];           // sc_j of the current and of the next reflector
    for (int x = threadIdx.x; x < c * c; x += NT) A[x % c + (int64_t)(x / c) * lda] = 0.0;
    if (threadIdx.x == 0) {
        int any = 0;
        for (int s = b; s < e; ++s) any |= segs[s].tri;
        anytri = any;
        wf = 0;
        ws = b;
        wo = 0;
    }
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {   // the rows of the next chunk, in nondecreasing f
            int h = 0, f = wf, s = ws, o = wo;
            for (int jj = 0; jj <= c; ++jj) nact[jj] = 0;
            while (h < ch && f < c) {
                if (s >= e) {   // next level (none after level 0 without triangular segments)
                    f = anytri ? f + 1 : c;
                    s = b;
                    o = 0;
                    continue;
                }
                const RowSeg sg = segs[s];
                if (sg.tri) {
                    if (f < sg.rows) {
                        rp[h] = sg.p + f;
                        rld[h] = sg.ld;
                        ++nact[f];
                        ++h;
                    }
                    ++s;
                } else if (f == 0) {
                    const int take = min(ch - h, sg.rows - o);
                    for (int i = 0; i < take; ++i) {
                        rp[h + i] = sg.p + o + i;
                        rld[h + i] = sg.ld;
                    }
                    nact[0] += take;
                    h += take;
                    o += take;
                    if (o >= sg.rows) {
                        ++s;
                        o = 0;
                    }
                } else {
                    ++s;
                }
            }
            wf = f;
            ws = s;
            wo = o;
            for (int jj = 1; jj <= c; ++jj) nact[jj] += nact[jj - 1];
            int j0 = 0;
            while (j0 < c && nact[j0] == 0) ++j0;
            j0s = j0;
            hs = h;
        }
        __syncthreads();
        const int h = hs;
        if (h == 0) break;
        const int j0 = j0s;
        for (int x = threadIdx.x; x < h * c; x += NT) {
            const int i = x % h, k = x / h;
            A[c + i + (int64_t)k * lda] = rp[i][(int64_t)k * rld[i]];
        }
        __syncthreads();
        // Column-by-column elimination of the chunk under R.  Reflector j is v = [e_j; sc_j y_j]
        // (y_j: the chunk part of column j, left unscaled), so for every column k > j
        //   w = R[j, k] + sc_j (y_j . y_k),  R[j, k] -= tau_j w,  y_k -= tau_j sc_j w y_j.
        // A group of ns consecutive lanes (ns a power of two <= 8) works on column k = j + 1 + t / ns,
        // lane t % ns on the rows t % ns, t % ns + ns, ...; the group's partial dot products meet by
        // warp shuffles.  Reflector j + 1 only needs y_{j+1} after reflector j and R[j+1, j+1]
        // (which reflector j does not touch), and the group of column j + 1 is the first lanes of
        // warp 0: it reduces the squared norm of y_{j+1} while updating it, and lane 0 forms
        // reflector j + 1 while the other warps still apply reflector j (look-ahead).  A column
        // costs two block barriers, and the serial reflector stays off the critical path.
        if (threadIdx.x < 32 && j0 < c) {   // the chunk's first reflector
            const int h0 = nact[j0];
            const double* y0 = A + c + (int64_t)j0 * lda;
            double x0 = 0.0, x1 = 0.0;
            int r = threadIdx.x;
            for (; r + 32 < h0; r += 64) {
                x0 = fma(y0[r], y0[r], x0);
                x1 = fma(y0[r + 32], y0[r + 32], x1);
            }
            if (r < h0) x0 = fma(y0[r], y0[r], x0);
            double x2 = x0 + x1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            if (threadIdx.x == 0) householder(A, lda, j0, x2, tau, scl);
        }
        __syncthreads();
        for (int j = j0; j < c; ++j) {
            // rows below ha are zero in column j (first nonzero column > j): reflector j and its
            // updates skip them; the update of column j + 1 covers hc rows for its norm
            const int ha = nact[j];
            const int hc = j + 1 < c ? nact[j + 1] : ha;
            const int nk = c - j - 1;
            const int m = nk > 0 ? min(8, NT / nk) : 1;
            const int ns = m >= 8 ? 8 : (m >= 4 ? 4 : (m >= 2 ? 2 : 1));
            const int t = threadIdx.x;
            const int ci = t / ns, sl = t - ci * ns;
            const bool act = ci < nk;
            const double* yj = A + c + (int64_t)j * lda;
            double* yk = A + c + (int64_t)(act ? j + 1 + ci : j) * lda;
            double d = 0.0;
            if (act) {   // four independent partial sums per lane
                double d1 = 0.0, d2 = 0.0, d3 = 0.0;
                int r = sl;
                for (; r + 3 * ns < ha; r += 4 * ns) {
                    d = fma(yj[r], yk[r], d);
                    d1 = fma(yj[r + ns], yk[r + ns], d1);
                    d2 = fma(yj[r + 2 * ns], yk[r + 2 * ns], d2);
                    d3 = fma(yj[r + 3 * ns], yk[r + 3 * ns], d3);
                }
                for (; r < ha; r += ns) d = fma(yj[r], yk[r], d);
                d = (d + d1) + (d2 + d3);
            }
            for (int o = ns >> 1; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
            __syncthreads();
            if (nk > 0) {
                const double tj = tau[j], scj = scl[j & 1];
                double g = 0.0;
                if (act && sl == 0 && tj != 0.0) {   // the group's first lane updates R[j, k]
                    double* rjk = A + j + (int64_t)(j + 1 + ci) * lda;
                    const double w = fma(scj, d, *rjk);
                    const double f = tj * w;
                    *rjk -= f;
                    g = f * scj;
                }
                g = __shfl_sync(0xffffffffu, g, (t & 31) & ~(ns - 1));
                double xn = 0.0;
                if (act && ci == 0) {   // y_{j+1}: rows ha..hc-1 have y_j = 0 (exact), only the norm needs them
                    double x1 = 0.0;
                    int r = sl;
                    for (; r + ns < hc; r += 2 * ns) {
                        const double y0 = fma(-g, yj[r], yk[r]);
                        const double y1 = fma(-g, yj[r + ns], yk[r + ns]);
                        yk[r] = y0;
                        yk[r + ns] = y1;
                        xn = fma(y0, y0, xn);
                        x1 = fma(y1, y1, x1);
                    }
                    if (r < hc) {
                        const double y0 = fma(-g, yj[r], yk[r]);
                        yk[r] = y0;
                        xn = fma(y0, y0, xn);
                    }
                    xn += x1;
                } else if (act && tj != 0.0) {
#pragma unroll 4
                    for (int r = sl; r < ha; r += ns) yk[r] = fma(-g, yj[r], yk[r]);
                }
                if (t < 32) {   // warp 0: the norm of y_{j+1} over its group, then reflector j + 1
                    for (int o = ns >> 1; o > 0; o >>= 1) xn += __shfl_xor_sync(0xffffffffu, xn, o);
                    if (t == 0) householder(A, lda, j + 1, xn, tau, scl);
                }
            }
            __syncthreads();
        }
    }
}

// Householder QR with column pivoting (largest remaining column norm first) of the c x c
// upper triangle R in rows 0..c-1 of A, in place: R P = Q3 R3.  perm[j] receives the column of
// R that became column j.  Used before the one-sided Jacobi method: on the pivoted triangle it
// needs about a third of the sweeps.
__device__ void pivoted_qr(double* A, int lda, int c, int* perm, double* cn, double* tau) {
    __shared__ int piv;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < c; k += SQ_NT) perm[k] = k;
    __syncthreads();
    for (int j = 0; j < c; ++j) {
        // norms of the trailing parts of columns j..c-1 (rows j..c-1), one warp per column
        for (int k = j + warp; k < c; k += SQ_NW) {
            double x = 0.0;
            for (int i = j + lane; i < c; i += 32) {
                const double a = A[i + (int64_t)k * lda];
                x = fma(a, a, x);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) cn[k] = x;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int p = j;
            for (int k = j + 1; k < c; ++k)
                if (cn[k] > cn[p]) p = k;
            piv = p;
            const int t = perm[j];
            perm[j] = perm[p];
            perm[p] = t;
        }
        __syncthreads();
        const int p = piv;
        if (p != j)
            for (int i = threadIdx.x; i < c; i += SQ_NT) {
                const double t = A[i + (int64_t)j * lda];
                A[i + (int64_t)j * lda] = A[i + (int64_t)p * lda];
                A[i + (int64_t)p * lda] = t;
            }
        __syncthreads();
        // reflector of column j on rows j..c-1 (one warp), then its application to columns > j
        if (warp == 0) {
            double x2 = 0.0;
            for (int i = j + 1 + lane; i < c; i += 32) {
                const double y = A[i + (int64_t)j * lda];
                x2 = fma(y, y, x2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x2 += __shfl_xor_sync(0xffffffffu, x2, o);
            const double alpha = A[j + (int64_t)j * lda];
            double tj = 0.0, scale = 0.0, beta = alpha;
            if (x2 > 0.0) {
                beta = -copysign(sqrt(fma(alpha, alpha, x2)), alpha);
                tj = (beta - alpha) / beta;
                scale = 1.0 / (alpha - beta);
            }
            if (tj != 0.0)
                for (int i = j + 1 + lane; i < c; i += 32) A[i + (int64_t)j * lda] *= scale;
            __syncwarp();
            if (lane == 0) {
                tau[j] = tj;
                A[j + (int64_t)j * lda] = beta;
            }
        }
        __syncthreads();
        const double tj = tau[j];
        if (tj != 0.0)
            for (int k = j + 1 + warp; k < c; k += SQ_NW) {
                double w = 0.0;
                for (int i = j + 1 + lane; i < c; i += 32) w = fma(A[i + (int64_t)j * lda], A[i + (int64_t)k * lda], w);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
                w += A[j + (int64_t)k * lda];
                const double f = tj * w;
                for (int i = j + 1 + lane; i < c; i += 32)
                    A[i + (int64_t)k * lda] = fma(-f, A[i + (int64_t)j * lda], A[i + (int64_t)k * lda]);
                __syncwarp();
                if (lane == 0) A[j + (int64_t)k * lda] -= f;
            }
        __syncthreads();
    }
    // the reflectors below the diagonal are not needed: only R3 is used
    for (int x = threadIdx.x; x < c * c; x += SQ_NT) {
        const int i = x % c, k = x / c;
        if (i > k) A[i + (int64_t)k * lda] = 0.0;
    }
    __syncthreads();
}

// One CTA per job.  A stack with at least c rows gives its c x c upper triangle as computed.
// With fewer rows the triangle holds the rank of the stack in the rows of the columns where it
// appears (leading zero columns leave other rows zero), so the output is compacted: the
// min(c, rows) rows of largest norm are written first (R^T R, the only use of R, does not depend
// on the order of its rows) and the remaining rows -- zero in exact arithmetic -- as zeros.
__global__ void __launch_bounds__(QR_NT) stacked_r_kernel(const StackJob* __restrict__ jobs, int njobs,
                                                          const RowSeg* __restrict__ segs) {
    extern __shared__ double smem[];
    __shared__ double tau[kSmemMaxC];
    __shared__ double rn[kSmemMaxC];
    __shared__ int src[kSmemMaxC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int jbi = blockIdx.x; jbi < njobs; jbi += gridDim.x) {
        const StackJob jb = jobs[jbi];
        const int c = jb.c;
        if (c <= 0) continue;
        const int lda = work_ld(c);
        double* A = smem;
        stacked_qr<QR_NT>(A, lda, c, chunk_rows(c), segs, jb.seg_begin, jb.seg_end, tau);
        int rows = 0;
        for (int i = jb.seg_begin; i < jb.seg_end; ++i) rows += segs[i].rows;
        const int reff = min(c, rows);
        if (rows >= c) {   // the triangle as computed (upper triangular: callers may mark it tri)
            for (int x = threadIdx.x; x < c * c; x += QR_NT) {
                const int r = x % c, k = x / c;
                jb.out[r + (int64_t)k * jb.ldo] = r <= k ? A[r + (int64_t)k * lda] : 0.0;
            }
            __syncthreads();
            continue;
        }
        for (int j = warp; j < c; j += QR_NW) {   // squared norms of the rows of R
            double x = 0.0;
            for (int k = j + lane; k < c; k += 32) {
                const double a = A[j + (int64_t)k * lda];
                x = fma(a, a, x);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) rn[j] = x;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < c; j += QR_NT) {   // rank by descending norm (ties by index)
            const double x = rn[j];
            int r = 0;
            for (int i = 0; i < c; ++i) {
                const double y = rn[i];
                r += (y > x || (y == x && i < j)) ? 1 : 0;
            }
            if (r < reff) src[r] = j;
        }
        __syncthreads();
        for (int x = threadIdx.x; x < c * c; x += QR_NT) {
            const int r = x % c, k = x / c;
            jb.out[r + (int64_t)k * jb.ldo] = (r < reff) ? A[src[r] + (int64_t)k * lda] : 0.0;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SQ_NT) stacked_svd_kernel(const StackJob* __restrict__ jobs,
                                                            const RowSeg* __restrict__ segs, double thr, int kmax,
                                                            int* __restrict__ cap_flag) {
    extern __shared__ double smem[];
    __shared__ double tau[SVD_MAXC];
    __shared__ double sig[SVD_MAXC + 1];
    __shared__ int rank[SVD_MAXC];
    __shared__ int perm[SVD_MAXC];
    __shared__ int cols[SVD_MAXC + 2];
    __shared__ int kk, mcols;
    const StackJob jb = jobs[blockIdx.x];
    const int c = jb.c;
    if (c <= 0) {
        if (threadIdx.x == 0) *jb.k_out = 0;
        return;
    }
    const int np = c + (c & 1);          // even order for the round-robin schedule (zero column added)
    const int lda = work_ld(c, kSvdChunk);
    const int ldb = c | 1;
    double* A = smem;                         // lda x c: [R; chunk]
    double* B = smem + (int64_t)lda * c;      // ldb x np: R^T and a zero padding column
    stacked_qr<SQ_NT>(A, lda, c, kSvdChunk, segs, jb.seg_begin, jb.seg_end, tau);
    // W^T = Q1 R1 and R1 P = Q3 R3 give W = P R3^T (Q1 Q3)^T: the left singular vectors of W
    // are those of R3^T with their rows permuted by P
    pivoted_qr(A, lda, c, perm, sig, tau);
    for (int x = threadIdx.x; x < c * np; x += SQ_NT) {
        const int i = x % c, k = x / c;
        B[i + (int64_t)k * ldb] = (k < c && i >= k) ? A[k + (int64_t)i * lda] : 0.0;
    }
    __syncthreads();
    const int g = threadIdx.x >> 3, sub = threadIdx.x & 7;
    // columns of B at rounding level (norm <= c eps max norm) are set to zero: a perturbation
    // of B at rounding level, and Jacobi rotations against them would not converge
    for (int j0 = 0; j0 < np; j0 += 32) {
        const int j = j0 + g;
        double s2 = 0.0;
        if (j < np)
            for (int i = sub; i < c; i += 8) {
                const double a = B[i + (int64_t)j * ldb];
                s2 = fma(a, a, s2);
            }
        s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
        s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
        s2 += __shfl_xor_sync(0xffffffffu, s2, 4);
        if (sub == 0 && j < np) sig[j] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int j = 0; j < np; ++j) mx = fmax(mx, sig[j]);
        tau[0] = mx * ((double)c * DBL_EPSILON) * ((double)c * DBL_EPSILON);
    }
    __syncthreads();
    const double floor2 = tau[0];
    for (int x = threadIdx.x; x < c * np; x += SQ_NT) {
        const int i = x % c, k = x / c;
        if (sig[k] <= floor2) B[i + (int64_t)k * ldb] = 0.0;
    }
    // the sweeps run over the columns above the floor only (a rotation against a zero column is
    // the identity), padded to an even count with a zero column, which exists since np is even
    if (threadIdx.x == 0) {
        int m = 0, z = -1;
        for (int j = 0; j < np; ++j) {
            if (sig[j] > floor2) cols[m++] = j;
            else if (z < 0) z = j;
        }
        if (m & 1) cols[m++] = z;
        mcols = m;
    }
    __syncthreads();
    // one-sided Jacobi on the columns of B = R^T (W = B Q^T): 8 threads per column pair,
    // 32 pairs at a time; at convergence the columns of B V are orthogonal and their
    // normalised values are the left singular vectors of W
    const int mp = mcols;
    const int half = mp / 2;
    const double tol = 2.0 * (double)c * DBL_EPSILON;   // orthogonality reached (rounding of the dot products)
    for (int sweep = 0; sweep < 60 && mp > 0; ++sweep) {
        int rotated = 0;
        for (int r = 0; r < mp - 1; ++r) {
            for (int k0 = 0; k0 < half; k0 += 32) {
                const int k = k0 + g;
                const bool act = k < half;
                int p = 0, q = 0;
                if (act) {   // round-robin pair k of round r over the listed columns
                    if (k == 0) { p = cols[mp - 1]; q = cols[r]; }
                    else { p = cols[(r + k) % (mp - 1)]; q = cols[(r - k + (mp - 1)) % (mp - 1)]; }
                    if (p > q) { const int t = p; p = q; q = t; }
                }
                double al = 0.0, be = 0.0, ga = 0.0;
                if (act)
                    for (int i = sub; i < c; i += 8) {
                        const double ap = B[i + (int64_t)p * ldb], aq = B[i + (int64_t)q * ldb];
                        al = fma(ap, ap, al);
                        be = fma(aq, aq, be);
                        ga = fma(ap, aq, ga);
                    }
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                if (act && ga != 0.0 && fabs(ga) > tol * sqrt(al) * sqrt(be)) {
                    const double zeta = (be - al) / (2.0 * ga);
                    const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
                    const double cs = 1.0 / sqrt(fma(t, t, 1.0));
                    const double sn = cs * t;
                    for (int i = sub; i < c; i += 8) {
                        const double ap = B[i + (int64_t)p * ldb], aq = B[i + (int64_t)q * ldb];
                        B[i + (int64_t)p * ldb] = cs * ap - sn * aq;
                        B[i + (int64_t)q * ldb] = sn * ap + cs * aq;
                    }
                    rotated = 1;
                }
            }
            __syncthreads();
        }
        if (!__syncthreads_or(rotated)) break;
    }
    // singular values = column norms; rank by descending value (ties by index)
    for (int j0 = 0; j0 < np; j0 += 32) {   // uniform trip count: the shuffles below need every lane
        const int j = j0 + g;
        double s2 = 0.0;
        if (j < np)
            for (int i = sub; i < c; i += 8) {
                const double a = B[i + (int64_t)j * ldb];
                s2 = fma(a, a, s2);
            }
        s2 += __shfl_xor_sync(0xffffffffu, s2, 1);
        s2 += __shfl_xor_sync(0xffffffffu, s2, 2);
        s2 += __shfl_xor_sync(0xffffffffu, s2, 4);
        if (sub == 0 && j < np) sig[j] = sqrt(s2);
    }
    __syncthreads();
    if (threadIdx.x < c) {
        const int i = threadIdx.x;
        const double si = sig[i];
        int rk = 0;
        for (int j = 0; j < c; ++j) {
            const double sj = sig[j];
            if (sj > si || (sj == si && j < i)) ++rk;
        }
        rank[i] = rk;
        if (jb.sv_out) jb.sv_out[rk] = si;
    }
    if (threadIdx.x == 0) {
        int k = 0;
        for (int j = 0; j < c; ++j) k += (sig[j] > thr) ? 1 : 0;
        if (k > kmax) {
            atomicExch(cap_flag, 1);
            k = kmax;
        }
        kk = k;
        *jb.k_out = k;
    }
    __syncthreads();
    const int k = kk;
    for (int x = threadIdx.x; x < c * c; x += SQ_NT) {
        const int row = x % c, j = x / c;
        const int rk = rank[j];
        if (rk < k) jb.out[perm[row] + (int64_t)rk * jb.ldo] = B[row + (int64_t)j * ldb] / sig[j];
    }
}

size_t qr_smem_bytes(int c) { return (size_t)work_ld(c) * c * sizeof(double); }

size_t svd_smem_bytes(int c) {   // increasing in c
    const int np = c + (c & 1);
    return (size_t)work_ld(c, kSvdChunk) * c * sizeof(double) + (size_t)(c | 1) * np * sizeof(double);
}

}  // namespace

namespace {

// Event timing of the stacked launches (enabled with the GEMM profile).
struct StackProfile {
    std::mutex mu;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used;
    std::vector<cudaEvent_t> pool;
    double ms = 0.0, flops = 0.0;
    int64_t launches = 0;
    cudaEvent_t take() {
        if (pool.empty()) {
            cudaEvent_t e;
            H2_CUDA(cudaEventCreate(&e));
            return e;
        }
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
};
StackProfile g_sprof[2];

double qr_flops(double m, double n) {
    return m >= n ? 2.0 * m * n * n - 2.0 * n * n * n / 3.0 : 2.0 * n * m * m - 2.0 * m * m * m / 3.0;
}

double job_rows(const StackJob& j, const std::vector<RowSeg>& segs) {
    double r = 0.0;
    for (int i = j.seg_begin; i < j.seg_end; ++i) r += segs[i].rows;
    return r;
}

// Records the start event of a profiled span of `launches` kernel launches (timed from this
// event on s to the one prof_end records on s); returns it (null when profiling is off).
cudaEvent_t prof_begin(int which, double flops, cudaStream_t s, int launches = 1) {
    if (!gemm_profile_on()) return nullptr;
    StackProfile& P = g_sprof[which];
    std::lock_guard<std::mutex> lock(P.mu);
    cudaEvent_t e = P.take();
    H2_CUDA(cudaEventRecord(e, s));
    P.flops += flops;
    P.launches += launches;
    return e;
}

void prof_end(int which, cudaEvent_t ea, cudaStream_t s) {
    if (!ea) return;
    StackProfile& P = g_sprof[which];
    std::lock_guard<std::mutex> lock(P.mu);
    cudaEvent_t eb = P.take();
    H2_CUDA(cudaEventRecord(eb, s));
    P.used.push_back({ea, eb});
}

}  // namespace

void stack_profile_read(int which, double* ms, double* flops, int64_t* launches) {
    H2_CUDA(cudaDeviceSynchronize());
    StackProfile& P = g_sprof[which & 1];
    std::lock_guard<std::mutex> lock(P.mu);
    for (auto& u : P.used) {
        float t = 0.f;
        H2_CUDA(cudaEventElapsedTime(&t, u.first, u.second));
        P.ms += t;
        P.pool.push_back(u.first);
        P.pool.push_back(u.second);
    }
    P.used.clear();
    if (ms) *ms = P.ms;
    if (flops) *flops = P.flops;
    if (launches) *launches = P.launches;
    P.ms = 0.0;
    P.flops = 0.0;
    P.launches = 0;
}

void stacked_r(const std::vector<StackJob>& jobs_in, const std::vector<RowSeg>& segs_in, StackWork& w,
               cudaStream_t s) {
    if (jobs_in.empty()) return;
    // A tall matrix is split over several CTAs (part jobs of about `target` rows, c x c R factors
    // in w.parts); its final job stacks the part factors.  The target spreads the launch's rows
    // over a few CTAs per SM, within [256, kSplitRows] rows.
    std::vector<StackJob> jobs, parts;
    std::vector<RowSeg> segs, psegs;
    struct Split { size_t job; size_t first_part; int count; };
    std::vector<Split> splits;
    int64_t total = 0;
    for (const StackJob& jb : jobs_in)
        for (int i = jb.seg_begin; i < jb.seg_end; ++i) total += segs_in[i].rows;
    const int target = (int)std::min<int64_t>(kSplitRows, std::max<int64_t>(128, total / (4 * 152)));
    for (const StackJob& jb : jobs_in) {
        if (jb.c <= 0) continue;
        if (jb.c > kSmemMaxC) fail(H2_ERR_INVALID_ARG, "stacked_r: more than 144 columns");
        int64_t rows = 0;
        for (int i = jb.seg_begin; i < jb.seg_end; ++i) rows += segs_in[i].rows;
        StackJob j = jb;
        if (rows <= 2 * (int64_t)std::max(target, jb.c)) {
            j.seg_begin = (int)segs.size();
            for (int i = jb.seg_begin; i < jb.seg_end; ++i) segs.push_back(segs_in[i]);
            j.seg_end = (int)segs.size();
            jobs.push_back(j);
            continue;
        }
        const int prows = std::max(target, jb.c);
        Split sp{jobs.size(), parts.size(), 0};
        int filled = prows;   // rows in the current part (start a new part first)
        for (int i = jb.seg_begin; i < jb.seg_end; ++i) {
            const RowSeg sg = segs_in[i];
            for (int r0 = 0; r0 < sg.rows;) {
                if (filled >= prows) {
                    parts.push_back(StackJob{(int)psegs.size(), (int)psegs.size(), jb.c, nullptr, jb.c, nullptr, nullptr});
                    ++sp.count;
                    filled = 0;
                }
                const int take = std::min(prows - filled, sg.rows - r0);
                psegs.push_back(RowSeg{sg.p + r0, take, sg.ld});
                parts.back().seg_end = (int)psegs.size();
                filled += take;
                r0 += take;
            }
        }
        splits.push_back(sp);
        jobs.push_back(j);   // segments filled once the part factors have addresses
    }
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(stacked_r_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    });
    // one launch per class of c (<= 32, 48, 64, 96, 128, 144), so that narrow jobs are not held to
    // the shared-memory occupancy of the widest; the working matrix's size is not monotone in c
    // (the chunk height steps down at 33, 49, 97 and 129 columns), so a launch takes the largest
    // requirement of its jobs
    // One launch per width class, each on its own side stream after the jobs are uploaded, so
    // that the classes overlap; within a class the jobs run longest first (CTAs start in job
    // order, so the launch's tail holds the short ones).
    auto launch = [&](const std::vector<StackJob>& js, const std::vector<RowSeg>& ss, DevBuf<StackJob>& dj,
                      DevBuf<RowSeg>& dsg, Stager& stj, Stager& sts) {
        constexpr int kBounds[kStackClasses] = {32, 48, 64, 96, 128, kSmemMaxC};
        std::vector<std::pair<double, int>> cls[kStackClasses];
        for (int i = 0; i < (int)js.size(); ++i) {
            const StackJob& j = js[i];
            int b = 0;
            while (j.c > kBounds[b]) ++b;
            cls[b].push_back({job_rows(j, ss) * j.c * j.c, i});
        }
        std::vector<StackJob> all;
        int off[kStackClasses + 1], nonempty = 0;
        for (int b = 0; b < kStackClasses; ++b) {
            std::stable_sort(cls[b].begin(), cls[b].end(),
                             [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; });
            off[b] = (int)all.size();
            for (auto& ci : cls[b]) all.push_back(js[ci.second]);
            nonempty += cls[b].empty() ? 0 : 1;
        }
        off[kStackClasses] = (int)all.size();
        if (all.empty()) return;
        upload(dj, all, s, stj);
        upload(dsg, ss, s, sts);
        // profiling: one span on s around all the classes' launches (they overlap)
        double fl = 0.0;
        if (gemm_profile_on())
            for (auto& j : all) fl += qr_flops(job_rows(j, ss), j.c);
        cudaEvent_t ev = prof_begin(0, fl, s, nonempty);
        const bool fork = nonempty > 1;
        if (fork) {
            if (!w.ev_fork) {
                H2_CUDA(cudaEventCreateWithFlags(&w.ev_fork, cudaEventDisableTiming));
                for (int b = 0; b < kStackClasses; ++b) {
                    H2_CUDA(cudaStreamCreateWithFlags(&w.side[b], cudaStreamNonBlocking));
                    H2_CUDA(cudaEventCreateWithFlags(&w.ev_join[b], cudaEventDisableTiming));
                }
            }
            H2_CUDA(cudaEventRecord(w.ev_fork, s));
        }
        for (int b = 0; b < kStackClasses; ++b) {
            const int n = off[b + 1] - off[b];
            if (!n) continue;
            cudaStream_t sb = fork ? w.side[b] : s;
            if (fork) H2_CUDA(cudaStreamWaitEvent(sb, w.ev_fork, 0));
            size_t dyn = 16;
            for (int i = off[b]; i < off[b + 1]; ++i) dyn = std::max(dyn, qr_smem_bytes(all[i].c));
            stacked_r_kernel<<<(unsigned)n, QR_NT, dyn, sb>>>(dj.p + off[b], n, dsg.p);
            after_launch("stacked_r");
            if (fork) {
                H2_CUDA(cudaEventRecord(w.ev_join[b], sb));
                H2_CUDA(cudaStreamWaitEvent(s, w.ev_join[b], 0));
            }
        }
        prof_end(0, ev, s);
    };
    if (!parts.empty()) {
        int64_t elems = 0;
        for (auto& pj : parts) elems += (int64_t)pj.c * pj.c;
        w.parts.reserve((size_t)elems);
        int64_t off = 0;
        for (auto& pj : parts) {
            pj.out = w.parts.p + off;
            off += (int64_t)pj.c * pj.c;
        }
        launch(parts, psegs, w.d_jobs2, w.d_segs2, w.st_jobs2, w.st_segs2);
        for (const Split& sp : splits) {
            StackJob& fj = jobs[sp.job];
            fj.seg_begin = (int)segs.size();
            for (int i = 0; i < sp.count; ++i) {
                const StackJob& pj = parts[sp.first_part + i];
                const int prow = (int)job_rows(pj, psegs);
                segs.push_back(RowSeg{pj.out, std::min(prow, pj.c), pj.c, prow >= pj.c});
            }
            fj.seg_end = (int)segs.size();
        }
    }
    launch(jobs, segs, w.d_jobs, w.d_segs, w.st_jobs, w.st_segs);
}

StackWork::~StackWork() {
    // teardown: errors are ignored (the context may already be gone at process exit)
    for (int b = 0; b < kStackClasses; ++b) {
        if (side[b]) cudaStreamDestroy(side[b]);
        if (ev_join[b]) cudaEventDestroy(ev_join[b]);
    }
    if (ev_fork) cudaEventDestroy(ev_fork);
}

void stacked_svd_trunc(const std::vector<StackJob>& jobs_in, const std::vector<RowSeg>& segs, StackWork& w,
                       double thr, int kmax, int* d_cap_flag, cudaStream_t s) {
    if (jobs_in.empty()) return;
    // longest first (QR of the stack plus the Jacobi sweeps): CTAs start in job order
    std::vector<std::pair<double, int>> cost;
    for (int i = 0; i < (int)jobs_in.size(); ++i) {
        const double c = jobs_in[i].c;
        cost.push_back({job_rows(jobs_in[i], segs) * c * c + 4.0 * c * c * c, i});
    }
    std::stable_sort(cost.begin(), cost.end(),
                     [](const std::pair<double, int>& x, const std::pair<double, int>& y) { return x.first > y.first; });
    std::vector<StackJob> jobs;
    jobs.reserve(jobs_in.size());
    for (auto& ci : cost) jobs.push_back(jobs_in[ci.second]);
    int cm = 0;
    for (auto& j : jobs) cm = std::max(cm, j.c);
    if (cm > SVD_MAXC) fail(H2_ERR_INVALID_ARG, "stacked_svd: matrix order above 96");
    upload(w.d_jobs, jobs, s, w.st_jobs);
    upload(w.d_segs, segs, s, w.st_segs);
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(stacked_svd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)svd_smem_bytes(SVD_MAXC)));
    });
    double fl = 0.0;
    if (gemm_profile_on())
        for (auto& j : jobs) fl += qr_flops(job_rows(j, segs), j.c) + 4.0 * j.c * (double)j.c * j.c / 3.0;
    cudaEvent_t ev = prof_begin(1, fl, s);
    stacked_svd_kernel<<<(unsigned)jobs.size(), SQ_NT, svd_smem_bytes(std::max(cm, 1)), s>>>(
        w.d_jobs.p, w.d_segs.p, thr, kmax, d_cap_flag);
    after_launch("stacked_svd");
    prof_end(1, ev, s);
}

int svd_max_order() { return SVD_MAXC; }

int stacked_r_max_columns() { return kSmemMaxC; }

namespace {

// Cholesky factorisation with symmetric (diagonal) pivoting of a symmetric positive
// semidefinite matrix (the rank-revealing form: the largest remaining diagonal is the next
// pivot, and the factorisation stops once it is at rounding level), one CTA per matrix.
// The trailing Schur complement is kept in full (both triangles) so that rows and columns can
// be swapped; columns 0..j-1 hold the finished columns of L.
__global__ void __launch_bounds__(SQ_NT) psd_chol_small_kernel(const CholItem* __restrict__ items) {
    extern __shared__ double A[];   // m x m, leading dimension m + 1
    __shared__ int perm[SVD_MAXC];
    __shared__ int piv;
    __shared__ double pval, drop_s;
    const CholItem it = items[blockIdx.x];
    const int m = it.m, ld = m + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int x = threadIdx.x; x < m * m; x += SQ_NT) {
        const int i = x % m, j = x / m;
        A[i + j * ld] = (i >= j) ? it.G[i + (int64_t)j * it.ldg] : it.G[j + (int64_t)i * it.ldg];
    }
    if (threadIdx.x < m) perm[threadIdx.x] = threadIdx.x;
    __syncthreads();
    if (warp == 0) {
        double mx = 0.0;
        for (int i = lane; i < m; i += 32) mx = fmax(mx, A[i + i * ld]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) drop_s = (double)m * 0x1p-52 * mx;
    }
    __syncthreads();
    const double drop = drop_s;
    int jend = m;
    for (int j = 0; j < m; ++j) {
        if (warp == 0) {   // pivot: the largest remaining diagonal
            double bv = -1.0;
            int bi = j;
            for (int i = j + lane; i < m; i += 32) {
                const double v = A[i + i * ld];
                if (v > bv) { bv = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
            }
            if (lane == 0) { piv = bi; pval = bv; }
        }
        __syncthreads();
        if (!(pval > drop)) { jend = j; break; }   // the same in every thread: the rest is rounding
        const int p = piv;
        if (p != j) {
            for (int c = threadIdx.x; c < m; c += SQ_NT) {   // swap rows j and p
                const double t = A[j + c * ld];
                A[j + c * ld] = A[p + c * ld];
                A[p + c * ld] = t;
            }
            __syncthreads();
            for (int r = threadIdx.x; r < m; r += SQ_NT) {   // swap columns j and p
                const double t = A[r + j * ld];
                A[r + j * ld] = A[r + p * ld];
                A[r + p * ld] = t;
            }
            if (threadIdx.x == 0) { const int t = perm[j]; perm[j] = perm[p]; perm[p] = t; }
            __syncthreads();
        }
        const double ljj = sqrt(A[j + j * ld]);
        __syncthreads();
        for (int i = j + threadIdx.x; i < m; i += SQ_NT) A[i + j * ld] = (i == j) ? ljj : A[i + j * ld] / ljj;
        __syncthreads();
        const int r = m - j - 1;
        for (int x = threadIdx.x; x < r * r; x += SQ_NT) {   // full trailing Schur complement
            const int i = j + 1 + x % r, k = j + 1 + x / r;
            A[i + k * ld] -= A[i + j * ld] * A[k + j * ld];
        }
        __syncthreads();
    }
    // out = F^T with F = P L (F F^T = G): row j of out holds column j of L at the original indices
    for (int x = threadIdx.x; x < m * m; x += SQ_NT) {
        const int jr = x % m, i = x / m;   // out row jr, pivot position i
        const double v = (jr < jend && i >= jr) ? A[i + jr * ld] : 0.0;
        it.out[jr + (int64_t)perm[i] * it.ldo] = v;
    }
}

}  // namespace

void psd_chol_small(const std::vector<CholItem>& items, StackWork& w, cudaStream_t s) {
    if (items.empty()) return;
    for (const CholItem& it : items)
        if (it.m < 1 || it.m > SVD_MAXC) fail(H2_ERR_INVALID_ARG, "psd_chol_small: order out of range");
    int mm = 1;
    for (const CholItem& it : items) mm = std::max(mm, it.m);
    std::vector<unsigned char> raw(items.size() * sizeof(CholItem));
    std::memcpy(raw.data(), items.data(), raw.size());
    upload(w.d_chol, raw, s, w.st_chol);
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(psd_chol_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(SVD_MAXC * (SVD_MAXC + 1) * sizeof(double))));
    });
    psd_chol_small_kernel<<<(unsigned)items.size(), SQ_NT, (size_t)mm * (mm + 1) * sizeof(double), s>>>(
        reinterpret_cast<const CholItem*>(w.d_chol.p));
    after_launch("psd_chol_small");
}

}  // namespace h2
