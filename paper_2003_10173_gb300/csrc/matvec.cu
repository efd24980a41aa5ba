// Multi-right-hand-side H^2 matvec (Section 3.2, Eq. (3.2)).
//
//   Y = D X + U (S (U^T X))
//
// in five marshaled stages, each a list of small block products grouped by
// output block (one CTA per output block and right-hand-side tile; no atomics,
// so results are deterministic):
//   1. leaf upsweep      xh_t = U_t^T X_t                    (X read through the tree permutation)
//   2. upsweep           xh_p = E_c1^T xh_c1 + E_c2^T xh_c2   (one stage per level, leaves to root)
//   3. couplings         yh_t = sum_s S_ts xh_s                (all levels in one stage)
//   4. downsweep         yh_c += E_c yh_p                      (one stage per level, root to leaves)
//   5. leaf expansion    Y_t = U_t yh_t + sum_s D_ts X_s       (written through the permutation)
// Only the lower triangle of S and D is stored; upper blocks are used as
// transposes of the stored ones.
#include <type_traits>
#include <algorithm>
#include <functional>
#include <mutex>

#include "handle.h"

namespace h2 {

namespace {

constexpr int NT = 256;
constexpr int RMAX = 96;     // largest block dimension (leaf size / rank)
constexpr int RT = 32;       // right-hand sides per CTA
constexpr int OPT = (RMAX * RT + NT - 1) / NT;
constexpr int64_t kMaxNrhs = 2000000;   // keeps the grid's y dimension (nrhs / RT) below 65536

template <class T> __device__ __forceinline__ float to_f(T x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <class TA, class T> __device__ __forceinline__ TA cvt(T x) { return (TA)to_f<T>(x); }
template <> __device__ __forceinline__ double cvt<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float cvt<float, float>(float x) { return x; }

// Compensated FP32 value hi + lo (an unevaluated pair of floats): about 48 significant bits
// computed on the FP32 pipe (H2_FP32C).  Products and sums use the error-free transformations
// of Dekker and Knuth (the product's rounding error from one FMA, the sum's from the two-sum
// sequence), so that the stored factors' FP32 rounding is the only reduced-precision step.
struct CF {
    float hi, lo;
    CF() = default;
    __host__ __device__ constexpr CF(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit constexpr CF(int x) : hi((float)x), lo(0.f) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};
__device__ __forceinline__ CF two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    return CF(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ CF fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = a + b;
    return CF(s, b - (s - a));
}
// c + a b (an overload beside the library's fma, which stays visible for the other types).  The
// high part takes the exact two-sum of c.hi and the rounded product; the product's rounding
// error, the cross terms and the sum's error go to the low part, which is not renormalised here:
// hi + lo stays an unevaluated pair whose low part accumulates terms of about 2^-24 of the
// products, so its own rounding costs about 2^-48 of them.
using ::fma;
__device__ __forceinline__ CF fma(CF a, CF b, CF c) {
    const float p = a.hi * b.hi;
    const float pe = fmaf(a.hi, b.hi, -p);
    const float err = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, pe));
    const CF t = two_sum(c.hi, p);
    return CF(t.hi, c.lo + (t.lo + err));
}
__device__ __forceinline__ CF operator+(CF a, CF b) {
    const CF t = two_sum(a.hi, b.hi);
    return fast_two_sum(t.hi, t.lo + (a.lo + b.lo));
}
__device__ __forceinline__ double operator+(double a, CF b) { return a + (double)b; }
template <> __device__ __forceinline__ CF cvt<CF, float>(float x) { return CF(x, 0.f); }
template <> __device__ __forceinline__ CF cvt<CF, double>(double x) {
    const float h = __double2float_rn(x);
    return CF(h, __double2float_rn(x - (double)h));
}

// TS: factor storage type, TX: type of X, TY: type of Y, TA: arithmetic / workspace type.
template <class TS, class TX, class TY, class TA, bool OUT_Y, int RTT>
__device__ __forceinline__ void mv_stage_body(const MvOut& o, const MvItem* __restrict__ items,
                                              const TS* __restrict__ fac, TA* __restrict__ ws, int64_t ws_ld,
                                              const int32_t* __restrict__ perm, const TX* __restrict__ X,
                                              int64_t ldx, TY* __restrict__ Y, int64_t ldy, int nrhs,
                                              int accumulate) {
    constexpr int OPTT = (RMAX * RTT + NT - 1) / NT;
    extern __shared__ unsigned char smem_raw[];
    TA* Ms = reinterpret_cast<TA*>(smem_raw);             // [RMAX cols][RMAX+1 rows] column-major
    TA* IN = Ms + RMAX * (RMAX + 1);                        // [RMAX rows][RTT]
    const int r0 = blockIdx.y * RTT;
    const int nr = min(RTT, nrhs - r0);
    const int rows = o.rows;
    const int nel = rows * nr;
    TA acc[OPTT];
#pragma unroll
    for (int q = 0; q < OPTT; ++q) acc[q] = (TA)0;
    // FP32 arithmetic is bound by the shared-memory reads of its operands rather than by the FMA
    // pipe: there every thread computes a TI x TR block of the output, so that each staged factor
    // entry and input value feeds several products (batched FP32 matvec of 64 Hessians, nrhs 64:
    // 62 -> 39 ms).  FP64 and the compensated form keep one output per thread and step: their
    // arithmetic per product is the bound (the compensated form measured 388 -> 448 ms tiled).
    constexpr bool TILED = std::is_same<TA, float>::value;
    constexpr int TI = 3, TR = 4;
    const int ngr = (rows + TI - 1) / TI;
    const bool tile_live = threadIdx.x < ngr * (RTT / TR);
    const int ti0 = TI * (threadIdx.x % max(ngr, 1)), tr0 = TR * (threadIdx.x / max(ngr, 1));
    TA tacc[TI][TR];
#pragma unroll
    for (int u = 0; u < TI; ++u)
#pragma unroll
        for (int v = 0; v < TR; ++v) tacc[u][v] = (TA)0;

    for (int it = o.beg; it < o.end; ++it) {
        const MvItem m = items[it];
        const int cols = m.cols;
        const TS* M = fac + m.m_off;
        const bool tr = (m.trans & 1) != 0;
        const int ne = rows * cols;
        for (int e = threadIdx.x; e < ne; e += NT) {
            int i, j;
            if (!tr) { i = e % rows; j = e / rows; }   // contiguous along i
            else     { j = e % cols; i = e / cols; }   // contiguous along j
            const TS v = tr ? M[j + (int64_t)i * m.ldm] : M[i + (int64_t)j * m.ldm];
            Ms[j * (RMAX + 1) + i] = cvt<TA>(v);
        }
        const int ni = cols * nr;
        if (m.trans & 2) {
            for (int e = threadIdx.x; e < ni; e += NT) {
                const int j = e % cols, r = e / cols;
                IN[j * RTT + r] = cvt<TA>(X[perm[m.in_off + j] + (int64_t)(r0 + r) * ldx]);
            }
        } else {
            for (int e = threadIdx.x; e < ni; e += NT) {
                const int j = e % cols, r = e / cols;
                IN[j * RTT + r] = ws[m.in_off + j + (int64_t)(r0 + r) * ws_ld];
            }
        }
        __syncthreads();
        if constexpr (TILED) {
            if (tile_live) {
                for (int j = 0; j < cols; ++j) {
                    TA mv[TI], xv[TR];
#pragma unroll
                    for (int u = 0; u < TI; ++u) mv[u] = Ms[j * (RMAX + 1) + ti0 + u];
#pragma unroll
                    for (int v = 0; v < TR; ++v) xv[v] = IN[j * RTT + tr0 + v];
#pragma unroll
                    for (int u = 0; u < TI; ++u)
#pragma unroll
                        for (int v = 0; v < TR; ++v) tacc[u][v] = fma(mv[u], xv[v], tacc[u][v]);
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < OPTT; ++q) {
                const int e = threadIdx.x + q * NT;
                if (e < nel) {
                    const int i = e % rows, r = e / rows;
                    TA s = acc[q];
                    for (int j = 0; j < cols; ++j) s = fma(Ms[j * (RMAX + 1) + i], IN[j * RTT + r], s);
                    acc[q] = s;
                }
            }
        }
        __syncthreads();
    }
    auto store = [&](int i, int r, TA v) {
        if (OUT_Y) {
            TY* y = Y + perm[o.out_off + i] + (int64_t)(r0 + r) * ldy;
            *y = accumulate ? (TY)(*y + v) : (TY)v;
        } else {
            TA* y = ws + o.out_off + i + (int64_t)(r0 + r) * ws_ld;
            *y = accumulate ? (TA)(*y + v) : v;
        }
    };
    if constexpr (TILED) {
        if (tile_live)
#pragma unroll
            for (int u = 0; u < TI; ++u)
#pragma unroll
                for (int v = 0; v < TR; ++v)
                    if (ti0 + u < rows && tr0 + v < nr) store(ti0 + u, tr0 + v, tacc[u][v]);
    } else {
#pragma unroll
        for (int q = 0; q < OPTT; ++q) {
            const int e = threadIdx.x + q * NT;
            if (e < nel) store(e % rows, e / rows, acc[q]);
        }
    }
}

// Stages whose outputs are coefficient blocks (upsweep, couplings, downsweep, leaf upsweep).
template <class TS, class TX, class TY, class TA>
__global__ void __launch_bounds__(NT) mv_stage_kernel(const MvOut* __restrict__ outs, const MvItem* __restrict__ items,
                                                       const TS* __restrict__ fac, TA* __restrict__ ws, int64_t ws_ld,
                                                       const int32_t* __restrict__ perm, const TX* __restrict__ X,
                                                       int64_t ldx, TY* __restrict__ Y, int64_t ldy, int nrhs,
                                                       int accumulate) {
    mv_stage_body<TS, TX, TY, TA, false, RT>(outs[blockIdx.x], items, fac, ws, ws_ld, perm, X, ldx, Y, ldy, nrhs,
                                             accumulate);
}

// Transfer stages of the tree sweeps (upsweep x_p = sum_c E_c^T x_c, downsweep y_c += E_c y_p):
// inputs and outputs are coefficient rows of the workspace, blocks at most KB x KB.  One CTA per
// (output box, TR_RC right-hand sides), one thread per right-hand side: the thread keeps the
// box's output column in registers while the item matrices are broadcast from shared memory;
// inputs and outputs pass through a padded shared tile so that global accesses run along the
// coefficient rows.
constexpr int TR_RC = 128;

template <class TS, class TA, int KB>
__global__ void __launch_bounds__(TR_RC) mv_transfer_kernel(const MvOut* __restrict__ outs,
                                                            const MvItem* __restrict__ items,
                                                            const TS* __restrict__ fac, TA* __restrict__ ws,
                                                            int64_t ws_ld, int nrhs, int accumulate) {
    constexpr int XS = KB + 1;   // odd stride: a thread's staged column is conflict-free
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TA* Ms = reinterpret_cast<TA*>(smem_raw);   // item matrix, [col j][row i], rows zero padded to 4
    TA* XT = Ms + KB * KB;                        // [TR_RC][XS]: input columns, then output columns
    const MvOut o = outs[blockIdx.x];
    const int tid = threadIdx.x;
    const int r0 = blockIdx.y * TR_RC;
    const int nr = min(TR_RC, nrhs - r0);
    const int rows = o.rows;
    const int rows4 = (rows + 3) & ~3;
    TA acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = (TA)0;
    for (int it = o.beg; it < o.end; ++it) {
        const MvItem m = items[it];
        const int cols = m.cols;
        const bool tr = (m.trans & 1) != 0;
        const TS* M = fac + m.m_off;
        for (int e = tid; e < rows4 * cols; e += TR_RC) {
            int i, j;
            if (!tr) { i = e % rows4; j = e / rows4; }   // contiguous along i
            else     { j = e % cols; i = e / cols; }     // contiguous along j
            TA v = (TA)0;
            if (i < rows) v = cvt<TA>(tr ? M[j + (int64_t)i * m.ldm] : M[i + (int64_t)j * m.ldm]);
            Ms[j * KB + i] = v;
        }
        for (int e = tid; e < cols * nr; e += TR_RC) {
            const int j = e % cols, r = e / cols;
            XT[r * XS + j] = ws[m.in_off + j + (int64_t)(r0 + r) * ws_ld];
        }
        __syncthreads();
        if (tid < nr) {
            const TA* x = XT + tid * XS;
            for (int j = 0; j < cols; ++j) {
                const TA xv = x[j];
                const TA* mj = Ms + j * KB;
#pragma unroll
                for (int i4 = 0; i4 < KB / 4; ++i4) {
                    if (4 * i4 < rows4) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) acc[4 * i4 + q] = fma(mj[4 * i4 + q], xv, acc[4 * i4 + q]);
                    }
                }
            }
        }
        __syncthreads();
    }
    if (tid < nr) {
#pragma unroll
        for (int i = 0; i < KB; ++i)
            if (i < rows) XT[tid * XS + i] = acc[i];
    }
    __syncthreads();
    for (int e = tid; e < rows * nr; e += TR_RC) {
        const int i = e % rows, r = e / rows;
        TA* y = ws + o.out_off + i + (int64_t)(r0 + r) * ws_ld;
        const TA v = XT[r * XS + i];
        *y = accumulate ? (TA)(*y + v) : v;
    }
}

// The same transfer stages on a right-hand-side-major workspace (ws[row * ld + rhs], the
// tensor-core path's layout), for outputs with at most two items (a parent's two children in the
// upsweep, the parent in the downsweep): the item matrices go to shared memory once; each thread
// keeps its right-hand side's output column in registers and reads its inputs straight from
// global memory (consecutive threads, consecutive addresses); many resident warps hide their
// latency.  When accumulating, old output values are loaded eight at a time before their stores.
template <class TS, int KB>
__device__ __forceinline__ void transfer_rm_body(const MvOut& o, const MvItem* __restrict__ items,
                                                 const TS* __restrict__ fac, float* __restrict__ ws, int64_t ld,
                                                 int nrhs, int accumulate) {
    __shared__ __align__(16) float Ms[2][KB * KB];   // item matrices, [col j][row i], zero beyond the rows
    const int tid = threadIdx.x;
    const int r = blockIdx.y * TR_RC + tid;
    const bool live = r < nrhs;
    const int rows = o.rows;
    const int nit = o.end - o.beg;   // 1 or 2 (host-checked)
    float acc[KB];
#pragma unroll
    for (int i = 0; i < KB; ++i) acc[i] = 0.f;
    for (int q = 0; q < nit; ++q) {
        const MvItem m = items[o.beg + q];
        const bool tr = (m.trans & 1) != 0;
        const TS* M = fac + m.m_off;
        for (int e = tid; e < KB * m.cols; e += TR_RC) {
            int i, j;
            if (!tr) { i = e % KB; j = e / KB; }
            else     { j = e % m.cols; i = e / m.cols; }
            float v = 0.f;
            if (i < rows) v = cvt<float>(tr ? M[j + (int64_t)i * m.ldm] : M[i + (int64_t)j * m.ldm]);
            Ms[q][j * KB + i] = v;
        }
    }
    __syncthreads();
    if (!live) return;
    for (int q = 0; q < nit; ++q) {
        const MvItem m = items[o.beg + q];
        const float* Mq = Ms[q];
        const float* x = ws + m.in_off * ld + r;
        // four input entries in flight per step
#pragma unroll 1
        for (int j0 = 0; j0 < m.cols; j0 += 4) {
            float xv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) xv[u] = (j0 + u < m.cols) ? x[(int64_t)(j0 + u) * ld] : 0.f;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j0 + u >= m.cols) break;
                const float4* mj = reinterpret_cast<const float4*>(Mq + (j0 + u) * KB);
#pragma unroll
                for (int i4 = 0; i4 < KB / 4; ++i4) {
                    const float4 w = mj[i4];
                    acc[4 * i4 + 0] = fmaf(w.x, xv[u], acc[4 * i4 + 0]);
                    acc[4 * i4 + 1] = fmaf(w.y, xv[u], acc[4 * i4 + 1]);
                    acc[4 * i4 + 2] = fmaf(w.z, xv[u], acc[4 * i4 + 2]);
                    acc[4 * i4 + 3] = fmaf(w.w, xv[u], acc[4 * i4 + 3]);
                }
            }
        }
    }
    float* y = ws + o.out_off * ld + r;
#pragma unroll
    for (int i0 = 0; i0 < KB; i0 += 8) {
        if (i0 >= rows) break;
        // eight old values in flight together, then their stores
        float old[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) old[u] = (accumulate && i0 + u < rows) ? y[(int64_t)(i0 + u) * ld] : 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (i0 + u < rows) y[(int64_t)(i0 + u) * ld] = acc[i0 + u] + old[u];
    }
}

template <class TS, int KB>
__global__ void __launch_bounds__(TR_RC) mv_transfer_rm_kernel(const MvOut* __restrict__ outs,
                                                               const MvItem* __restrict__ items,
                                                               const TS* __restrict__ fac, float* __restrict__ ws,
                                                               int64_t ld, int nrhs, int accumulate) {
    transfer_rm_body<TS, KB>(outs[blockIdx.x], items, fac, ws, ld, nrhs, accumulate);
}

// The merged sweep stage of a batch on the handles' right-hand-side-major workspaces (leading
// dimension nrhs for every handle): output o belongs to handle o.h.
template <class TS, int KB>
__global__ void __launch_bounds__(TR_RC) mv_batch_transfer_rm_kernel(const MvOut* __restrict__ outs,
                                                                     const MvItem* __restrict__ items,
                                                                     const BatchBase* __restrict__ bases, int nrhs,
                                                                     int accumulate) {
    const MvOut o = outs[blockIdx.x];
    const BatchBase B = bases[o.h];
    transfer_rm_body<TS, KB>(o, items, static_cast<const TS*>(B.fac), static_cast<float*>(B.ws), (int64_t)nrhs, nrhs,
                             accumulate);
}

template <class TS, int KB>
void launch_transfer_rm(const MvStage& st, const TS* fac, float* ws, int64_t ld, int nrhs, cudaStream_t s) {
    dim3 grid((unsigned)st.outs.size(), (unsigned)((nrhs + TR_RC - 1) / TR_RC));
    mv_transfer_rm_kernel<TS, KB><<<grid, TR_RC, 0, s>>>(st.d_outs.p, st.d_items.p, fac, ws, ld, nrhs,
                                                         st.accumulate);
    after_launch("mv_transfer_rm");
}

template <class TS, class TA, int KB>
void launch_transfer(const MvStage& st, const TS* fac, TA* ws, int64_t ws_ld, int nrhs, cudaStream_t s) {
    const size_t smem = (size_t)(KB * KB + TR_RC * (KB + 1)) * sizeof(TA);
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(mv_transfer_kernel<TS, TA, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    });
    dim3 grid((unsigned)st.outs.size(), (unsigned)((nrhs + TR_RC - 1) / TR_RC));
    mv_transfer_kernel<TS, TA, KB><<<grid, TR_RC, smem, s>>>(st.d_outs.p, st.d_items.p, fac, ws, ws_ld, nrhs,
                                                             st.accumulate);
    after_launch("mv_transfer");
}

// Final stage: leaf expansion plus the dense near field, written to Y.
template <class TS, class TX, class TY, class TA>
__global__ void __launch_bounds__(NT) mv_leaf_near_kernel(const MvOut* __restrict__ outs,
                                                           const MvItem* __restrict__ items,
                                                           const TS* __restrict__ fac, TA* __restrict__ ws,
                                                           int64_t ws_ld, const int32_t* __restrict__ perm,
                                                           const TX* __restrict__ X, int64_t ldx, TY* __restrict__ Y,
                                                           int64_t ldy, int nrhs, int accumulate) {
    mv_stage_body<TS, TX, TY, TA, true, RT>(outs[blockIdx.x], items, fac, ws, ws_ld, perm, X, ldx, Y, ldy, nrhs,
                                            accumulate);
}

// Small-nrhs stages (tree sweeps, leaf upsweep, leaf expansion for nrhs <= 4): one warp per
// output block, lanes over its rows (at most 96, three per lane), inputs read straight from X or
// the workspace (the same value for every lane: a broadcast), no shared memory, so that the many
// tiny blocks of a level run as one wave of warps.
template <class TS, class TX, class TY, class TA, bool OUT_Y, int NR>
__global__ void __launch_bounds__(256) mv_small_stage_kernel(const MvOut* __restrict__ outs, int nouts,
                                                              const MvItem* __restrict__ items,
                                                              const TS* __restrict__ fac, TA* __restrict__ ws,
                                                              int64_t ws_ld, const int32_t* __restrict__ perm,
                                                              const TX* __restrict__ X, int64_t ldx,
                                                              TY* __restrict__ Y, int64_t ldy, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (idx >= nouts) return;
    const MvOut o = outs[idx];
    const int rows = o.rows;
    TA acc[3][NR];
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[q][r] = (TA)0;
    for (int it = o.beg; it < o.end; ++it) {
        const MvItem m = items[it];
        const TS* M = fac + m.m_off;
        const bool tr = (m.trans & 1) != 0;
        for (int j = 0; j < m.cols; ++j) {
            TA in[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r)
                in[r] = (m.trans & 2) ? cvt<TA>(X[perm[m.in_off + j] + (int64_t)r * ldx])
                                      : ws[m.in_off + j + (int64_t)r * ws_ld];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const int i = lane + 32 * q;
                if (i < rows) {
                    const TA d = cvt<TA>(tr ? M[j + (int64_t)i * m.ldm] : M[i + (int64_t)j * m.ldm]);
#pragma unroll
                    for (int r = 0; r < NR; ++r) acc[q][r] = fma(d, in[r], acc[q][r]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int i = lane + 32 * q;
        if (i >= rows) continue;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            if (OUT_Y) {
                // the near-field scatter may be adding into Y concurrently (another stream): atomic
                TY* y = Y + perm[o.out_off + i] + (int64_t)r * ldy;
                if (accumulate) atomicAdd(y, (TY)acc[q][r]);
                else *y = (TY)acc[q][r];
            } else {
                TA* y = ws + o.out_off + i + (int64_t)r * ws_ld;
                *y = accumulate ? (TA)(*y + acc[q][r]) : acc[q][r];
            }
        }
    }
}

// Batched stages: outputs of several handles in one launch; each output names its handle and the
// handle's bases (factors, workspace, permutation, X, Y) come from a device table.
template <class TS, class TX, class TY, class TA, bool OUT_Y, int RTT>
__global__ void __launch_bounds__(NT) mv_batch_stage_kernel(const MvOut* __restrict__ outs,
                                                             const MvItem* __restrict__ items,
                                                             const BatchBase* __restrict__ bases, int nrhs,
                                                             int accumulate) {
    const MvOut o = outs[blockIdx.x];
    const BatchBase b = bases[o.h];
    mv_stage_body<TS, TX, TY, TA, OUT_Y, RTT>(o, items, (const TS*)b.fac, (TA*)b.ws, b.ws_ld, b.perm, (const TX*)b.X,
                                              b.ldx, (TY*)b.Y, b.ldy, nrhs, accumulate);
}

template <class TS, class TA>
__global__ void convert_kernel(const double* __restrict__ src, TS* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = (TS)src[i];
}
template <>
__global__ void convert_kernel<__nv_bfloat16, float>(const double* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16_rn((float)src[i]);
}

// Small-nrhs scatter product: one warp per stored block, read once in 32 x 32 tiles
// (coalesced along rows); out_t += M in_s from registers and out_s += M^T in_t from a
// per-warp shared-memory copy of the tile; both added with atomics.
constexpr int SW = 8;   // warps per CTA

template <class TA, class TX, bool VIA_PERM>
__device__ __forceinline__ TA sc_in(const TX* __restrict__ X, int64_t ldx, const TA* __restrict__ ws, int64_t ws_ld,
                                    const int32_t* __restrict__ perm, int64_t off, int j, int r) {
    if constexpr (VIA_PERM) return cvt<TA>(X[perm[off + j] + (int64_t)r * ldx]);
    else return ws[off + j + (int64_t)r * ws_ld];
}

template <class TA, class TY, bool VIA_PERM>
__device__ __forceinline__ void sc_add(TY* __restrict__ Y, int64_t ldy, TA* __restrict__ ws, int64_t ws_ld,
                                       const int32_t* __restrict__ perm, int64_t off, int i, int r, TA v) {
    if constexpr (VIA_PERM) atomicAdd(Y + perm[off + i] + (int64_t)r * ldy, (TY)v);
    else atomicAdd(ws + off + i + (int64_t)r * ws_ld, v);
}

template <class TS, class TX, class TY, class TA, int NR, bool VIA_PERM>
__global__ void __launch_bounds__(SW * 32) mv_scatter_kernel(const SymItem* __restrict__ items, int nitems,
                                                              const TS* __restrict__ fac, TA* __restrict__ ws,
                                                              int64_t ws_ld, const int32_t* __restrict__ perm,
                                                              const TX* __restrict__ X, int64_t ldx,
                                                              TY* __restrict__ Y, int64_t ldy) {
    __shared__ TA tile[SW][32][33];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int idx = blockIdx.x * SW + warp;
    if (idx >= nitems) return;
    const SymItem it = items[idx];
    const TS* M = fac + it.m_off;
    TA (*T)[33] = tile[warp];
    for (int i0 = 0; i0 < it.rows; i0 += 32) {
        const int i = i0 + lane;
        const bool rin = i < it.rows;
        TA xt[NR], yt[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            yt[r] = (TA)0;
            xt[r] = (!it.diag && rin) ? sc_in<TA, TX, VIA_PERM>(X, ldx, ws, ws_ld, perm, it.in_t, i, r) : (TA)0;
        }
        for (int j0 = 0; j0 < it.cols; j0 += 32) {
            const int jl = j0 + lane;
            const bool cin = jl < it.cols;
            TA xs[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r)
                xs[r] = cin ? sc_in<TA, TX, VIA_PERM>(X, ldx, ws, ws_ld, perm, it.in_s, jl, r) : (TA)0;
            const int nc = min(32, it.cols - j0);
            if constexpr (sizeof(TS) <= 4) {
                // bandwidth-bound storage: the whole 32 x 32 tile is requested before any of it is
                // used (32 independent coalesced loads per warp in flight)
                TS dv[32];
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    dv[c] = TS(0);
                    if (rin && c < nc) dv[c] = M[i + (int64_t)(j0 + c) * it.ldm];
                }
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const TA d = cvt<TA>(dv[c]);
                    T[c][lane] = d;
#pragma unroll
                    for (int r = 0; r < NR; ++r) yt[r] = fma(d, __shfl_sync(0xffffffffu, xs[r], c), yt[r]);
                }
            } else {
                // FP64 storage is FP64-pipe bound: loop over the tile's actual columns only (a
                // coupling block of rank k < 32 costs k, not 32, FP64 instructions per lane)
#pragma unroll 4
                for (int c = 0; c < nc; ++c) {
                    TA d = (TA)0;
                    if (rin) d = cvt<TA>(M[i + (int64_t)(j0 + c) * it.ldm]);
                    T[c][lane] = d;
#pragma unroll
                    for (int r = 0; r < NR; ++r) yt[r] = fma(d, __shfl_sync(0xffffffffu, xs[r], c), yt[r]);
                }
            }
            if (!it.diag) {
                __syncwarp();
                TA ys[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) ys[r] = (TA)0;
                // rows of this tile (the FP32 path fills all 32, with zeros beyond the block)
                const int nr = (sizeof(TS) <= 4) ? 32 : min(32, it.rows - i0);
#pragma unroll 4
                for (int row = 0; row < nr; ++row) {
                    const TA d = T[lane][row];
#pragma unroll
                    for (int r = 0; r < NR; ++r) ys[r] = fma(d, __shfl_sync(0xffffffffu, xt[r], row), ys[r]);
                }
                if (cin)
#pragma unroll
                    for (int r = 0; r < NR; ++r) sc_add<TA, TY, VIA_PERM>(Y, ldy, ws, ws_ld, perm, it.out_s, jl, r, ys[r]);
            }
            __syncwarp();
        }
        if (rin)
#pragma unroll
            for (int r = 0; r < NR; ++r) sc_add<TA, TY, VIA_PERM>(Y, ldy, ws, ws_ld, perm, it.out_t, i, r, yt[r]);
    }
}

template <class TS, class TX, class TY, class TA, int NR>
void launch_scatter_nr(const SymStage& st, const TS* fac, TA* ws, int64_t ws_ld, const int32_t* perm, const TX* X,
                       int64_t ldx, TY* Y, int64_t ldy, cudaStream_t s) {
    const unsigned grid = (unsigned)((st.items.size() + SW - 1) / SW);
    if (st.via_perm)
        mv_scatter_kernel<TS, TX, TY, TA, NR, true><<<grid, SW * 32, 0, s>>>(st.d_items.p, (int)st.items.size(), fac,
                                                                             ws, ws_ld, perm, X, ldx, Y, ldy);
    else
        mv_scatter_kernel<TS, TX, TY, TA, NR, false><<<grid, SW * 32, 0, s>>>(st.d_items.p, (int)st.items.size(), fac,
                                                                              ws, ws_ld, perm, X, ldx, Y, ldy);
    after_launch(st.via_perm ? "mv_near_scatter" : "mv_couple_scatter");
}

template <class TS, class TX, class TY, class TA>
void launch_scatter(const SymStage& st, const TS* fac, TA* ws, int64_t ws_ld, const int32_t* perm, const TX* X,
                    int64_t ldx, TY* Y, int64_t ldy, int nrhs, cudaStream_t s) {
    if (st.items.empty()) return;
    switch (nrhs) {
        case 1: launch_scatter_nr<TS, TX, TY, TA, 1>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        case 2: launch_scatter_nr<TS, TX, TY, TA, 2>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        case 3: launch_scatter_nr<TS, TX, TY, TA, 3>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        default: launch_scatter_nr<TS, TX, TY, TA, 4>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
    }
}

template <class TS, class TX, class TY, class TA, int NR>
void launch_small_stage_nr(const MvStage& st, const TS* fac, TA* ws, int64_t ws_ld, const int32_t* perm,
                           const TX* X, int64_t ldx, TY* Y, int64_t ldy, cudaStream_t s) {
    const int n = (int)st.outs.size();
    const unsigned grid = (unsigned)((n + 7) / 8);
    if (st.out_to_y)
        mv_small_stage_kernel<TS, TX, TY, TA, true, NR><<<grid, 256, 0, s>>>(st.d_outs.p, n, st.d_items.p, fac, ws,
                                                                             ws_ld, perm, X, ldx, Y, ldy, st.accumulate);
    else
        mv_small_stage_kernel<TS, TX, TY, TA, false, NR><<<grid, 256, 0, s>>>(st.d_outs.p, n, st.d_items.p, fac, ws,
                                                                              ws_ld, perm, X, ldx, Y, ldy, st.accumulate);
    after_launch("mv_small_stage");
}

template <class TS, class TX, class TY, class TA>
void launch_small_stage(const MvStage& st, const TS* fac, TA* ws, int64_t ws_ld, const int32_t* perm, const TX* X,
                        int64_t ldx, TY* Y, int64_t ldy, int nrhs, cudaStream_t s) {
    if (st.outs.empty()) return;
    switch (nrhs) {
        case 1: launch_small_stage_nr<TS, TX, TY, TA, 1>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        case 2: launch_small_stage_nr<TS, TX, TY, TA, 2>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        case 3: launch_small_stage_nr<TS, TX, TY, TA, 3>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
        default: launch_small_stage_nr<TS, TX, TY, TA, 4>(st, fac, ws, ws_ld, perm, X, ldx, Y, ldy, s); break;
    }
}

template <class TS, class TX, class TY, class TA>
void launch_stage(const MvStage& st, const TS* fac, TA* ws, int64_t ws_ld, const int32_t* perm,
                  const TX* X, int64_t ldx, TY* Y, int64_t ldy, int nrhs, cudaStream_t s) {
    if (st.outs.empty()) return;
    // tree sweeps with at least half a tile of right-hand sides: one thread per right-hand side
    if ((st.kind == H2_STAGE_UP || st.kind == H2_STAGE_DOWN) && !st.out_to_y && !st.in_from_x &&
        nrhs >= TR_RC / 2 && (nrhs + TR_RC - 1) / TR_RC <= 65535) {
        const int kb = std::max(st.max_rows, st.max_cols);
        if (kb <= 32) { launch_transfer<TS, TA, 32>(st, fac, ws, ws_ld, nrhs, s); return; }
        if (kb <= 64) { launch_transfer<TS, TA, 64>(st, fac, ws, ws_ld, nrhs, s); return; }
    }
    const size_t smem = (size_t)(RMAX * (RMAX + 1) + RMAX * RT) * sizeof(TA);
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(mv_stage_kernel<TS, TX, TY, TA>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        H2_CUDA(cudaFuncSetAttribute(mv_leaf_near_kernel<TS, TX, TY, TA>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    });
    dim3 grid((unsigned)st.outs.size(), (unsigned)((nrhs + RT - 1) / RT));
    if (st.out_to_y) {
        mv_leaf_near_kernel<TS, TX, TY, TA><<<grid, NT, smem, s>>>(st.d_outs.p, st.d_items.p, fac, ws, ws_ld, perm,
                                                                   X, ldx, Y, ldy, nrhs, st.accumulate);
        after_launch("mv_leaf_near");
    } else {
        mv_stage_kernel<TS, TX, TY, TA><<<grid, NT, smem, s>>>(st.d_outs.p, st.d_items.p, fac, ws, ws_ld, perm, X,
                                                               ldx, Y, ldy, nrhs, st.accumulate);
        after_launch("mv_stage");
    }
}

cudaEvent_t take_event(h2_handle_s* h) {
    if (h->ev_pool.empty()) {
        cudaEvent_t e;
        H2_CUDA(cudaEventCreate(&e));
        return e;
    }
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
}

constexpr int kSmallNrhs = 4;

template <class TS, class TX, class TY, class TA>
void run_small(h2_handle_s* h, const TS* fac, TA* ws, const TX* X, int64_t ldx, TY* Y, int64_t ldy, int nrhs,
               cudaStream_t s, bool prof, bool may_fork) {
    const MatvecPlan& P = h->plan;
    const int64_t wld = P.ws_rows;
    auto timed = [&](int kind, auto&& fn) {
        if (!prof) { fn(); return; }
        cudaEvent_t a = take_event(h), b = take_event(h);
        H2_CUDA(cudaEventRecord(a, s));
        fn();
        H2_CUDA(cudaEventRecord(b, s));
        h->ev_used.push_back({kind, {a, b}});
    };
    // Y and yh start at zero: the scatter stages add into them
    H2_CUDA(cudaMemset2DAsync(Y, ldy * sizeof(TY), 0, h->N * sizeof(TY), nrhs, s));
    if (wld > P.yh_row0)
        H2_CUDA(cudaMemset2DAsync(ws + P.yh_row0, wld * sizeof(TA), 0, (wld - P.yh_row0) * sizeof(TA), nrhs, s));
    // The near field (the bulk of the arithmetic, independent of the coefficient sweeps) runs
    // beside the latency-bound chain of tree stages; both add into Y atomically.  The chain goes
    // to a second stream of the highest priority, so that each of its small launches takes SMs
    // ahead of the near field's remaining CTAs instead of queueing behind them; the near field
    // stays on the caller's stream.  Profiled calls keep one stream so that every stage is timed
    // on its own.
    const bool overlap = may_fork && !prof && !P.near.items.empty();
    cudaStream_t cs = s;   // the chain's stream
    if (overlap) {
        if (!h->side) fail(H2_ERR_CUDA, "matvec: the handle's second stream is missing");
        H2_CUDA(cudaEventRecord(h->ev_fork, s));
        H2_CUDA(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
        cs = h->side;
    }
    for (const MvStage& st : P.small_up)
        timed(st.kind, [&] { launch_small_stage<TS, TX, TY, TA>(st, fac, ws, wld, h->d_perm.p, X, ldx, Y, ldy, nrhs, cs); });
    timed(H2_STAGE_COUPLE, [&] { launch_scatter<TS, TX, TY, TA>(P.couple, fac, ws, wld, h->d_perm.p, X, ldx, Y, ldy, nrhs, cs); });
    for (const MvStage& st : P.small_down)
        timed(st.kind, [&] { launch_small_stage<TS, TX, TY, TA>(st, fac, ws, wld, h->d_perm.p, X, ldx, Y, ldy, nrhs, cs); });
    timed(H2_STAGE_LEAF_NEAR, [&] {
        launch_small_stage<TS, TX, TY, TA>(P.small_expand, fac, ws, wld, h->d_perm.p, X, ldx, Y, ldy, nrhs, cs);
    });
    if (overlap) H2_CUDA(cudaEventRecord(h->ev_join, cs));
    timed(H2_STAGE_NEAR, [&] { launch_scatter<TS, TX, TY, TA>(P.near, fac, ws, wld, h->d_perm.p, X, ldx, Y, ldy, nrhs, s); });
    if (overlap) H2_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
}

template <class TS, class TX, class TY, class TA>
void run_all(h2_handle_s* h, const TS* fac, TA* ws, const TX* X, int64_t ldx, TY* Y, int64_t ldy,
             int nrhs, cudaStream_t s, bool allow_prof = true) {
    if constexpr (!std::is_same<TA, CF>::value) {   // the compensated form has no atomics: gather at every nrhs
        if (nrhs <= kSmallNrhs) {
            // the no-allocation entry point (allow_prof false) creates no second stream
            run_small<TS, TX, TY, TA>(h, fac, ws, X, ldx, Y, ldy, nrhs, s, allow_prof && h->prof, allow_prof);
            return;
        }
    }
    for (const MvStage& st : h->plan.stages) {
        if (allow_prof && h->prof && !st.outs.empty()) {
            cudaEvent_t a = take_event(h), b = take_event(h);
            H2_CUDA(cudaEventRecord(a, s));
            launch_stage<TS, TX, TY, TA>(st, fac, ws, h->plan.ws_rows, h->d_perm.p, X, ldx, Y, ldy, nrhs, s);
            H2_CUDA(cudaEventRecord(b, s));
            h->ev_used.push_back({st.kind, {a, b}});
        } else {
            launch_stage<TS, TX, TY, TA>(st, fac, ws, h->plan.ws_rows, h->d_perm.p, X, ldx, Y, ldy, nrhs, s);
        }
    }
}

// Scratch of h2_matvec_noalloc: a fixed array in the library's device image, so that
// the entry point needs no allocation.  Every device that loads the library holds it.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 256;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  The name of a __device__
// variable is only a host-side stand-in, so its address is looked up once per device
// (with that device current) and cached.
void* noalloc_scratch() {
    int dev = 0;
    H2_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            fail(H2_ERR_CUDA, std::string("h2_matvec_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = p;
    }
    return g_scratch_addr[dev];
}

constexpr int kTcMinNrhs = 64;

// Tensor-core path: leaf upsweep, couplings and near field + leaf expansion on tcgen05; the
// transfer upsweep and downsweep on the SIMT stage kernels.
template <class TS, class TX>
void run_tc(h2_handle_s* h, int mode, const TS* fac, float* ws, const TX* X, int64_t ldx, float* Y, int64_t ldy,
            int nrhs, cudaStream_t s) {
    const MatvecPlan& P = h->plan;
    const bool prof = h->prof;
    std::function<void(int, std::function<void()>)> timed = [&](int kind, std::function<void()> fn) {
        if (!prof) { fn(); return; }
        cudaEvent_t a = take_event(h), b = take_event(h);
        H2_CUDA(cudaEventRecord(a, s));
        fn();
        H2_CUDA(cudaEventRecord(b, s));
        h->ev_used.push_back({kind, {a, b}});
    };
    // right-hand-side-major coefficient workspace (ws[row * nrhs + rhs]) when the sweeps' blocks fit
    // the register kernel, else the coefficient-major layout of the SIMT stage kernels
    int kb = 0;
    for (const MvStage& st : P.stages)
        if (st.kind == H2_STAGE_UP || st.kind == H2_STAGE_DOWN) kb = std::max({kb, st.max_rows, st.max_cols});
    bool rmaj = kb <= 64 && (nrhs + TR_RC - 1) / TR_RC <= 65535;
    for (const MvStage& st : P.stages)
        if (st.kind == H2_STAGE_UP || st.kind == H2_STAGE_DOWN)
            for (const MvOut& o : st.outs) rmaj = rmaj && o.end - o.beg <= 2;
    const int64_t ws_ld = rmaj ? (int64_t)nrhs : P.ws_rows;
    std::function<void(int)> sweeps = [&](int down) {
        for (const MvStage& st : P.stages) {
            if (st.kind != (down ? H2_STAGE_DOWN : H2_STAGE_UP) || st.outs.empty()) continue;
            timed(st.kind, [&] {
                if (!rmaj)
                    launch_stage<TS, TX, float, float>(st, fac, ws, P.ws_rows, h->d_perm.p, X, ldx, Y, ldy, nrhs, s);
                else if (kb <= 32)
                    launch_transfer_rm<TS, 32>(st, fac, ws, ws_ld, nrhs, s);
                else
                    launch_transfer_rm<TS, 64>(st, fac, ws, ws_ld, nrhs, s);
            });
        }
    };
    tc_matvec(h, mode, X, ldx, Y, ldy, nrhs, ws, ws_ld, rmaj ? 1 : 0, s, sweeps, timed);
}

}  // namespace

void run_matvec_noalloc(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs, int mode,
                        cudaStream_t s) {
    if (nrhs <= 0) return;
    if (nrhs > kMaxNrhs) fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: nrhs above 2,000,000");
    if (mode == H2_FP32C) fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: H2_FP32C is not available here");
    if (mode == H2_TF32 || mode == H2_TF32X3)
        fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: H2_TF32 and H2_TF32X3 need the tensor-core path's operand "
                                 "workspace; use H2_FP32, H2_BF16 or h2_matvec");
    const size_t elt = (mode == H2_FP64) ? sizeof(double) : sizeof(float);
    const size_t need = (size_t)h->plan.ws_rows * (size_t)nrhs * elt;
    if (need > kNoAllocScratchBytes)
        fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: needs " + std::to_string(need) + " bytes of scratch (" +
                                     std::to_string(h->plan.ws_rows) + " coefficient rows x " + std::to_string(nrhs) +
                                     " right-hand sides), above the fixed " + std::to_string(kNoAllocScratchBytes) +
                                     " bytes; use fewer right-hand sides per call or h2_matvec");
    void* ws = noalloc_scratch();
    switch (mode) {
        case H2_FP64:
            run_all<double, double, double, double>(h, h->fac64.p, (double*)ws, (const double*)X, ldx, (double*)Y, ldy,
                                                    (int)nrhs, s, false);
            break;
        case H2_FP32:
            if (!h->fac32.p) fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: FP32 copy of the factors was not kept");
            run_all<float, float, float, float>(h, h->fac32.p, (float*)ws, (const float*)X, ldx, (float*)Y, ldy,
                                                (int)nrhs, s, false);
            break;
        case H2_BF16:
            if (!h->fac16.p) fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: BF16 copy of the factors was not kept");
            run_all<__nv_bfloat16, __nv_bfloat16, float, float>(h, h->fac16.p, (float*)ws, (const __nv_bfloat16*)X,
                                                                ldx, (float*)Y, ldy, (int)nrhs, s, false);
            break;
        default:
            fail(H2_ERR_INVALID_ARG, "h2_matvec_noalloc: mode not supported");
    }
}

namespace {

template <class TS, class TX, class TY, class TA, int RTT>
void launch_batch_t(int out_y, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                    const BatchBase* bases, int nrhs, cudaStream_t s) {
    const size_t smem = (size_t)(RMAX * (RMAX + 1) + RMAX * RTT) * sizeof(TA);
    static std::once_flag once;
    std::call_once(once, [&] {
        H2_CUDA(cudaFuncSetAttribute(mv_batch_stage_kernel<TS, TX, TY, TA, false, RTT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        H2_CUDA(cudaFuncSetAttribute(mv_batch_stage_kernel<TS, TX, TY, TA, true, RTT>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    });
    dim3 grid((unsigned)nouts, (unsigned)((nrhs + RTT - 1) / RTT));
    if (out_y)
        mv_batch_stage_kernel<TS, TX, TY, TA, true, RTT><<<grid, NT, smem, s>>>(outs, items, bases, nrhs, accumulate);
    else
        mv_batch_stage_kernel<TS, TX, TY, TA, false, RTT><<<grid, NT, smem, s>>>(outs, items, bases, nrhs, accumulate);
    after_launch("mv_batch_stage");
}

template <class TS, class TX, class TY, class TA>
void launch_batch_rt(int rt, int out_y, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                     const BatchBase* bases, int nrhs, cudaStream_t s) {
    switch (rt) {
        case 8: launch_batch_t<TS, TX, TY, TA, 8>(out_y, accumulate, outs, nouts, items, bases, nrhs, s); break;
        case 16: launch_batch_t<TS, TX, TY, TA, 16>(out_y, accumulate, outs, nouts, items, bases, nrhs, s); break;
        default: launch_batch_t<TS, TX, TY, TA, 32>(out_y, accumulate, outs, nouts, items, bases, nrhs, s); break;
    }
}

}  // namespace

void launch_batch_transfer_rm(int mode, int kb, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                              const BatchBase* bases, int nrhs, cudaStream_t s) {
    if (nouts <= 0) return;
    const dim3 grid((unsigned)nouts, (unsigned)((nrhs + TR_RC - 1) / TR_RC));
    if (mode == H2_BF16) {
        if (kb <= 32) mv_batch_transfer_rm_kernel<__nv_bfloat16, 32><<<grid, TR_RC, 0, s>>>(outs, items, bases, nrhs, accumulate);
        else mv_batch_transfer_rm_kernel<__nv_bfloat16, 64><<<grid, TR_RC, 0, s>>>(outs, items, bases, nrhs, accumulate);
    } else {
        if (kb <= 32) mv_batch_transfer_rm_kernel<float, 32><<<grid, TR_RC, 0, s>>>(outs, items, bases, nrhs, accumulate);
        else mv_batch_transfer_rm_kernel<float, 64><<<grid, TR_RC, 0, s>>>(outs, items, bases, nrhs, accumulate);
    }
    after_launch("mv_batch_transfer_rm");
}

void launch_batch_stage(int mode, int rt, int out_y, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                        const BatchBase* bases, int nrhs, cudaStream_t s) {
    if (mode == H2_FP64)
        launch_batch_rt<double, double, double, double>(rt, out_y, accumulate, outs, nouts, items, bases, nrhs, s);
    else if (mode == H2_BF16)
        launch_batch_rt<__nv_bfloat16, __nv_bfloat16, float, float>(rt, out_y, accumulate, outs, nouts, items, bases,
                                                                    nrhs, s);
    else
        launch_batch_rt<float, float, float, float>(rt, out_y, accumulate, outs, nouts, items, bases, nrhs, s);
}


void layout_factors(h2_handle_s* h) {
    const h2_tree_s& T = *h->tree;
    const int L = T.L;
    int64_t off = 0;
    h->u_off.assign((size_t)1 << L, 0);
    for (int t = 0; t < (1 << L); ++t) {
        h->u_off[t] = off;
        off += T.size[L][t] * h->k[h->koff[L] + t];
    }
    h->entries_U = off;
    h->uh_off.assign(h->koff[L], 0);  // boxes of levels 0..L-1
    for (int l = 0; l < L; ++l)
        for (int p = 0; p < (1 << l); ++p) {
            const int kc = h->k[h->koff[l + 1] + 2 * p] + h->k[h->koff[l + 1] + 2 * p + 1];
            h->uh_off[h->koff[l] + p] = off;
            off += (int64_t)kc * h->k[h->koff[l] + p];
        }
    h->entries_E = off - h->entries_U;
    const int64_t s0 = off;
    h->far_lower.assign(L + 1, {});
    h->s_off.assign(L + 1, {});
    for (int l = 1; l <= L; ++l)
        for (auto [t, s] : T.far[l])
            if (t > s) {
                h->far_lower[l].push_back({t, s});
                h->s_off[l].push_back(off);
                off += (int64_t)h->k[h->koff[l] + t] * h->k[h->koff[l] + s];
            }
    h->entries_S = off - s0;
    const int64_t d0 = off;
    h->near_lower.clear();
    h->d_off.clear();
    for (auto [t, s] : T.near)
        if (t >= s) {
            h->near_lower.push_back({t, s});
            h->d_off.push_back(off);
            off += T.size[L][t] * T.size[L][s];
        }
    h->entries_D = off - d0;
    h->fac_entries = off;
    h->fac64.reserve((size_t)std::max<int64_t>(off, 1));
}

constexpr int64_t kReserveNrhs = 32;

void build_plan(h2_handle_s* h, cudaStream_t s) {
    // Every handle creation looks up the address of h2_matvec_noalloc's scratch array on the
    // current device here, while allocating is still allowed: the lookup loads this file's
    // device module (lazily loaded modules reserve their __device__ arrays when they load),
    // so that a later h2_matvec_noalloc call never triggers that reservation.
    noalloc_scratch();
    const h2_tree_s& T = *h->tree;
    const int L = T.L;
    auto K = [&](int l, int b) { return h->k[h->koff[l] + b]; };
    // coefficient workspace rows: xh of every box, then yh of every box
    std::vector<int64_t> box_row(h->k.size());
    int64_t rows = 0;
    for (size_t i = 0; i < h->k.size(); ++i) {
        box_row[i] = rows;
        rows += h->k[i];
    }
    const int64_t ytop = rows;
    rows *= 2;
    MatvecPlan& P = h->plan;
    P.ws_rows = std::max<int64_t>(rows, 1);
    P.yh_row0 = ytop;
    // the FP64 coefficient workspace for up to kReserveNrhs right-hand sides is reserved with the
    // handle, so that a first h2_matvec with few right-hand sides does not allocate
    h->ws.f64.reserve((size_t)P.ws_rows * kReserveNrhs);
    // the second stream of the small-nrhs matvec (highest priority: it carries the tree-stage
    // chain beside the near field) and its events, created with the handle
    if (!h->side) {
        int least = 0, greatest = 0;
        H2_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        H2_CUDA(cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, greatest));
        H2_CUDA(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        H2_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
    }
    auto xrow = [&](int l, int b) { return box_row[h->koff[l] + b]; };
    auto yrow = [&](int l, int b) { return ytop + box_row[h->koff[l] + b]; };
    const int64_t wld = P.ws_rows;
    P.stages.clear();
    P.small_up.clear();
    P.small_down.clear();
    auto add_out = [&](MvStage& st, int64_t off, int nrows) {
        st.outs.push_back(MvOut{off, (int)wld, nrows, (int)st.items.size(), (int)st.items.size()});
    };
    auto add_item = [&](MvStage& st, int64_t moff, int ldm, int r, int c, int trans, int64_t in_off) {
        if (r <= 0 || c <= 0) return;
        st.items.push_back(MvItem{moff, in_off, ldm, r, c, trans, (int)wld});
        st.outs.back().end = (int)st.items.size();
    };
    auto make_leaf_up = [&](MvStage& st) {
        st.kind = H2_STAGE_LEAF_UP;
        for (int t = 0; t < (1 << L); ++t) {
            const int kt = K(L, t), m = (int)T.size[L][t];
            if (!kt) continue;
            add_out(st, xrow(L, t), kt);
            add_item(st, h->u_off[t], m, kt, m, 1 | 2, T.start[L][t]);
        }
    };
    auto make_up = [&](MvStage& st, int l) {
        st.kind = H2_STAGE_UP;
        for (int p = 0; p < (1 << l); ++p) {
            const int kp = K(l, p);
            if (!kp) continue;
            const int k1 = K(l + 1, 2 * p), k2 = K(l + 1, 2 * p + 1);
            add_out(st, xrow(l, p), kp);
            const int64_t uo = h->uh_off[h->koff[l] + p];
            add_item(st, uo, k1 + k2, kp, k1, 1, xrow(l + 1, 2 * p));
            add_item(st, uo + k1, k1 + k2, kp, k2, 1, xrow(l + 1, 2 * p + 1));
        }
    };
    auto make_down = [&](MvStage& st, int l) {
        st.kind = H2_STAGE_DOWN;
        st.accumulate = 1;
        for (int c = 0; c < (1 << (l + 1)); ++c) {
            const int kc = K(l + 1, c), p = c >> 1, kp = K(l, p);
            if (!kc || !kp) continue;
            const int k1 = K(l + 1, 2 * p);
            add_out(st, yrow(l + 1, c), kc);
            const int64_t uo = h->uh_off[h->koff[l] + p] + ((c & 1) ? k1 : 0);
            add_item(st, uo, k1 + K(l + 1, 2 * p + 1), kc, kp, 0, yrow(l, p));
        }
    };
    auto make_expand = [&](MvStage& st, bool with_near) {
        st.kind = H2_STAGE_LEAF_NEAR;
        st.out_to_y = 1;
        std::vector<std::vector<int>> near_of(1 << L);
        std::vector<std::vector<int64_t>> mo(1 << L);
        std::vector<std::vector<int>> tr(1 << L);
        if (with_near)
            for (size_t i = 0; i < h->near_lower.size(); ++i) {
                auto [t, s2] = h->near_lower[i];
                near_of[t].push_back(s2); mo[t].push_back(h->d_off[i]); tr[t].push_back(0);
                if (t != s2) { near_of[s2].push_back(t); mo[s2].push_back(h->d_off[i]); tr[s2].push_back(1); }
            }
        for (int t = 0; t < (1 << L); ++t) {
            const int m = (int)T.size[L][t];
            st.outs.push_back(MvOut{T.start[L][t], 0, m, (int)st.items.size(), (int)st.items.size()});
            if (L >= 1) add_item(st, h->u_off[t], m, m, K(L, t), 0, yrow(L, t));
            for (size_t j = 0; j < near_of[t].size(); ++j) {
                const int sb = near_of[t][j], ms = (int)T.size[L][sb];
                const int ldm = tr[t][j] ? ms : m;
                add_item(st, mo[t][j], ldm, m, ms, tr[t][j] | 2, T.start[L][sb]);
            }
        }
    };
    // ---- gather plan (any nrhs) ----
    if (L >= 1) {
        P.stages.emplace_back();
        make_leaf_up(P.stages.back());
        for (int l = L - 1; l >= 1; --l) {
            P.stages.emplace_back();
            make_up(P.stages.back(), l);
        }
        P.stages.emplace_back();
        MvStage& st = P.stages.back();
        st.kind = H2_STAGE_COUPLE;
        for (int l = 1; l <= L; ++l) {
            std::vector<std::vector<int>> far_of(1 << l);
            std::vector<std::vector<int64_t>> mo(1 << l);
            std::vector<std::vector<int>> tr(1 << l);
            for (size_t i = 0; i < h->far_lower[l].size(); ++i) {
                auto [t, s2] = h->far_lower[l][i];
                far_of[t].push_back(s2); mo[t].push_back(h->s_off[l][i]); tr[t].push_back(0);
                far_of[s2].push_back(t); mo[s2].push_back(h->s_off[l][i]); tr[s2].push_back(1);
            }
            for (int t = 0; t < (1 << l); ++t) {
                const int kt = K(l, t);
                if (!kt) continue;
                add_out(st, yrow(l, t), kt);   // every box with a basis gets an output: yh starts at zero
                for (size_t j = 0; j < far_of[t].size(); ++j) {
                    const int sb = far_of[t][j], ks = K(l, sb);
                    const int ldm = tr[t][j] ? ks : kt;   // stored block is k_max x k_min, ld k_max
                    add_item(st, mo[t][j], ldm, kt, ks, tr[t][j], xrow(l, sb));
                }
            }
        }
        for (int l = 1; l <= L - 1; ++l) {
            P.stages.emplace_back();
            make_down(P.stages.back(), l);
        }
    }
    P.stages.emplace_back();
    make_expand(P.stages.back(), true);
    // ---- small-nrhs plan ----
    if (L >= 1) {
        P.small_up.emplace_back();
        make_leaf_up(P.small_up.back());
        for (int l = L - 1; l >= 1; --l) {
            P.small_up.emplace_back();
            make_up(P.small_up.back(), l);
        }
        for (int l = 1; l <= L - 1; ++l) {
            P.small_down.emplace_back();
            make_down(P.small_down.back(), l);
        }
    }
    P.small_expand = MvStage();
    make_expand(P.small_expand, false);
    P.small_expand.accumulate = 1;
    P.couple = SymStage();
    P.couple.kind = H2_STAGE_COUPLE;
    for (int l = 1; l <= L; ++l)
        for (size_t i = 0; i < h->far_lower[l].size(); ++i) {
            auto [t, s2] = h->far_lower[l][i];
            const int kt = K(l, t), ks = K(l, s2);
            if (!kt || !ks) continue;
            P.couple.items.push_back(SymItem{h->s_off[l][i], xrow(l, s2), yrow(l, t), xrow(l, t), yrow(l, s2), kt, kt, ks, 0});
        }
    P.near = SymStage();
    P.near.kind = H2_STAGE_NEAR;
    P.near.via_perm = 1;
    for (size_t i = 0; i < h->near_lower.size(); ++i) {
        auto [t, s2] = h->near_lower[i];
        const int mt = (int)T.size[L][t], ms = (int)T.size[L][s2];
        P.near.items.push_back(SymItem{h->d_off[i], T.start[L][s2], T.start[L][t], T.start[L][t], T.start[L][s2], mt, mt,
                                       ms, t == s2 ? 1 : 0});
    }
    Stager stg;
    auto up_stage = [&](MvStage& st) {
        st.max_rows = st.max_cols = 0;
        for (auto& it : st.items) {
            if (it.rows > RMAX || it.cols > RMAX) fail(H2_ERR_INVALID_ARG, "matvec: block larger than 96");
            if (it.trans & 2) st.in_from_x |= 1;
            st.max_rows = std::max(st.max_rows, it.rows);
            st.max_cols = std::max(st.max_cols, it.cols);
        }
        for (auto& o : st.outs) st.max_rows = std::max(st.max_rows, o.rows);
        upload(st.d_outs, st.outs, s, stg);
        upload(st.d_items, st.items, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
    };
    for (MvStage& st : P.stages) up_stage(st);
    for (MvStage& st : P.small_up) up_stage(st);
    for (MvStage& st : P.small_down) up_stage(st);
    up_stage(P.small_expand);
    for (SymStage* ss : {&P.couple, &P.near}) {
        for (auto& it : ss->items)
            if (it.rows > RMAX || it.cols > RMAX) fail(H2_ERR_INVALID_ARG, "matvec: block larger than 96");
        upload(ss->d_items, ss->items, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
    }
}

void profile_read(h2_handle_s* h, double* ms, int64_t* n) {
    H2_CUDA(cudaDeviceSynchronize());
    for (auto& u : h->ev_used) {
        float t = 0.f;
        H2_CUDA(cudaEventElapsedTime(&t, u.second.first, u.second.second));
        h->prof_ms[u.first] += t;
        h->prof_n[u.first] += 1;
        h->ev_pool.push_back(u.second.first);
        h->ev_pool.push_back(u.second.second);
    }
    h->ev_used.clear();
    for (int k = 0; k < H2_STAGE_COUNT; ++k) {
        if (ms) ms[k] = h->prof_ms[k];
        if (n) n[k] = h->prof_n[k];
        h->prof_ms[k] = 0.0;
        h->prof_n[k] = 0;
    }
}

void make_copies(h2_handle_s* h, int keep_fp32, int keep_bf16, cudaStream_t s) {
    const int64_t n = std::max<int64_t>(h->fac_entries, 1);
    const unsigned grid = (unsigned)std::min<int64_t>((n + NT - 1) / NT, 152 * 16);
    if (keep_fp32) {
        h->fac32.reserve(n);
        convert_kernel<float, float><<<grid, NT, 0, s>>>(h->fac64.p, h->fac32.p, n);
        after_launch("convert_fp32");
    }
    if (keep_bf16) {
        h->fac16.reserve(n);
        convert_kernel<__nv_bfloat16, float><<<grid, NT, 0, s>>>(h->fac64.p, h->fac16.p, n);
        after_launch("convert_bf16");
    }
    tc_prepare(h, keep_bf16, keep_fp32, s);
}

namespace {

// Reserves the buffers of a call and returns the function that enqueues its launches.
std::function<void(cudaStream_t)> matvec_launches(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy,
                                                  int64_t nrhs, int mode) {
    const int64_t need = h->plan.ws_rows * nrhs;
    switch (mode) {
        case H2_FP64:
            h->ws.f64.reserve((size_t)need);
            return [=](cudaStream_t s) {
                run_all<double, double, double, double>(h, h->fac64.p, h->ws.f64.p, (const double*)X, ldx, (double*)Y,
                                                        ldy, (int)nrhs, s);
            };
        case H2_FP32:
        case H2_TF32:
        case H2_TF32X3: {
            if (!h->fac32.p) fail(H2_ERR_INVALID_ARG, "h2_matvec: FP32 copy of the factors was not kept");
            h->ws.f32.reserve((size_t)need);
            if (mode != H2_FP32 && nrhs >= kTcMinNrhs && tc_supported(h) && h->tc.W32.p) {
                tc_reserve(h, mode, (int)nrhs);
                return [=](cudaStream_t s) {
                    run_tc<float, float>(h, mode, h->fac32.p, h->ws.f32.p, (const float*)X, ldx, (float*)Y, ldy,
                                         (int)nrhs, s);
                };
            }
            return [=](cudaStream_t s) {
                run_all<float, float, float, float>(h, h->fac32.p, h->ws.f32.p, (const float*)X, ldx, (float*)Y, ldy,
                                                    (int)nrhs, s);
            };
        }
        case H2_FP32C: {
            if (!h->fac32.p) fail(H2_ERR_INVALID_ARG, "h2_matvec: FP32 copy of the factors was not kept");
            h->ws.f64.reserve((size_t)need);   // one CF (two floats) per coefficient
            return [=](cudaStream_t s) {
                run_all<float, double, double, CF>(h, h->fac32.p, reinterpret_cast<CF*>(h->ws.f64.p), (const double*)X,
                                                   ldx, (double*)Y, ldy, (int)nrhs, s);
            };
        }
        case H2_BF16: {
            if (!h->fac16.p) fail(H2_ERR_INVALID_ARG, "h2_matvec: BF16 copy of the factors was not kept");
            h->ws.f32.reserve((size_t)need);
            if (nrhs >= kTcMinNrhs && tc_supported(h) && h->tc.W16.p) {
                tc_reserve(h, mode, (int)nrhs);
                return [=](cudaStream_t s) {
                    run_tc<__nv_bfloat16, __nv_bfloat16>(h, mode, h->fac16.p, h->ws.f32.p, (const __nv_bfloat16*)X,
                                                         ldx, (float*)Y, ldy, (int)nrhs, s);
                };
            }
            return [=](cudaStream_t s) {
                run_all<__nv_bfloat16, __nv_bfloat16, float, float>(h, h->fac16.p, h->ws.f32.p, (const __nv_bfloat16*)X,
                                                                    ldx, (float*)Y, ldy, (int)nrhs, s);
            };
        }
        default:
            fail(H2_ERR_INVALID_ARG, "h2_matvec: mode not supported");
    }
}

constexpr size_t kMaxGraphs = 8;

}  // namespace

// The launch sequence of a repeated call (same buffers, sizes and mode) is captured in a CUDA
// graph on its second occurrence and replayed afterwards, so that the many small launches of a
// few-right-hand-side product are not paced by the host.  Profiled calls always launch directly.
void run_matvec_host(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs, int mode,
                     cudaStream_t s) {
    if (nrhs <= 0) return;
    if (nrhs > kMaxNrhs) fail(H2_ERR_INVALID_ARG, "h2_matvec_host: nrhs above 2,000,000");
    const bool f64io = mode == H2_FP64 || mode == H2_FP32C;
    const size_t ex = f64io ? 8 : (mode == H2_BF16 ? 2 : 4);
    const size_t ey = f64io ? 8 : 4;
    const size_t n = (size_t)h->N;
    h->host_x.reserve(n * ex * (size_t)nrhs);
    h->host_y.reserve(n * ey * (size_t)nrhs);
    H2_CUDA(cudaMemcpy2DAsync(h->host_x.p, n * ex, X, (size_t)ldx * ex, n * ex, (size_t)nrhs, cudaMemcpyHostToDevice, s));
    run_matvec(h, h->host_x.p, h->N, h->host_y.p, h->N, nrhs, mode, s);
    H2_CUDA(cudaMemcpy2DAsync(Y, (size_t)ldy * ey, h->host_y.p, n * ey, n * ey, (size_t)nrhs, cudaMemcpyDeviceToHost, s));
    H2_CUDA(cudaStreamSynchronize(s));
}

void run_matvec(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs,
                int mode, cudaStream_t s) {
    if (nrhs <= 0) return;
    if (nrhs > kMaxNrhs) fail(H2_ERR_INVALID_ARG, "h2_matvec: nrhs above 2,000,000");
    auto launch = matvec_launches(h, X, ldx, Y, ldy, nrhs, mode);
    if (h->prof) {
        launch(s);
        return;
    }
    const void* ws = (mode == H2_FP64 || mode == H2_FP32C) ? (const void*)h->ws.f64.p : (const void*)h->ws.f32.p;
    const void* opnd = h->tc.opnd.p;
    MvGraph* g = nullptr;
    for (auto& e : h->graphs)
        if (e.X == X && e.Y == Y && e.ws == ws && e.opnd == opnd && e.ldx == ldx && e.ldy == ldy && e.nrhs == nrhs &&
            e.mode == mode)
            g = &e;
    if (!g) {
        if (h->graphs.size() >= kMaxGraphs) {
            auto old = std::min_element(h->graphs.begin(), h->graphs.end(),
                                        [](const MvGraph& a, const MvGraph& b) { return a.stamp < b.stamp; });
            if (old->exec) cudaGraphExecDestroy(old->exec);
            if (old->graph) cudaGraphDestroy(old->graph);
            h->graphs.erase(old);
        }
        MvGraph e;
        e.X = X;
        e.Y = Y;
        e.ws = ws;
        e.opnd = opnd;
        e.ldx = ldx;
        e.ldy = ldy;
        e.nrhs = nrhs;
        e.mode = mode;
        h->graphs.push_back(e);
        g = &h->graphs.back();
    }
    g->stamp = ++h->graph_clock;
    ++g->uses;
    if (!g->exec && g->uses >= 2) {
        if (!h->cap) H2_CUDA(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
        const int64_t l0 = g_launches.load();
        H2_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
        try {
            launch(h->cap);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(h->cap, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        H2_CUDA(cudaStreamEndCapture(h->cap, &g->graph));
        // node priorities kept: the small-nrhs chain's launches come from its high-priority stream
        H2_CUDA(cudaGraphInstantiate(&g->exec, g->graph, cudaGraphInstantiateFlagUseNodePriority));
        g->launches = g_launches.load() - l0;
        g_launches.fetch_sub(g->launches);   // counted again at every replay
    }
    if (g->exec) {
        H2_CUDA(cudaGraphLaunch(g->exec, s));
        g_launches.fetch_add(g->launches);
    } else {
        launch(s);
    }
}

}  // namespace h2
