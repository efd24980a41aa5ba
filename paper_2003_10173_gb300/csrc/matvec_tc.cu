// Multi-RHS matvec products on the 5th-generation tensor cores (tcgen05), BF16 or TF32 operands
// with FP32 accumulation in tensor memory (the precision pattern: the multi-RHS basis,
// coupling and near-field products at reduced precision, everything else in FP32/FP64).
//
// Three block-sparse product lists, each output a tile of 128 right-hand sides:
//   leaf upsweep     xh_t^T = X_t^T U_t                    (N = k_t, K = leaf rows)
//   couplings        yh_t^T = sum_s xh_s^T S_ts^T           (N = k_t, K = k_s)
//   near + leaves    Y_t^T  = sum_s X_s^T op(D_ts)^T + yh_t^T U_t^T   (N = leaf rows)
// computed as chains of 128 x N x K MMAs (M = right-hand sides).  A operands are rows of one
// padded operand buffer (X in tree order, xh and yh of every box, K-major per right-hand
// side); B operands are the factors' blocks, one tile per use, pre-rounded and pre-laid out
// in the canonical K-major core-matrix layout so that a tile load is a contiguous copy.
// A producer thread stages each item's A and B tiles in shared memory with bulk asynchronous
// copies (cp.async.bulk, completion counted in bytes on a per-stage mbarrier) into a ring of
// 2 stages (so that several CTAs share an SM and one CTA's epilogue overlaps another's main loop);
// a thread of another warp issues the MMAs as the operands land and commits them to a per-stage
// mbarrier that releases the stage to the producer.  The accumulator is read
// with tcgen05.ld, transposed through shared memory and written to Y (through the tree
// permutation) or to the coefficient workspace.  Every mbarrier wait is bounded: on timeout
// the kernel records a device error, drains its copies, frees its tensor memory and returns.
#include <algorithm>
#include <functional>

#include <mutex>

#include "handle.h"

namespace h2 {

namespace {

constexpr int TC_M = 128;      // right-hand sides per CTA (MMA M)
constexpr int TC_THREADS = 128;
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // about one second
constexpr int TC_ITEM_CACHE = 256;                   // item descriptors staged in shared memory

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Canonical K-major, no-swizzle position (bytes) of element (row, k): 8-row x 16-byte core
// matrices, consecutive along K (LBO = 128 B), core-matrix rows SBO = (K bytes / 16) * 128 B apart.
template <int EB>
__host__ __device__ __forceinline__ uint32_t kmaj_off(int row, int k, int kdim) {
    constexpr int EPC = 16 / EB;   // elements per 16-byte core row
    return (uint32_t)(((row >> 3) * (kdim / EPC) + (k / EPC)) * 128 + (row & 7) * 16 + (k % EPC) * EB);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of tcgen05; no swizzle, base offset 0
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok)
                     : "r"(bar), "r"(parity));
        if (ok) return true;
        if (clock64() - t0 > TC_WAIT_CYCLES) {
            atomicExch(err, 1);
            return false;
        }
    }
}

template <int EB>
struct TcTraits;
template <>
struct TcTraits<2> {   // BF16 operands, kind::f16, K = 16 per MMA
    static constexpr int KSTEP = 16;
    static constexpr uint32_t ab_fmt = 1;   // BF16
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
};
template <>
struct TcTraits<4> {   // TF32 operands, kind::tf32, K = 8 per MMA
    static constexpr int KSTEP = 8;
    static constexpr uint32_t ab_fmt = 2;   // TF32
    __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc));
    }
};

// Block-sparse product list on tensor cores.  Output o (N_o rows, padded to 16) for a tile of
// 128 right-hand sides: acc[r][i] = sum over items of A_item[r][k] * B_item[i][k], with
//   A_item = rows [a_row, a_row + K) of the padded operand buffer (K-major: rows are contiguous
//            per right-hand side), and
//   B_item = a pre-laid-out N_o x K tile of the tile pool.
// Two kernels run these lists: tc_products_kernel (one output per CTA; the near field + leaf
// expansion, written to Y through the tree permutation via a shared-memory transpose) and
// tc_group_kernel (several coefficient outputs per CTA; the leaf upsweep and the couplings,
// stored to the coefficient workspace straight from tensor memory).
constexpr int TC_NMAX = 64, TC_KMAX = 64;
constexpr int TC_GCOLS = 128;   // tensor-memory columns of a CTA: its outputs side by side (4 CTAs per SM)
constexpr int TC_GMAX = 8;      // outputs per CTA
constexpr int TC_GROUP_ITEMS = 84;   // items per CTA group (x3 for split TF32 <= TC_ITEM_CACHE)

// Operand ring: S stages, each an A tile (128 x KM) and a B tile (NM x KM).  64 x 64 tiles in two
// stages for the leaf upsweep and the near field; items of at most 48 x 48 (the couplings) in
// three stages of the same total size, so that more copies are in flight per CTA.
template <int EB, int KM = TC_KMAX, int NM = TC_NMAX, int S = 2>
struct TcCfg {
    static constexpr int STAGES = S;
    static constexpr int KMAX = KM, NMAX = NM;
    static constexpr int A_BYTES = TC_M * KM * EB;
    static constexpr int B_BYTES = NM * KM * EB;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int SMEM = STAGES * STAGE_BYTES;
    // item descriptors cached in shared memory by the grouped kernel: a group holds at most
    // TC_GROUP_ITEMS items, three times that in split TF32; the smaller BF16 cache keeps four
    // three-stage CTAs per SM
    static constexpr int CACHE = (EB == 2) ? 96 : 256;
    static_assert(STAGE_BYTES % 128 == 0, "stages must stay 128-byte aligned");
};

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// One output per CTA (the near field + leaf expansion: outputs are rows of Y through the
// permutation, transposed through shared memory).
template <int EB>
__global__ void __launch_bounds__(TC_THREADS) tc_products_kernel(
    const TcOut* __restrict__ outs, const TcItem* __restrict__ items, const unsigned char* __restrict__ W,
    const unsigned char* __restrict__ opnd, const int32_t* __restrict__ perm, float* __restrict__ Y, int64_t ldy,
    float* __restrict__ ws, int64_t ws_ld, int nrhs, int* __restrict__ err) {
    using Tr = TcTraits<EB>;
    using C = TcCfg<EB>;
    constexpr int S = C::STAGES;
    constexpr int TMEM_COLS = 64;   // one output of at most TC_NMAX columns
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ uint32_t tmem_slot;
    __shared__ int okflag, prod_issued, cons_done;
    __shared__ TcItem sitems[TC_ITEM_CACHE];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int rt = blockIdx.x;
    const int r0 = rt * TC_M;
    const TcOut o = outs[blockIdx.y];
    const int nitem = o.end - o.beg;
    const int N = o.n;

    // the output's item descriptors, staged once in shared memory (off the producer's critical path)
    const bool cached = nitem <= TC_ITEM_CACHE;
    if (cached)
        for (int i = tid; i < nitem; i += TC_THREADS) sitems[i] = items[o.beg + i];
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
        }
        okflag = 1;
        prod_issued = 0;
        cons_done = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    auto item_at = [&](int it) -> TcItem { return cached ? sitems[it] : items[o.beg + it]; };

    // warp-specialised pipeline: thread 0 copies operands into the stage ring, thread 32 issues
    // the MMAs; a stage is refilled as soon as the MMAs that read it have completed
    if (tid == 0) {
        int issued = 0;
        for (; issued < nitem; ++issued) {
            const int st = issued % S;
            if (issued >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((issued / S) - 1) & 1), err)) break;
            const TcItem m = item_at(issued);
            const uint32_t abytes = (uint32_t)(TC_M * m.k * EB);
            const uint32_t bbytes = (uint32_t)(N * m.k * EB);
            const uint32_t sa = smem_u32(smem + st * C::STAGE_BYTES);
            const uint32_t fb = smem_u32(&full[st]);
            mbar_expect(fb, abytes + bbytes);
            // block base (rows) x tiles x 128 columns, then this tile
            const int64_t aoff = ((int64_t)m.a_row * gridDim.x * TC_M + (int64_t)rt * TC_M * m.k) * EB;
            bulk_g2s(sa, opnd + aoff, abytes, fb);
            bulk_g2s(sa + C::A_BYTES, W + m.b_off, bbytes, fb);
        }
        prod_issued = issued;
    } else if (tid == 32) {
        const uint32_t idesc = (1u << 4) | (Tr::ab_fmt << 7) | (Tr::ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) |
                               ((uint32_t)(TC_M >> 4) << 24);
        int it = 0;
        for (; it < nitem; ++it) {
            const int st = it % S;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((it / S) & 1), err)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int K = item_at(it).k;
            const uint32_t a0 = smem_u32(smem + st * C::STAGE_BYTES);
            const uint32_t b0 = a0 + C::A_BYTES;
            const uint32_t SBO = (uint32_t)(K * EB / 16) * 128;
            for (int kk = 0; kk < K / Tr::KSTEP; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, SBO);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, SBO);
                Tr::mma(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&empty[st])));
        }
        cons_done = it;
        // every MMA issued completes before the accumulator is read or released
        if (it > 0 && !mbar_wait(smem_u32(&empty[(it - 1) % S]), (uint32_t)(((it - 1) / S) & 1), err)) it = -1;
        if (it != nitem) okflag = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // copies issued for items that were never consumed land before the memory is reused
        for (int j = cons_done; j < prod_issued; ++j)
            mbar_wait(smem_u32(&full[j % S]), (uint32_t)((j / S) & 1), err);
        if (prod_issued != nitem) okflag = 0;
    }
    __syncthreads();
    const bool ok = okflag != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    float* stage = reinterpret_cast<float*>(smem);
    constexpr int SLD = TC_NMAX + 1;
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < N; c0 += 16) {
            uint32_t v[16];
            if (nitem > 0) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0u;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) stage[r * SLD + c0 + j] = __uint_as_float(v[j]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
    if (!ok) return;
    const int m = o.rows;
    for (int e = tid; e < m * TC_M; e += TC_THREADS) {
        const int i = e % m, r = e / m;
        if (r0 + r >= nrhs) continue;
        const float v = stage[r * SLD + i];
        if (o.to_y) Y[perm[o.out_off + i] + (int64_t)(r0 + r) * ldy] = v;
        else ws[o.out_off + i + (int64_t)(r0 + r) * ws_ld] = v;
    }
}

// Several consecutive coefficient outputs per CTA (leaf upsweep, couplings): one operand ring
// across all their items, each output accumulating in its own columns of tensor memory, stored
// to the workspace straight from the tensor-memory loads.
template <int EB, class C>
__global__ void __launch_bounds__(TC_THREADS) tc_group_kernel(
    const TcGroup* __restrict__ groups, const TcOut* __restrict__ outs, const TcItem* __restrict__ items,
    const unsigned char* __restrict__ W, const unsigned char* __restrict__ opnd, float* __restrict__ ws,
    int64_t ws_ld, int ws_rmaj, int nrhs, int tmem_cols, int* __restrict__ err) {
    using Tr = TcTraits<EB>;
    constexpr int S = C::STAGES;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[S], empty[S];
    __shared__ uint32_t tmem_slot;
    __shared__ int okflag, prod_issued, cons_done;
    __shared__ TcItem sitems[C::CACHE];
    __shared__ TcOut souts[TC_GMAX];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int rt = blockIdx.x;
    const int r0 = rt * TC_M;
    const TcGroup g = groups[blockIdx.y];
    const int nout = g.oend - g.obeg;   // 1..TC_GMAX (host-checked)
    const int ibeg = g.ibeg;
    const int nitem = g.iend - g.ibeg;
    // the group's outputs and item descriptors, staged once in shared memory (off the producer's
    // critical path)
    if (tid < nout) souts[tid] = outs[g.obeg + tid];
    const bool cached = nitem <= C::CACHE;
    if (cached)
        for (int i = tid; i < nitem; i += TC_THREADS) sitems[i] = items[ibeg + i];
    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[i])));
        }
        okflag = 1;
        prod_issued = 0;
        cons_done = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    auto item_at = [&](int it) -> TcItem { return cached ? sitems[it - ibeg] : items[it]; };

    // warp-specialised pipeline over all items of the group's outputs, in output order: thread 0
    // copies operands into the stage ring, thread 32 issues the MMAs into the output's columns of
    // tensor memory; a stage is refilled as soon as the MMAs that read it have completed
    if (tid == 0) {
        int issued = 0;
        bool run = true;
        for (int j = 0; j < nout && run; ++j) {
            const TcOut o = souts[j];
            for (int it = o.beg; it < o.end; ++it) {
                const int st = issued % S;
                if (issued >= S && !mbar_wait(smem_u32(&empty[st]), (uint32_t)(((issued / S) - 1) & 1), err)) {
                    run = false;
                    break;
                }
                const TcItem m = item_at(it);
                const uint32_t abytes = (uint32_t)(TC_M * m.k * EB);
                const uint32_t bbytes = (uint32_t)(o.n * m.k * EB);
                const uint32_t sa = smem_u32(smem + st * C::STAGE_BYTES);
                const uint32_t fb = smem_u32(&full[st]);
                mbar_expect(fb, abytes + bbytes);
                // block base (rows) x tiles x 128 columns, then this tile
                const int64_t aoff = ((int64_t)m.a_row * gridDim.x * TC_M + (int64_t)rt * TC_M * m.k) * EB;
                bulk_g2s(sa, opnd + aoff, abytes, fb);
                bulk_g2s(sa + C::A_BYTES, W + m.b_off, bbytes, fb);
                ++issued;
            }
        }
        prod_issued = issued;
    } else if (tid == 32) {
        int done = 0, col = 0;
        bool run = true;
        for (int j = 0; j < nout && run; ++j) {
            const TcOut o = souts[j];
            const uint32_t idesc = (1u << 4) | (Tr::ab_fmt << 7) | (Tr::ab_fmt << 10) |
                                   ((uint32_t)(o.n >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
            const uint32_t d = tmem + (uint32_t)col;
            col += o.n;
            for (int it = o.beg; it < o.end; ++it) {
                const int st = done % S;
                if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((done / S) & 1), err)) {
                    run = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const int K = item_at(it).k;
                const uint32_t a0 = smem_u32(smem + st * C::STAGE_BYTES);
                const uint32_t b0 = a0 + C::A_BYTES;
                const uint32_t SBO = (uint32_t)(K * EB / 16) * 128;
                for (int kk = 0; kk < K / Tr::KSTEP; ++kk) {
                    const uint64_t ad = smem_desc(a0 + kk * 256, 128, SBO);
                    const uint64_t bd = smem_desc(b0 + kk * 256, 128, SBO);
                    Tr::mma(d, ad, bd, idesc, (it > o.beg || kk > 0) ? 1u : 0u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&empty[st])));
                ++done;
            }
        }
        cons_done = done;
        // every MMA issued completes before the accumulators are read or released
        if (done > 0 && !mbar_wait(smem_u32(&empty[(done - 1) % S]), (uint32_t)(((done - 1) / S) & 1), err))
            done = -1;
        if (done != nitem) okflag = 0;
    }
    __syncthreads();
    if (tid == 0) {
        // copies issued for items that were never consumed land before the memory is reused
        for (int j = cons_done; j < prod_issued; ++j)
            mbar_wait(smem_u32(&full[j % S]), (uint32_t)((j / S) & 1), err);
        if (prod_issued != nitem) okflag = 0;
    }
    __syncthreads();
    const bool ok = okflag != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // coefficient outputs: each thread stores its right-hand side's entries of every block
    // straight from the tensor-memory loads (right-hand-side-major workspace: consecutive
    // threads write consecutive addresses; coefficient-major: each thread a contiguous run)
    const int r = warp * 32 + (tid & 31);
    const bool live = r0 + r < nrhs;
    const int64_t rstep = ws_rmaj ? ws_ld : 1;
    int col = 0;
    for (int j = 0; j < nout && ok; ++j) {
        const TcOut o = souts[j];
        const bool any = o.end > o.beg;
        float* dst = ws_rmaj ? ws + o.out_off * ws_ld + (r0 + r) : ws + o.out_off + (int64_t)(r0 + r) * ws_ld;
        for (int c0 = 0; c0 < o.n; c0 += 16) {
            uint32_t v[16];
            if (any) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(col + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            } else {
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = 0u;
            }
            if (live)
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (c0 + q < o.rows) dst[(int64_t)(c0 + q) * rstep] = __uint_as_float(v[q]);
        }
        col += o.n;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// TF32 rounding (nearest, ties away) as an FP32 bit pattern, and the rounded low part of the rest:
// v = hi + lo + O(2^-22 |v|) (the three-pass "split TF32" products).
__device__ __forceinline__ uint32_t tf32_rna(float f) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
    return u;
}

// B tiles: tile b is op(M) (valid rows x cols, zero padded to n x k) laid out as an n x k
// K-major operand at byte offset dst[b] of the pool.  With lo_off > 0 (TF32 only) the low part
// of every entry goes to the same position lo_off bytes further on.
template <int EB>
__global__ void tc_pack_tiles_kernel(const double* __restrict__ fac, const TcTileSrc* __restrict__ src,
                                     unsigned char* __restrict__ W, int64_t lo_off) {
    const TcTileSrc d = src[blockIdx.x];
    const double* M = fac + d.m_off;
    unsigned char* out = W + d.dst;
    for (int e = threadIdx.x; e < d.n * d.k; e += blockDim.x) {
        const int i = e % d.n, j = e / d.n;
        double v = 0.0;
        if (i < d.rows && j < d.cols) v = d.trans ? M[j + (int64_t)i * d.ldm] : M[i + (int64_t)j * d.ldm];
        const uint32_t o = kmaj_off<EB>(i, j, d.k);
        if constexpr (EB == 2) {
            *reinterpret_cast<__nv_bfloat16*>(out + o) = __double2bfloat16(v);
        } else {
            const float f = (float)v;
            const uint32_t hi = tf32_rna(f);
            *reinterpret_cast<uint32_t*>(out + o) = hi;
            if (lo_off > 0) *reinterpret_cast<uint32_t*>(out + lo_off + o) = tf32_rna(f - __uint_as_float(hi));
        }
    }
}

__device__ __forceinline__ void store_opnd_bf16(unsigned char* dst, float v) {
    *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ void store_opnd_tf32(unsigned char* dst, float v, int64_t lo_off) {
    const uint32_t hi = tf32_rna(v);
    *reinterpret_cast<uint32_t*>(dst) = hi;
    if (lo_off > 0) *reinterpret_cast<uint32_t*>(dst + lo_off) = tf32_rna(v - __uint_as_float(hi));
}

// The operand buffer is tiled: operand block b (K rows: the points of a leaf, or the padded
// coefficients of a box) and right-hand-side tile rt (128 columns) form one contiguous
// 128 x K chunk in the canonical K-major layout, at byte base_b * nrt + rt * 128 * K * EB, where
// base_b is the block's offset in units of 128-column tiles.  A tile load is one bulk copy.
//
// Operand packing: one CTA per (operand block, right-hand-side tile) stages a 128 x PK_KS slice
// of the block in shared memory (coalesced reads along the block's rows), then writes it out
// as whole 16-byte core-matrix rows, consecutive threads to consecutive addresses.
constexpr int PK_KS = 64;        // K columns staged per slice
constexpr int PK_PAD = 4;        // floats of padding per staged row: conflict-free 16-byte reads
constexpr int PK_THREADS = 256;

// Write columns [ks0, ks0 + w) of the staged 128 x K chunk to dst (the chunk's base, K-major).
template <int EB>
__device__ __forceinline__ void pack_store_slice(const float (*tile)[PK_KS + PK_PAD], int K, int ks0, int w,
                                                 unsigned char* __restrict__ dst, int64_t lo_off) {
    constexpr int EPC = 16 / EB;   // elements per 16-byte core row
    const int nkc = w / EPC;
    for (int u = threadIdx.x; u < TC_M * nkc; u += PK_THREADS) {
        const int g = u / (8 * nkc), rem = u - g * 8 * nkc;
        const int kc = rem >> 3, rw = rem & 7;
        const float* src = &tile[g * 8 + rw][kc * EPC];
        unsigned char* o = dst + ((int64_t)(g * (K / EPC) + ks0 / EPC + kc) * 8 + rw) * 16;
        if constexpr (EB == 2) {
            const float4 a = *reinterpret_cast<const float4*>(src);
            const float4 b = *reinterpret_cast<const float4*>(src + 4);
            __nv_bfloat162 q[4] = {__floats2bfloat162_rn(a.x, a.y), __floats2bfloat162_rn(a.z, a.w),
                                   __floats2bfloat162_rn(b.x, b.y), __floats2bfloat162_rn(b.z, b.w)};
            *reinterpret_cast<uint4*>(o) = *reinterpret_cast<const uint4*>(q);
        } else {
            const float4 a = *reinterpret_cast<const float4*>(src);
            const uint4 hi = make_uint4(tf32_rna(a.x), tf32_rna(a.y), tf32_rna(a.z), tf32_rna(a.w));
            *reinterpret_cast<uint4*>(o) = hi;
            if (lo_off > 0)
                *reinterpret_cast<uint4*>(o + lo_off) =
                    make_uint4(tf32_rna(a.x - __uint_as_float(hi.x)), tf32_rna(a.y - __uint_as_float(hi.y)),
                               tf32_rna(a.z - __uint_as_float(hi.z)), tf32_rna(a.w - __uint_as_float(hi.w)));
        }
    }
}

// X (caller order) -> leaf blocks (zero padded rows and right-hand sides); grid (leaves, tiles)
template <class TX, int EB>
__global__ void __launch_bounds__(PK_THREADS) tc_pack_x_kernel(const TX* __restrict__ X, int64_t ldx,
                                                               const int32_t* __restrict__ perm,
                                                               const int64_t* __restrict__ leaf_start,
                                                               const int* __restrict__ leaf_size, int LP, int nrhs,
                                                               unsigned char* __restrict__ opnd, int64_t lo_off) {
    __shared__ __align__(16) float tile[TC_M][PK_KS + PK_PAD];
    const int t = blockIdx.x, rt = blockIdx.y, nrt = gridDim.y;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int m = leaf_size[t];
    const int64_t s0 = leaf_start[t];
    const int r0 = rt * TC_M;
    unsigned char* dst = opnd + ((int64_t)t * LP * TC_M * nrt + (int64_t)rt * TC_M * LP) * EB;
    for (int ks0 = 0; ks0 < LP; ks0 += PK_KS) {
        const int w = min(PK_KS, LP - ks0);
        for (int i = tx; i < w; i += 32) {
            const int p = ks0 + i;
            const int64_t row = p < m ? (int64_t)perm[s0 + p] : -1;
            for (int rr = ty; rr < TC_M; rr += PK_THREADS / 32) {
                float v = 0.f;
                if (row >= 0 && r0 + rr < nrhs) {
                    const TX x = X[row + (int64_t)(r0 + rr) * ldx];
                    if constexpr (std::is_same<TX, __nv_bfloat16>::value) v = __bfloat162float(x);
                    else v = (float)x;
                }
                tile[rr][i] = v;
            }
        }
        __syncthreads();
        pack_store_slice<EB>(tile, LP, ks0, w, dst, lo_off);
        __syncthreads();
    }
}

// coefficient rows of the workspace -> box blocks: box list (block base row, k, kpad); grid
// (boxes, tiles)
template <int EB>
__global__ void __launch_bounds__(PK_THREADS) tc_pack_coef_kernel(const int4* __restrict__ boxes,
                                                                  const float* __restrict__ ws, int64_t ws_ld,
                                                                  int ws_rmaj, const int64_t* __restrict__ src_row,
                                                                  int nrhs, unsigned char* __restrict__ opnd,
                                                                  int64_t lo_off) {
    __shared__ __align__(16) float tile[TC_M][PK_KS + PK_PAD];
    const int b = blockIdx.x, rt = blockIdx.y, nrt = gridDim.y;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int4 d = boxes[b];   // x: block base row, y: k, z: kpad
    const int64_t s0 = src_row[b];
    const int kp = d.z;
    const int r0 = rt * TC_M;
    unsigned char* dst = opnd + ((int64_t)d.x * nrt * TC_M + (int64_t)rt * TC_M * kp) * EB;
    for (int ks0 = 0; ks0 < kp; ks0 += PK_KS) {
        const int w = min(PK_KS, kp - ks0);
        if (ws_rmaj) {
            // right-hand-side-major workspace: lanes run along the right-hand sides
            for (int i = ty; i < w; i += PK_THREADS / 32) {
                const bool valid = ks0 + i < d.y;
                const float* src = ws + (s0 + ks0 + i) * ws_ld + r0;
                for (int rr = tx; rr < TC_M; rr += 32) tile[rr][i] = (valid && r0 + rr < nrhs) ? src[rr] : 0.f;
            }
        } else {
            for (int i = tx; i < w; i += 32) {
                const bool valid = ks0 + i < d.y;
                for (int rr = ty; rr < TC_M; rr += PK_THREADS / 32)
                    tile[rr][i] = (valid && r0 + rr < nrhs) ? ws[s0 + ks0 + i + (int64_t)(r0 + rr) * ws_ld] : 0.f;
            }
        }
        __syncthreads();
        pack_store_slice<EB>(tile, kp, ks0, w, dst, lo_off);
        __syncthreads();
    }
}

template <int EB>
void launch_products(const TcStage& st, const TcGroup* d_groups, const TcOut* d_outs, const TcItem* d_items,
                     const unsigned char* W,
                     const unsigned char* opnd, const int32_t* perm, float* Y, int64_t ldy, float* ws, int64_t ws_ld,
                     int ws_rmaj, int nrhs, int* err, cudaStream_t s) {
    if (st.outs.empty()) return;
    using Big = TcCfg<EB>;
    using Small = TcCfg<EB, 48, 48, 3>;
    const size_t smem = std::max((size_t)Big::SMEM, (size_t)TC_M * (TC_NMAX + 1) * sizeof(float));
    static std::once_flag attr;
    std::call_once(attr, [&] {
        H2_CUDA(cudaFuncSetAttribute(tc_products_kernel<EB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        H2_CUDA(cudaFuncSetAttribute(tc_group_kernel<EB, Big>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Big::SMEM));
        H2_CUDA(cudaFuncSetAttribute(tc_group_kernel<EB, Small>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)Small::SMEM));
    });
    const unsigned nrt = (unsigned)((nrhs + TC_M - 1) / TC_M);
    if (st.outs[0].to_y) {
        tc_products_kernel<EB><<<dim3(nrt, (unsigned)st.outs.size()), TC_THREADS, smem, s>>>(
            d_outs, d_items, W, opnd, perm, Y, ldy, ws, ws_ld, nrhs, err);
        after_launch("tc_products");
    } else if (st.kmax_item <= Small::KMAX && st.nmax_out <= Small::NMAX) {
        tc_group_kernel<EB, Small><<<dim3(nrt, (unsigned)st.groups.size()), TC_THREADS, Small::SMEM, s>>>(
            d_groups, d_outs, d_items, W, opnd, ws, ws_ld, ws_rmaj, nrhs, st.tmem_cols, err);
        after_launch("tc_group");
    } else {
        tc_group_kernel<EB, Big><<<dim3(nrt, (unsigned)st.groups.size()), TC_THREADS, Big::SMEM, s>>>(
            d_groups, d_outs, d_items, W, opnd, ws, ws_ld, ws_rmaj, nrhs, st.tmem_cols, err);
        after_launch("tc_group");
    }
}

inline int pad16(int k) { return (k + 15) / 16 * 16; }

}  // namespace

bool tc_supported(const h2_handle_s* h) { return h->tc.nleaf > 0; }

// Builds the tensor-core plan: operand rows (X of every leaf, xh and yh of every box with a
// basis), the product lists of the leaf upsweep, the couplings and the near field + leaf
// expansion, and the B-tile pools (BF16 and/or TF32).  Requires leaves of at most 64 points.
void tc_prepare(h2_handle_s* h, int want_bf16, int want_tf32, cudaStream_t s) {
    TcPlan& P = h->tc;
    const h2_tree_s& T = *h->tree;
    const int L = T.L;
    if (T.leaf_max > TC_NMAX || (!want_bf16 && !want_tf32)) return;
    const int nleaf = 1 << L;
    P.LP = pad16(T.leaf_max);
    P.nleaf = nleaf;
    auto K = [&](int l, int b) { return h->k[h->koff[l] + b]; };
    // coefficient rows of the workspace (same layout as build_plan)
    std::vector<int64_t> box_row(h->k.size());
    int64_t rows = 0;
    for (size_t i = 0; i < h->k.size(); ++i) { box_row[i] = rows; rows += h->k[i]; }
    const int64_t ytop = rows;
    // operand rows: X of leaves, then xh (padded) of every box, then yh (padded) of leaves
    int64_t orow = (int64_t)nleaf * P.LP;
    std::vector<int64_t> xop(h->k.size(), -1), yop(nleaf, -1);
    P.xh_boxes.clear();
    P.xh_src.clear();
    for (int l = 1; l <= L; ++l)
        for (int b = 0; b < (1 << l); ++b) {
            const int k = K(l, b);
            if (!k) continue;
            xop[h->koff[l] + b] = orow;
            P.xh_boxes.push_back(make_int4((int)orow, k, pad16(k), 0));
            P.xh_src.push_back(box_row[h->koff[l] + b]);
            orow += pad16(k);
        }
    P.yh_boxes.clear();
    P.yh_src.clear();
    for (int t = 0; t < nleaf; ++t) {
        const int k = K(L, t);
        if (!k || L == 0) continue;
        yop[t] = orow;
        P.yh_boxes.push_back(make_int4((int)orow, k, pad16(k), 0));
        P.yh_src.push_back(ytop + box_row[h->koff[L] + t]);
        orow += pad16(k);
    }
    P.op_rows = (orow + 7) / 8 * 8;
    // product lists and tile sources (byte offsets are per element size; both pools share them)
    std::vector<TcTileSrc> tiles;
    int64_t wpos = 0;   // in elements
    auto add_tile = [&](int64_t m_off, int ldm, int trans, int rows_, int cols_, int n, int k) {
        tiles.push_back(TcTileSrc{m_off, wpos, ldm, trans, rows_, cols_, n, k});
        wpos += (int64_t)n * k;
        return tiles.size() - 1;
    };
    auto build = [&](TcStage& st, std::vector<TcOut>& outs, std::vector<TcItem>& items) {
        st.outs = outs;
        st.items = items;
    };
    // 1. leaf upsweep: xh_t = U_t^T X_t   (N = pad(k_t), K = LP)
    {
        std::vector<TcOut> outs;
        std::vector<TcItem> items;
        for (int t = 0; t < nleaf && L >= 1; ++t) {
            const int kt = K(L, t);
            if (!kt) continue;
            const int m = (int)T.size[L][t];
            outs.push_back(TcOut{box_row[h->koff[L] + t], kt, pad16(kt), (int)items.size(), 0, 0});
            const size_t ti = add_tile(h->u_off[t], m, 1, kt, m, pad16(kt), P.LP);
            items.push_back(TcItem{(int64_t)t * P.LP, P.LP, (int64_t)ti});
            outs.back().end = (int)items.size();
        }
        build(P.leaf_up, outs, items);
    }
    // 2. couplings: yh_t = sum_s S_ts xh_s   (N = pad(k_t), K = pad(k_s))
    {
        std::vector<TcOut> outs;
        std::vector<TcItem> items;
        for (int l = 1; l <= L; ++l) {
            std::vector<std::vector<int>> far_of(1 << l), trn(1 << l);
            std::vector<std::vector<int64_t>> mo(1 << l);
            for (size_t i = 0; i < h->far_lower[l].size(); ++i) {
                auto [t, s2] = h->far_lower[l][i];
                far_of[t].push_back(s2); mo[t].push_back(h->s_off[l][i]); trn[t].push_back(0);
                far_of[s2].push_back(t); mo[s2].push_back(h->s_off[l][i]); trn[s2].push_back(1);
            }
            for (int t = 0; t < (1 << l); ++t) {
                const int kt = K(l, t);
                if (!kt) continue;
                outs.push_back(TcOut{ytop + box_row[h->koff[l] + t], kt, pad16(kt), (int)items.size(), 0, 0});
                for (size_t j = 0; j < far_of[t].size(); ++j) {
                    const int sb = far_of[t][j], ks = K(l, sb);
                    if (!ks) continue;
                    const int ldm = trn[t][j] ? ks : kt;
                    const size_t ti = add_tile(mo[t][j], ldm, trn[t][j], kt, ks, pad16(kt), pad16(ks));
                    items.push_back(TcItem{xop[h->koff[l] + sb], pad16(ks), (int64_t)ti});
                }
                outs.back().end = (int)items.size();
            }
        }
        build(P.couple, outs, items);
    }
    // 3. near field + leaf expansion: Y_t = sum_s op(D_ts) X_s + U_t yh_t   (N = LP)
    {
        std::vector<std::vector<int>> src(nleaf), trn(nleaf);
        std::vector<std::vector<int64_t>> mo(nleaf);
        for (size_t i = 0; i < h->near_lower.size(); ++i) {
            auto [t, s2] = h->near_lower[i];
            src[t].push_back(s2); mo[t].push_back(h->d_off[i]); trn[t].push_back(0);
            if (t != s2) { src[s2].push_back(t); mo[s2].push_back(h->d_off[i]); trn[s2].push_back(1); }
        }
        std::vector<TcOut> outs;
        std::vector<TcItem> items;
        for (int t = 0; t < nleaf; ++t) {
            const int m = (int)T.size[L][t];
            outs.push_back(TcOut{T.start[L][t], m, P.LP, (int)items.size(), 0, 1});
            for (size_t j = 0; j < src[t].size(); ++j) {
                const int sb = src[t][j], ms = (int)T.size[L][sb];
                const int ldm = trn[t][j] ? ms : m;
                const size_t ti = add_tile(mo[t][j], ldm, trn[t][j], m, ms, P.LP, P.LP);
                items.push_back(TcItem{(int64_t)sb * P.LP, P.LP, (int64_t)ti});
            }
            const int kt = L >= 1 ? K(L, t) : 0;
            if (kt) {
                const size_t ti = add_tile(h->u_off[t], m, 0, m, kt, P.LP, pad16(kt));
                items.push_back(TcItem{yop[t], pad16(kt), (int64_t)ti});
            }
            outs.back().end = (int)items.size();
        }
        build(P.near, outs, items);
    }
    for (TcStage* st : {&P.leaf_up, &P.couple, &P.near})
        for (auto& o : st->outs)
            if (o.n > TC_NMAX || o.n % 16) fail(H2_ERR_INVALID_ARG, "tensor-core plan: output rows out of range");
    for (TcStage* st : {&P.leaf_up, &P.couple, &P.near}) {
        st->kmax_item = 0;
        st->nmax_out = 0;
        for (const auto& it : st->items) st->kmax_item = std::max(st->kmax_item, it.k);
        for (const auto& o : st->outs) st->nmax_out = std::max(st->nmax_out, o.n);
    }
    // CTA groups: consecutive outputs (neighbouring boxes in tree order) side by side in tensor
    // memory, one operand ring across all their items; coefficient outputs only (the near-field
    // outputs go through the permutation and keep one CTA each), and at most TC_GROUP_ITEMS items
    // so that the split-TF32 lists (three items per product) stay in the shared-memory cache
    for (TcStage* st : {&P.leaf_up, &P.couple, &P.near}) {
        st->groups.clear();
        st->tmem_cols = 32;
        int cols = 0, nit = 0;
        for (int o = 0; o < (int)st->outs.size(); ++o) {
            const TcOut& out = st->outs[o];
            const int n = out.n, ni = out.end - out.beg;
            if (st->groups.empty() || out.to_y || st->outs[st->groups.back().obeg].to_y || cols + n > TC_GCOLS ||
                nit + ni > TC_GROUP_ITEMS || st->groups.back().oend - st->groups.back().obeg >= TC_GMAX) {
                st->groups.push_back(TcGroup{o, o, out.beg, out.beg});
                cols = 0;
                nit = 0;
            }
            st->groups.back().oend = o + 1;
            st->groups.back().iend = out.end;
            cols += n;
            nit += ni;
            while (st->tmem_cols < cols) st->tmem_cols *= 2;
        }
        if (st->groups.size() > 65535) fail(H2_ERR_INVALID_ARG, "tensor-core plan: more than 65535 output groups");
        for (const auto& o : st->outs)
            if (o.to_y != st->outs[0].to_y) fail(H2_ERR_INVALID_ARG, "tensor-core plan: mixed output kinds in a stage");
    }
    P.w_elems = wpos;
    Stager stg;
    for (TcStage* st : {&P.leaf_up, &P.couple, &P.near}) {
        upload(st->d_outs, st->outs, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
        upload(st->d_groups, st->groups, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
        std::vector<TcGroup> g3 = st->groups;
        for (auto& g : g3) {
            g.ibeg *= 3;
            g.iend *= 3;
        }
        upload(st->d_groups32x3, g3, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
    }
    P.d_err.reserve(1);
    H2_CUDA(cudaMemsetAsync(P.d_err.p, 0, sizeof(int), s));
    std::vector<int64_t> lst(nleaf);
    std::vector<int> lsz(nleaf);
    for (int t = 0; t < nleaf; ++t) { lst[t] = T.start[L][t]; lsz[t] = (int)T.size[L][t]; }
    upload(P.d_leaf_start, lst, s, stg);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(P.d_leaf_size, lsz, s, stg);
    H2_CUDA(cudaStreamSynchronize(s));
    for (int which = 0; which < 2; ++which) {
        std::vector<int4>& bx = which ? P.yh_boxes : P.xh_boxes;
        std::vector<int64_t>& sr = which ? P.yh_src : P.xh_src;
        upload(which ? P.d_yh_boxes : P.d_xh_boxes, bx, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
        upload(which ? P.d_yh_src : P.d_xh_src, sr, s, stg);
        H2_CUDA(cudaStreamSynchronize(s));
    }
    // tiles: byte offsets per precision; items refer to tile indices until here
    DevBuf<TcTileSrc> d_tiles;
    for (int eb : {2, 4}) {
        if ((eb == 2 && !want_bf16) || (eb == 4 && !want_tf32) || tiles.empty()) continue;
        std::vector<TcTileSrc> tb = tiles;
        for (auto& t : tb) t.dst *= eb;
        upload(d_tiles, tb, s, stg);
        DevBuf<unsigned char>& Wp = (eb == 2) ? P.W16 : P.W32;
        // the TF32 pool also holds the low parts of the split-TF32 products, after the high parts
        const int64_t lo_off = (eb == 4) ? P.w_elems * 4 : 0;
        Wp.reserve((size_t)P.w_elems * eb * (eb == 4 ? 2 : 1));
        if (eb == 2) tc_pack_tiles_kernel<2><<<(unsigned)tb.size(), 256, 0, s>>>(h->fac64.p, d_tiles.p, Wp.p, 0);
        else tc_pack_tiles_kernel<4><<<(unsigned)tb.size(), 256, 0, s>>>(h->fac64.p, d_tiles.p, Wp.p, lo_off);
        after_launch("tc_pack_tiles");
        H2_CUDA(cudaStreamSynchronize(s));
        // per-precision item lists (byte offsets of B tiles)
        for (TcStage* st : {&P.leaf_up, &P.couple, &P.near}) {
            std::vector<TcItem> it = st->items;
            for (auto& x : it) x.b_off = tiles[(size_t)x.b_off].dst * eb;
            upload(eb == 2 ? st->d_items16 : st->d_items32, it, s, stg);
            H2_CUDA(cudaStreamSynchronize(s));
            if (eb == 4) {
                // split TF32: hi x hi, hi(A) x lo(B), lo(A) x hi(B), accumulated in one TMEM tile;
                // low operand rows follow the high ones at op_rows
                std::vector<TcItem> x3;
                x3.reserve(it.size() * 3);
                for (const auto& x : it) {
                    x3.push_back(x);
                    x3.push_back(TcItem{x.a_row, x.k, x.b_off + lo_off});
                    x3.push_back(TcItem{x.a_row + P.op_rows, x.k, x.b_off});
                }
                std::vector<TcOut> o3 = st->outs;
                for (auto& o : o3) {
                    o.beg *= 3;
                    o.end *= 3;
                }
                upload(st->d_items32x3, x3, s, stg);
                H2_CUDA(cudaStreamSynchronize(s));
                upload(st->d_outs32x3, o3, s, stg);
                H2_CUDA(cudaStreamSynchronize(s));
            }
        }
    }
}

// Tensor-core matvec for BF16 (X bf16) or TF32 (X fp32): leaf upsweep, couplings and near field
// + leaf expansion on tcgen05; the transfer sweeps on the SIMT stage kernels (run_tree_sweeps).
// Operand buffer of a tensor-core matvec with nrhs right-hand sides in the precision of mode
// (split TF32 keeps a low part of every operand row after the high parts).
void tc_reserve(h2_handle_s* h, int mode, int nrhs) {
    TcPlan& P = h->tc;
    const int EB = (mode == H2_BF16) ? 2 : 4;
    const int nrt = (nrhs + TC_M - 1) / TC_M;
    P.opnd.reserve((size_t)(P.op_rows * nrt * TC_M * EB) * (mode == H2_TF32X3 ? 2 : 1));
}

// One phase of the tensor-core matvec: 0 packs X and computes the leaf coefficients xh, 1 packs
// xh and computes the couplings into yh, 2 packs yh and computes Y = U yh + near field.  The
// transfer sweeps between the phases run on the SIMT path.
void tc_phase(h2_handle_s* h, int mode, int phase, const void* X, int64_t ldx, float* Y, int64_t ldy, int nrhs,
              float* ws, int64_t ws_ld, int ws_rmaj, cudaStream_t s) {
    TcPlan& P = h->tc;
    const int EB = (mode == H2_BF16) ? 2 : 4;
    const bool split = mode == H2_TF32X3;
    const int nrt = (nrhs + TC_M - 1) / TC_M;
    tc_reserve(h, mode, nrhs);
    const unsigned char* W = (mode == H2_BF16) ? P.W16.p : P.W32.p;
    if (!W) fail(H2_ERR_INVALID_ARG, "h2_matvec: tensor-core tiles of this precision were not kept");
    // byte distance from an operand's high part to its low part
    const int64_t lo_off = split ? P.op_rows * nrt * TC_M * 4 : 0;
    auto run = [&](TcStage& st) {
        if (st.outs.empty()) return;
        if (EB == 2)
            launch_products<2>(st, st.d_groups.p, st.d_outs.p, st.d_items16.p, W, P.opnd.p, h->d_perm.p, Y, ldy, ws,
                               ws_ld, ws_rmaj, nrhs, P.d_err.p, s);
        else if (split)
            launch_products<4>(st, st.d_groups32x3.p, st.d_outs32x3.p, st.d_items32x3.p, W, P.opnd.p, h->d_perm.p, Y,
                               ldy, ws, ws_ld, ws_rmaj, nrhs, P.d_err.p, s);
        else
            launch_products<4>(st, st.d_groups.p, st.d_outs.p, st.d_items32.p, W, P.opnd.p, h->d_perm.p, Y, ldy, ws,
                               ws_ld, ws_rmaj, nrhs, P.d_err.p, s);
    };
    if (nrt > 65535) fail(H2_ERR_INVALID_ARG, "h2_matvec: more than 65535 tiles of 128 right-hand sides");
    auto pack_coef = [&](const std::vector<int4>& bx, const DevBuf<int4>& dbx, const DevBuf<int64_t>& dsrc) {
        if (bx.empty()) return;
        const dim3 g((unsigned)bx.size(), (unsigned)nrt);
        if (EB == 2)
            tc_pack_coef_kernel<2><<<g, PK_THREADS, 0, s>>>(dbx.p, ws, ws_ld, ws_rmaj, dsrc.p, nrhs, P.opnd.p, 0);
        else
            tc_pack_coef_kernel<4><<<g, PK_THREADS, 0, s>>>(dbx.p, ws, ws_ld, ws_rmaj, dsrc.p, nrhs, P.opnd.p,
                                                            lo_off);
        after_launch("tc_pack_coef");
    };
    P.cur_eb = EB;
    if (phase == 0) {
        const dim3 g((unsigned)P.nleaf, (unsigned)nrt);
        if (EB == 2)
            tc_pack_x_kernel<__nv_bfloat16, 2><<<g, PK_THREADS, 0, s>>>((const __nv_bfloat16*)X, ldx, h->d_perm.p,
                                                                        P.d_leaf_start.p, P.d_leaf_size.p, P.LP,
                                                                        nrhs, P.opnd.p, 0);
        else
            tc_pack_x_kernel<float, 4><<<g, PK_THREADS, 0, s>>>((const float*)X, ldx, h->d_perm.p, P.d_leaf_start.p,
                                                               P.d_leaf_size.p, P.LP, nrhs, P.opnd.p, lo_off);
        after_launch("tc_pack_x");
        run(P.leaf_up);
    } else if (phase == 1) {
        pack_coef(P.xh_boxes, P.d_xh_boxes, P.d_xh_src);
        run(P.couple);
    } else {
        pack_coef(P.yh_boxes, P.d_yh_boxes, P.d_yh_src);
        run(P.near);
    }
}

void tc_matvec(h2_handle_s* h, int mode, const void* X, int64_t ldx, float* Y, int64_t ldy, int nrhs, float* ws,
               int64_t ws_ld, int ws_rmaj, cudaStream_t s, const std::function<void(int)>& sweeps,
               const std::function<void(int, std::function<void()>)>& timed) {
    timed(H2_STAGE_LEAF_UP, [&] { tc_phase(h, mode, 0, X, ldx, Y, ldy, nrhs, ws, ws_ld, ws_rmaj, s); });
    sweeps(0);   // transfer upsweep (SIMT)
    timed(H2_STAGE_COUPLE, [&] { tc_phase(h, mode, 1, X, ldx, Y, ldy, nrhs, ws, ws_ld, ws_rmaj, s); });
    sweeps(1);   // transfer downsweep (SIMT)
    timed(H2_STAGE_NEAR, [&] { tc_phase(h, mode, 2, X, ldx, Y, ldy, nrhs, ws, ws_ld, ws_rmaj, s); });
}

int tc_device_error(h2_handle_s* h) {
    if (!h->tc.d_err.p) return 0;
    int v = 0;
    H2_CUDA(cudaMemcpy(&v, h->tc.d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    return v;
}

}  // namespace h2
