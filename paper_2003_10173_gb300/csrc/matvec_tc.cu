// Near field of the multi-RHS matvec on the 5th-generation tensor cores (tcgen05).
//
// For every leaf t and a tile of 128 right-hand sides, Y_t^T = sum_s X_s^T op(D_ts)^T is
// computed as a chain of 128 x LP x 16 (BF16) or 128 x LP x 8 (TF32) MMAs with the FP32
// accumulator in tensor memory:
//   A operand  X_s^T  (M = rhs, K = rows of s): read from a tree-ordered, leaf-padded copy of X;
//   B operand  op(D_ts) (N = rows of t, K = rows of s): every use of a near block (both
//              triangles) stored once, pre-rounded and pre-laid out in the canonical
//              K-major core-matrix layout, so a tile load is a contiguous copy.
// Operands are staged in shared memory by cp.async (3-stage ring); one thread issues the MMAs
// and commits them to a per-stage mbarrier that releases the stage.  The accumulator is read
// with tcgen05.ld, transposed through shared memory and written to Y through the tree
// permutation.  Every mbarrier wait is bounded: on timeout the kernel records a device error,
// drains its copies, frees its tensor memory and returns.
#include <algorithm>

#include "handle.h"

namespace h2 {

namespace {

constexpr int TC_M = 128;      // right-hand sides per CTA (MMA M)
constexpr int TC_STAGES = 3;
constexpr int TC_THREADS = 128;
constexpr long long TC_WAIT_CYCLES = 2000000000LL;   // about one second

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

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(n));
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

// EB: operand element bytes (2: BF16, 4: TF32 in FP32 containers); LP: padded leaf rows.
template <int EB, int LP>
__global__ void __launch_bounds__(TC_THREADS) mv_near_tc_kernel(
    const int* __restrict__ item_beg, const int* __restrict__ item_src, const unsigned char* __restrict__ W,
    const unsigned char* __restrict__ Xp, int64_t ldxp, const int32_t* __restrict__ perm,
    const int64_t* __restrict__ leaf_start, const int* __restrict__ leaf_size, float* __restrict__ Y, int64_t ldy,
    int nrhs, int* __restrict__ err) {
    using Tr = TcTraits<EB>;
    constexpr int A_BYTES = TC_M * LP * EB;
    constexpr int B_BYTES = LP * LP * EB;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    constexpr int TMEM_COLS = LP <= 32 ? 32 : (LP <= 64 ? 64 : 128);
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[TC_STAGES];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int t = blockIdx.x;
    const int r0 = blockIdx.y * TC_M;
    const int ibeg = item_beg[t], iend = item_beg[t + 1];
    const int nitem = iend - ibeg;

    if (tid == 0)
        for (int s = 0; s < TC_STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[s])));
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

    // issue the copies of item `it` into stage `st`
    auto load = [&](int it, int st) {
        unsigned char* sA = smem + st * STAGE_BYTES;
        unsigned char* sB = sA + A_BYTES;
        const int s = item_src[ibeg + it];
        const unsigned char* xs = Xp + (int64_t)s * LP * EB;
        constexpr int ACH = TC_M * LP * EB / 16;   // 16-byte chunks of A
        for (int c = tid; c < ACH; c += TC_THREADS) {
            const int r = c / (LP * EB / 16);
            const int k = (c % (LP * EB / 16)) * (16 / EB);
            const bool valid = (r0 + r) < nrhs;
            const unsigned char* src = xs + ((int64_t)(valid ? r0 + r : 0) * ldxp + k) * EB;
            cp_async16(smem_u32(sA + kmaj_off<EB>(r, k, LP)), src, valid);
        }
        const unsigned char* wb = W + (int64_t)(ibeg + it) * B_BYTES;
        for (int c = tid; c < B_BYTES / 16; c += TC_THREADS) cp_async16(smem_u32(sB + c * 16), wb + c * 16, true);
        asm volatile("cp.async.commit_group;");
    };

    bool ok = true;
    const uint32_t idesc = (1u << 4) | (Tr::ab_fmt << 7) | (Tr::ab_fmt << 10) | ((uint32_t)(LP >> 3) << 17) |
                           ((uint32_t)(TC_M >> 4) << 24);
    // prologue: first TC_STAGES-1 items
    for (int p = 0; p < TC_STAGES - 1; ++p) {
        if (p < nitem) load(p, p);
        else asm volatile("cp.async.commit_group;");
    }
    for (int it = 0; it < nitem && ok; ++it) {
        const int nxt = it + TC_STAGES - 1;
        if (nxt < nitem) {
            const int st = nxt % TC_STAGES;
            if (nxt >= TC_STAGES) {   // stage previously used by item nxt - TC_STAGES
                const int prev = nxt - TC_STAGES;
                ok = mbar_wait(smem_u32(&mbar[st]), (uint32_t)((prev / TC_STAGES) & 1), err);
            }
            if (ok) load(nxt, st);
            else asm volatile("cp.async.commit_group;");
        } else {
            asm volatile("cp.async.commit_group;");
        }
        asm volatile("cp.async.wait_group %0;" ::"n"(TC_STAGES - 1));
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        ok = __syncthreads_and(ok);
        if (!ok) break;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int st = it % TC_STAGES;
            const uint32_t a0 = smem_u32(smem + st * STAGE_BYTES);
            const uint32_t b0 = a0 + A_BYTES;
            constexpr uint32_t SBO = (uint32_t)(LP * EB / 16) * 128;
            for (int kk = 0; kk < LP / Tr::KSTEP; ++kk) {
                const uint64_t ad = smem_desc(a0 + kk * 256, 128, SBO);
                const uint64_t bd = smem_desc(b0 + kk * 256, 128, SBO);
                Tr::mma(tmem, ad, bd, idesc, (it > 0 || kk > 0) ? 1u : 0u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&mbar[st])));
        }
    }
    asm volatile("cp.async.wait_group 0;");
    if (ok && nitem > 0) {
        const int last = nitem - 1;
        ok = mbar_wait(smem_u32(&mbar[last % TC_STAGES]), (uint32_t)((last / TC_STAGES) & 1), err);
    }
    ok = __syncthreads_and(ok);
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: accumulator (lane = rhs r, column = row i of t) -> shared [r][i] -> Y
    const int m = leaf_size[t];
    float* stage = reinterpret_cast<float*>(smem);
    constexpr int SLD = LP + 1;
    if (ok) {
        const int r = warp * 32 + (tid & 31);
        for (int c0 = 0; c0 < LP; c0 += 16) {
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
    const int64_t st0 = leaf_start[t];
    for (int e = tid; e < m * TC_M; e += TC_THREADS) {
        const int i = e % m, r = e / m;
        if (r0 + r < nrhs) Y[perm[st0 + i] + (int64_t)(r0 + r) * ldy] = stage[r * SLD + i];
    }
}

// near-block tile of one use: op(D) (rows of t x rows of s) rounded and laid out as the B operand
template <int EB>
__global__ void tc_pack_blocks_kernel(const double* __restrict__ fac, const int64_t* __restrict__ m_off,
                                      const int* __restrict__ ldm, const int* __restrict__ trans,
                                      const int* __restrict__ rows, const int* __restrict__ cols, int LP,
                                      unsigned char* __restrict__ W) {
    const int b = blockIdx.x;
    const int nr = rows[b], nc = cols[b];
    const double* M = fac + m_off[b];
    unsigned char* out = W + (int64_t)b * LP * LP * EB;
    for (int e = threadIdx.x; e < LP * LP; e += blockDim.x) {
        const int i = e % LP, j = e / LP;
        double v = 0.0;
        if (i < nr && j < nc) v = trans[b] ? M[j + (int64_t)i * ldm[b]] : M[i + (int64_t)j * ldm[b]];
        const uint32_t o = kmaj_off<EB>(i, j, LP);
        if constexpr (EB == 2) {
            *reinterpret_cast<__nv_bfloat16*>(out + o) = __double2bfloat16(v);
        } else {
            float f = (float)v;
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(f));
            *reinterpret_cast<uint32_t*>(out + o) = u;
        }
    }
}

// X (caller order) -> tree-ordered, leaf-padded operand copy (BF16 or TF32-rounded FP32)
template <class TX, int EB>
__global__ void tc_pack_x_kernel(const TX* __restrict__ X, int64_t ldx, const int32_t* __restrict__ perm,
                                 const int64_t* __restrict__ leaf_start, const int* __restrict__ leaf_size, int LP,
                                 int nleaf, int nrhs, unsigned char* __restrict__ Xp, int64_t ldxp) {
    const int64_t total = (int64_t)nleaf * LP * nrhs;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e % ((int64_t)nleaf * LP);
        const int r = (int)(e / ((int64_t)nleaf * LP));
        const int t = (int)(row / LP), i = (int)(row % LP);
        float v = 0.f;
        if (i < leaf_size[t]) {
            const TX x = X[perm[leaf_start[t] + i] + (int64_t)r * ldx];
            if constexpr (std::is_same<TX, __nv_bfloat16>::value) v = __bfloat162float(x);
            else v = (float)x;
        }
        unsigned char* dst = Xp + (row + (int64_t)r * ldxp) * EB;
        if constexpr (EB == 2) {
            *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
        } else {
            uint32_t u;
            asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
            *reinterpret_cast<uint32_t*>(dst) = u;
        }
    }
}

template <int EB, int LP>
void launch_near_tc(h2_handle_s* h, TcPlan& P, const unsigned char* W, const unsigned char* Xp, int64_t ldxp, float* Y,
                    int64_t ldy, int nrhs, cudaStream_t s) {
    constexpr int STAGE_BYTES = TC_M * LP * EB + LP * LP * EB;
    const size_t smem = std::max((size_t)TC_STAGES * STAGE_BYTES, (size_t)TC_M * (LP + 1) * sizeof(float));
    static bool attr = false;
    if (!attr) {
        H2_CUDA(cudaFuncSetAttribute(mv_near_tc_kernel<EB, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    dim3 grid((unsigned)P.nleaf, (unsigned)((nrhs + TC_M - 1) / TC_M));
    mv_near_tc_kernel<EB, LP><<<grid, TC_THREADS, smem, s>>>(P.d_beg.p, P.d_src.p, W, Xp, ldxp, h->d_perm.p,
                                                             P.d_leaf_start.p, P.d_leaf_size.p, Y, ldy, nrhs, P.d_err.p);
    after_launch("mv_near_tc");
}

}  // namespace

bool tc_supported(const h2_handle_s* h) { return h->tc.nleaf > 0; }

// Lists the near-block uses per leaf and packs their tensor-core tiles (both precisions kept
// if requested).  Leaves must be at most 64 rows (padded to 16 or 32 or 64).
void tc_prepare(h2_handle_s* h, int want_bf16, int want_tf32, cudaStream_t s) {
    TcPlan& P = h->tc;
    const h2_tree_s& T = *h->tree;
    const int L = T.L;
    if (T.leaf_max > 64 || (!want_bf16 && !want_tf32)) return;
    const int nleaf = 1 << L;
    P.LP = T.leaf_max <= 16 ? 16 : (T.leaf_max <= 32 ? 32 : 64);
    P.nleaf = nleaf;
    std::vector<std::vector<int>> src(nleaf), tr(nleaf);
    std::vector<std::vector<int64_t>> mo(nleaf);
    for (size_t i = 0; i < h->near_lower.size(); ++i) {
        auto [t, s2] = h->near_lower[i];
        src[t].push_back(s2); mo[t].push_back(h->d_off[i]); tr[t].push_back(0);
        if (t != s2) { src[s2].push_back(t); mo[s2].push_back(h->d_off[i]); tr[s2].push_back(1); }
    }
    std::vector<int> beg(nleaf + 1, 0), isrc, ild, itr, irows, icols, lsz(nleaf);
    std::vector<int64_t> imo, lst(nleaf);
    for (int t = 0; t < nleaf; ++t) {
        lst[t] = T.start[L][t];
        lsz[t] = (int)T.size[L][t];
        for (size_t j = 0; j < src[t].size(); ++j) {
            const int sb = src[t][j];
            isrc.push_back(sb);
            imo.push_back(mo[t][j]);
            itr.push_back(tr[t][j]);
            irows.push_back((int)T.size[L][t]);
            icols.push_back((int)T.size[L][sb]);
            ild.push_back(tr[t][j] ? (int)T.size[L][sb] : (int)T.size[L][t]);
        }
        beg[t + 1] = (int)isrc.size();
    }
    P.nitems = (int64_t)isrc.size();
    Stager st;
    upload(P.d_beg, beg, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(P.d_src, isrc, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(P.d_leaf_start, lst, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(P.d_leaf_size, lsz, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    DevBuf<int64_t> d_mo;
    DevBuf<int> d_ld, d_tr, d_rows, d_cols;
    upload(d_mo, imo, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(d_ld, ild, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(d_tr, itr, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(d_rows, irows, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    upload(d_cols, icols, s, st);
    H2_CUDA(cudaStreamSynchronize(s));
    P.d_err.reserve(1);
    H2_CUDA(cudaMemsetAsync(P.d_err.p, 0, sizeof(int), s));
    const unsigned nb = (unsigned)std::max<int64_t>(P.nitems, 1);
    if (want_bf16 && P.nitems) {
        P.W16.reserve((size_t)P.nitems * P.LP * P.LP * 2);
        tc_pack_blocks_kernel<2><<<nb, 256, 0, s>>>(h->fac64.p, d_mo.p, d_ld.p, d_tr.p, d_rows.p, d_cols.p, P.LP, P.W16.p);
        after_launch("tc_pack_bf16");
    }
    if (want_tf32 && P.nitems) {
        P.W32.reserve((size_t)P.nitems * P.LP * P.LP * 4);
        tc_pack_blocks_kernel<4><<<nb, 256, 0, s>>>(h->fac64.p, d_mo.p, d_ld.p, d_tr.p, d_rows.p, d_cols.p, P.LP, P.W32.p);
        after_launch("tc_pack_tf32");
    }
    H2_CUDA(cudaStreamSynchronize(s));
}

// Y = near field of X for a BF16 (X bf16) or TF32 (X fp32) matvec with nrhs right-hand sides.
void tc_near(h2_handle_s* h, int mode, const void* X, int64_t ldx, float* Y, int64_t ldy, int nrhs, cudaStream_t s) {
    TcPlan& P = h->tc;
    const int EB = (mode == H2_BF16) ? 2 : 4;
    const int64_t rows = (int64_t)P.nleaf * P.LP;
    const int64_t ldxp = rows;
    P.Xp.reserve((size_t)(rows * nrhs * EB));
    const int64_t total = rows * nrhs;
    const unsigned g = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    if (mode == H2_BF16) {
        tc_pack_x_kernel<__nv_bfloat16, 2><<<g, 256, 0, s>>>((const __nv_bfloat16*)X, ldx, h->d_perm.p, P.d_leaf_start.p,
                                                              P.d_leaf_size.p, P.LP, P.nleaf, nrhs, P.Xp.p, ldxp);
    } else {
        tc_pack_x_kernel<float, 4><<<g, 256, 0, s>>>((const float*)X, ldx, h->d_perm.p, P.d_leaf_start.p,
                                                     P.d_leaf_size.p, P.LP, P.nleaf, nrhs, P.Xp.p, ldxp);
    }
    after_launch("tc_pack_x");
    const unsigned char* W = (mode == H2_BF16) ? P.W16.p : P.W32.p;
    if (!W) fail(H2_ERR_INVALID_ARG, "h2_matvec: tensor-core tiles of this precision were not kept");
    switch (P.LP * 10 + EB) {
        case 162: launch_near_tc<2, 16>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        case 322: launch_near_tc<2, 32>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        case 642: launch_near_tc<2, 64>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        case 164: launch_near_tc<4, 16>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        case 324: launch_near_tc<4, 32>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        case 644: launch_near_tc<4, 64>(h, P, W, P.Xp.p, ldxp, Y, ldy, nrhs, s); break;
        default: fail(H2_ERR_INVALID_ARG, "h2_matvec: unsupported padded leaf size for tensor cores");
    }
}

int tc_device_error(h2_handle_s* h) {
    if (!h->tc.d_err.p) return 0;
    int v = 0;
    H2_CUDA(cudaMemcpy(&v, h->tc.d_err.p, sizeof(int), cudaMemcpyDeviceToHost));
    return v;
}

}  // namespace h2
