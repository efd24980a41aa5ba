// Variable-size batched FP64 GEMM for the construction phase.
//
// The peeling construction (Section 3.3) and the recompression (Section 3.2)
// reduce to many small dense products of uneven sizes: removing coarser
// pieces from samples, projecting sample blocks against their bases, Gram
// matrices of block rows, couplings and near blocks.  All of them go through
// one marshaled launch: the host lists the output tiles of every problem and
// each CTA computes one 64x64 tile (FP64 on the SIMT pipe; GB300's FP64 rate
// is low enough that a register-blocked 4x4 per thread keeps it busy).  Long
// reductions with few output tiles are split along k into slots of a
// workspace and summed in a fixed order afterwards, so results do not depend
// on scheduling.  Launches with fewer output tiles than two per SM split every reduction so
// that the grid covers the GPU (e.g. the heat operator on one or a few vectors).
#include <algorithm>
#include <mutex>

#include "common.h"

namespace h2 {

namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;
constexpr int64_t kFillCtas = 2 * 152;   // two resident CTAs on each of the 152 SMs
constexpr int kMinChunk = 32;            // shortest k range of a split

// One TMv x 64 output tile (TMv = 64, 32 or 16): 256 threads, each TMv/16 x 4 outputs.
template <int TMv>
__device__ __forceinline__ void gemm_tile(const GemmProb& P, int m0, int n0, int kbeg, int kend, int slot,
                                          double* __restrict__ work, double (*As)[TM + 1], double (*Bs)[TN + 1]) {
    constexpr int RI = TMv / 16;
    const int tid = threadIdx.x;
    const int tr = tid & 15, tc = tid >> 4;
    double acc[RI][4];
#pragma unroll
    for (int i = 0; i < RI; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

    for (int k0 = kbeg; k0 < kend; k0 += TK) {
        // load op(A) tile: TMv x 16
#pragma unroll
        for (int r = 0; r < RI; ++r) {
            const int e = tid + r * NT;
            int i, kk;
            if (!P.ta) { i = e % TMv; kk = e / TMv; }   // coalesced along i
            else       { kk = e & 15; i = e >> 4; }     // coalesced along k
            const int gi = m0 + i, gk = k0 + kk;
            double v = 0.0;
            if (gi < P.m && gk < kend)
                v = P.ta ? P.A[gk + (int64_t)gi * P.lda] : P.A[gi + (int64_t)gk * P.lda];
            As[kk][i] = v;
        }
        // load op(B) tile: 16 x 64
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * NT;
            int j, kk;
            if (!P.tb) { kk = e & 15; j = e >> 4; }   // coalesced along k
            else       { j = e & 63; kk = e >> 6; }   // coalesced along j
            const int gj = n0 + j, gk = k0 + kk;
            double v = 0.0;
            if (gj < P.n && gk < kend)
                v = P.tb ? P.B[gj + (int64_t)gk * P.ldb] : P.B[gk + (int64_t)gj * P.ldb];
            Bs[kk][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            double a[RI], b[4];
#pragma unroll
            for (int i = 0; i < RI; ++i) a[i] = As[kk][tr + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
            for (int i = 0; i < RI; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }

    if (slot < 0) {
#pragma unroll
        for (int i = 0; i < RI; ++i) {
            const int gi = m0 + tr + 16 * i;
            if (gi >= P.m) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int gj = n0 + tc + 16 * j;
                if (gj >= P.n) continue;
                double* c = P.C + (P.tc ? (gj + (int64_t)gi * P.ldc) : (gi + (int64_t)gj * P.ldc));
                const double v = P.alpha * acc[i][j];
                *c = (P.beta == 0.0) ? v : fma(P.beta, *c, v);
            }
        }
    } else {
        double* w = work + (int64_t)slot * (TM * TN);
#pragma unroll
        for (int i = 0; i < RI; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) w[(tr + 16 * i) + (tc + 16 * j) * TM] = acc[i][j];
    }
}

__global__ void __launch_bounds__(NT) gemm_tiles_kernel(const GemmProb* __restrict__ probs,
                                                         const int4* __restrict__ tiles,
                                                         double* __restrict__ work) {
    const int4 t = tiles[blockIdx.x];
    const GemmProb P = probs[t.x];
    const int tm = t.y & 0xffff, tn = t.y >> 16;
    const int split = t.z, slot = t.w;
    const int m0 = tm * P.tm, n0 = tn * TN;

    int kbeg = 0, kend = P.k;
    if (slot >= 0) {
        // k range of this split; split count stored in the high bits of z
        const int ns = split >> 16, ks = split & 0xffff;
        int chunk = (P.k + ns - 1) / ns;
        chunk = (chunk + TK - 1) / TK * TK;
        kbeg = ks * chunk;
        kend = min(P.k, kbeg + chunk);
    }

    __shared__ double As[TK][TM + 1];
    __shared__ double Bs[TK][TN + 1];
    if (P.tm == 16) gemm_tile<16>(P, m0, n0, kbeg, kend, slot, work, As, Bs);
    else if (P.tm == 32) gemm_tile<32>(P, m0, n0, kbeg, kend, slot, work, As, Bs);
    else gemm_tile<64>(P, m0, n0, kbeg, kend, slot, work, As, Bs);
}

// Sums the split-k partial tiles in slot order and applies alpha/beta.
__global__ void __launch_bounds__(NT) gemm_reduce_kernel(const GemmProb* __restrict__ probs,
                                                          const int4* __restrict__ red,
                                                          const double* __restrict__ work) {
    const int4 r = red[blockIdx.x];
    const GemmProb P = probs[r.x];
    const int m0 = (r.y & 0xffff) * P.tm, n0 = (r.y >> 16) * TN;
    const int ns = r.z, slot0 = r.w;
    for (int e = threadIdx.x; e < P.tm * TN; e += NT) {
        const int i = e % P.tm, j = e / P.tm;
        const int gi = m0 + i, gj = n0 + j;
        if (gi >= P.m || gj >= P.n) continue;
        double s = 0.0;
        for (int q = 0; q < ns; ++q) s += work[(int64_t)(slot0 + q) * (TM * TN) + i + j * TM];
        double* c = P.C + (P.tc ? (gj + (int64_t)gi * P.ldc) : (gi + (int64_t)gj * P.ldc));
        const double v = P.alpha * s;
        *c = (P.beta == 0.0) ? v : fma(P.beta, *c, v);
    }
}

// zero-k problems still have to apply beta
__global__ void gemm_scale_kernel(const GemmProb* __restrict__ probs, const int4* __restrict__ tiles) {
    const int4 t = tiles[blockIdx.x];
    const GemmProb P = probs[t.x];
    const int m0 = (t.y & 0xffff) * P.tm, n0 = (t.y >> 16) * TN;
    for (int e = threadIdx.x; e < P.tm * TN; e += blockDim.x) {
        const int gi = m0 + e % P.tm, gj = n0 + e / P.tm;
        if (gi >= P.m || gj >= P.n) continue;
        double* c = P.C + (P.tc ? (gj + (int64_t)gi * P.ldc) : (gi + (int64_t)gj * P.ldc));
        *c = (P.beta == 0.0) ? 0.0 : P.beta * *c;
    }
}

struct GemmProfile {
    std::mutex mu;   // construction workers of a batched build may run concurrently
    int on = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> used;
    std::vector<cudaEvent_t> pool;
    double ms = 0.0, flops = 0.0, bytes = 0.0;
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
GemmProfile g_prof;

}  // namespace

void gemm_profile_enable(int on) { g_prof.on = on; }

int gemm_profile_on() { return g_prof.on; }

void gemm_profile_read(double* ms, double* flops, int64_t* launches, double* bytes) {
    H2_CUDA(cudaDeviceSynchronize());
    std::lock_guard<std::mutex> lock(g_prof.mu);
    for (auto& u : g_prof.used) {
        float t = 0.f;
        H2_CUDA(cudaEventElapsedTime(&t, u.first, u.second));
        g_prof.ms += t;
        g_prof.pool.push_back(u.first);
        g_prof.pool.push_back(u.second);
    }
    g_prof.used.clear();
    if (ms) *ms = g_prof.ms;
    if (flops) *flops = g_prof.flops;
    if (launches) *launches = g_prof.launches;
    if (bytes) *bytes = g_prof.bytes;
    g_prof.ms = 0.0;
    g_prof.flops = 0.0;
    g_prof.bytes = 0.0;
    g_prof.launches = 0;
}

namespace {

// Tile shape of a problem: a narrow n (<= 32, narrower than m) is turned into a narrow m by
// computing C^T = op(B)^T op(A)^T; the tile height is the smallest of 16/32/64 covering m.
void shape(GemmProb& p) {
    if (p.n <= 32 && p.n < p.m) {
        std::swap(p.A, p.B);
        std::swap(p.lda, p.ldb);
        const int ta = p.ta;
        p.ta = !p.tb;
        p.tb = !ta;
        std::swap(p.m, p.n);
        p.tc = 1;
    }
    p.tm = p.m <= 16 ? 16 : (p.m <= 32 ? 32 : 64);
}

}  // namespace

void GemmBatch::run(cudaStream_t s) {
    if (probs_.empty()) return;
    std::vector<int4> tiles, red, scale;
    int slots = 0;
    for (GemmProb& p : probs_) shape(p);
    // output tiles of the whole launch; below two CTAs per SM every reduction is split (chunks of
    // at least kMinChunk) until the launch fills the GPU
    int64_t base_tiles = 0;
    for (const GemmProb& p : probs_)
        if (p.k > 0) base_tiles += (int64_t)((p.m + p.tm - 1) / p.tm) * ((p.n + TN - 1) / TN);
    const int fill = (base_tiles > 0 && base_tiles < kFillCtas) ? (int)((kFillCtas + base_tiles - 1) / base_tiles) : 1;
    for (size_t pi = 0; pi < probs_.size(); ++pi) {
        const GemmProb& p = probs_[pi];
        if (p.m >= (1 << 16) * p.tm || p.n >= (1 << 16) * TN)
            fail(H2_ERR_INVALID_ARG, "gemm: dimension too large");
        const int mt = (p.m + p.tm - 1) / p.tm, nt = (p.n + TN - 1) / TN;
        if (p.k <= 0) {
            for (int a = 0; a < mt; ++a)
                for (int b = 0; b < nt; ++b) scale.push_back(make_int4((int)pi, a | (b << 16), 0, -1));
            continue;
        }
        int ns = std::min(fill, std::max(1, p.k / kMinChunk));
        // long reductions with few output tiles are split further
        const int ntile = mt * nt;
        if (p.k >= 2048 && ntile < 64) ns = std::max(ns, std::min(std::max(1, p.k / 1024), std::max(1, 128 / ntile)));
        ns = std::min(ns, 64);
        for (int a = 0; a < mt; ++a)
            for (int b = 0; b < nt; ++b) {
                const int tyx = a | (b << 16);
                if (ns == 1) {
                    tiles.push_back(make_int4((int)pi, tyx, 0, -1));
                } else {
                    red.push_back(make_int4((int)pi, tyx, ns, slots));
                    for (int q = 0; q < ns; ++q) tiles.push_back(make_int4((int)pi, tyx, (ns << 16) | q, slots + q));
                    slots += ns;
                }
            }
    }
    upload(d_probs_, probs_, s, st_probs_);
    std::vector<int4> all = tiles;
    all.insert(all.end(), red.begin(), red.end());
    all.insert(all.end(), scale.begin(), scale.end());
    upload(d_tiles_, all, s, st_tiles_);
    if (slots) d_work_.reserve((size_t)slots * TM * TN);
    if (!tiles.empty()) {
        cudaEvent_t ea = nullptr, eb = nullptr;
        std::unique_lock<std::mutex> lock(g_prof.mu, std::defer_lock);
        if (g_prof.on) lock.lock();
        if (g_prof.on) {
            ea = g_prof.take();
            eb = g_prof.take();
            H2_CUDA(cudaEventRecord(ea, s));
            for (const GemmProb& p : probs_) {
                g_prof.flops += 2.0 * p.m * (double)p.n * (double)p.k;
                g_prof.bytes += 8.0 * ((double)p.m * p.k + (double)p.k * p.n + (double)p.m * p.n * (p.beta != 0.0 ? 2 : 1));
            }
            g_prof.launches += 1;
        }
        gemm_tiles_kernel<<<(unsigned)tiles.size(), NT, 0, s>>>(d_probs_.p, d_tiles_.p, d_work_.p);
        after_launch("gemm_tiles");
        if (g_prof.on) {
            H2_CUDA(cudaEventRecord(eb, s));
            g_prof.used.push_back({ea, eb});
        }
    }
    if (!red.empty()) {
        gemm_reduce_kernel<<<(unsigned)red.size(), NT, 0, s>>>(d_probs_.p, d_tiles_.p + tiles.size(), d_work_.p);
        after_launch("gemm_reduce");
    }
    if (!scale.empty()) {
        gemm_scale_kernel<<<(unsigned)scale.size(), NT, 0, s>>>(d_probs_.p, d_tiles_.p + tiles.size() + red.size());
        after_launch("gemm_scale");
    }
    probs_.clear();
}

}  // namespace h2
