// Batched construction and application of many H^2 matrices of uneven sizes.
//
// Construction: the Hessians are distributed over a pool of host workers, each with its own
// CUDA stream, so that the many small per-level launches of different Hessians overlap on the
// GPU (the per-Hessian arithmetic is exactly that of h2_build).
//
// Application: the matvec stages of all handles are merged into one launch per stage and per
// tree level (upsweep levels aligned from the leaves, downsweep levels from the root; the
// couplings of all levels and the leaf expansion + near field of all handles in one launch
// each).  Every output block carries its handle's index; the handles' bases (factors,
// workspace, permutation, X, Y) are read from a device table refreshed at every call.  For each
// (nrhs, mode) the project's autotuner times the candidate right-hand-side tiles (8, 16, 32)
// once, keeps the fastest and captures the whole launch sequence in a CUDA graph, which every
// later call replays.
#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

#include "handle.h"

namespace h2 {

int build_handle(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o,
                 h2_handle_s* h);
void finish_handle(h2_handle_s* h, const h2_build_opts& o, cudaStream_t s);

namespace {

constexpr int NT = 256;
constexpr int RMAX = 96;
constexpr int64_t kBatchTcMinNrhs = 64;   // tensor-core products from this many right-hand sides on

struct BStage {
    int kind = 0, out_y = 0, accumulate = 0;
    std::vector<MvOut> outs;
    std::vector<MvItem> items;
    DevBuf<MvOut> d_outs;
    DevBuf<MvItem> d_items;
};

struct Tuned {
    int rt = 32;
    int64_t launches = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

// Key of a captured batch sequence: right-hand sides, mode, and for the tensor-core sequence
// (whose per-handle launches take X and Y as arguments) a digest of the X/Y pointers and strides.
struct TuneKey {
    int64_t nrhs;
    int mode;
    uint64_t io;
    bool operator<(const TuneKey& o) const { return std::tie(nrhs, mode, io) < std::tie(o.nrhs, o.mode, o.io); }
};

}  // namespace
}  // namespace h2

struct h2_batch_s {
    std::vector<h2_handle_s*> hs;
    std::vector<h2::BStage> stages;
    h2::DevBuf<h2::BatchBase> d_bases;
    h2::Stager st_bases;
    std::map<h2::TuneKey, h2::Tuned> tuned;
    cudaStream_t cap = nullptr;
    // side streams of the per-handle tensor-core phases (fork/join with events, also when captured)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;
    cudaEvent_t fork_ev = nullptr;
    ~h2_batch_s() {
        for (auto& kv : tuned) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        for (auto st : side) cudaStreamDestroy(st);
        for (auto e : side_ev) cudaEventDestroy(e);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace h2 {

// defined in matvec.cu (the batched stage kernels live next to the stage bodies)
void launch_batch_transfer_rm(int mode, int kb, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                              const BatchBase* bases, int nrhs, cudaStream_t s);
void launch_batch_stage(int mode, int rt, int out_y, int accumulate, const MvOut* outs, int nouts, const MvItem* items,
                        const BatchBase* bases, int nrhs, cudaStream_t s);

namespace {

void merge(h2_batch_s* b) {
    int max_up = 0, max_down = 0;
    for (auto* h : b->hs) {
        int up = 0, down = 0;
        for (auto& st : h->plan.stages) {
            if (st.kind == H2_STAGE_UP) ++up;
            if (st.kind == H2_STAGE_DOWN) ++down;
        }
        max_up = std::max(max_up, up);
        max_down = std::max(max_down, down);
    }
    // merged order: leaf upsweep, upsweep levels (from the leaves), couplings, downsweep levels
    // (from the root), leaf expansion + near field
    const int n = 3 + max_up + max_down;
    b->stages.clear();
    b->stages.resize(n);
    auto slot = [&](int kind, int j) {
        if (kind == H2_STAGE_LEAF_UP) return 0;
        if (kind == H2_STAGE_UP) return 1 + j;
        if (kind == H2_STAGE_COUPLE) return 1 + max_up;
        if (kind == H2_STAGE_DOWN) return 2 + max_up + j;
        return 2 + max_up + max_down;
    };
    for (size_t hi = 0; hi < b->hs.size(); ++hi) {
        h2_handle_s* h = b->hs[hi];
        int up = 0, down = 0;
        for (auto& st : h->plan.stages) {
            int j = 0;
            if (st.kind == H2_STAGE_UP) j = up++;
            if (st.kind == H2_STAGE_DOWN) j = down++;
            BStage& m = b->stages[slot(st.kind, j)];
            m.kind = st.kind;
            m.out_y = st.out_to_y;
            m.accumulate = st.accumulate;
            const int ib = (int)m.items.size();
            for (const MvOut& o : st.outs) {
                MvOut x = o;
                x.beg += ib;
                x.end += ib;
                x.h = (int)hi;
                m.outs.push_back(x);
            }
            m.items.insert(m.items.end(), st.items.begin(), st.items.end());
        }
    }
    Stager stg;
    for (BStage& m : b->stages) {
        upload(m.d_outs, m.outs, nullptr, stg);
        H2_CUDA(cudaStreamSynchronize(nullptr));
        upload(m.d_items, m.items, nullptr, stg);
        H2_CUDA(cudaStreamSynchronize(nullptr));
    }
}

void launch_all(h2_batch_s* b, int mode, int rt, int nrhs, cudaStream_t s) {
    for (BStage& m : b->stages) {
        if (m.outs.empty()) continue;
        launch_batch_stage(mode, rt, m.out_y, m.accumulate, m.d_outs.p, (int)m.outs.size(), m.d_items.p,
                           b->d_bases.p, nrhs, s);
    }
}

// Tensor-core sequence (TF32 / BF16, nrhs >= 64): every handle's leaf upsweep, couplings and
// near field + leaf expansion on tcgen05, between the merged SIMT transfer sweeps of all handles.
void launch_tc(h2_batch_s* b, int mode, int md, int rt, int nrhs, const void* const* X, const int64_t* ldx,
               void* const* Y, const int64_t* ldy, cudaStream_t s) {
    constexpr int kSide = 8;
    if (b->side.empty()) {
        b->side.resize(kSide);
        b->side_ev.resize(kSide);
        for (int k = 0; k < kSide; ++k) {
            H2_CUDA(cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking));
            H2_CUDA(cudaEventCreateWithFlags(&b->side_ev[k], cudaEventDisableTiming));
        }
        H2_CUDA(cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
    }
    // right-hand-side-major workspaces when every merged transfer output has at most two items of
    // at most 64 x 64 (the register sweep kernel), else the coefficient-major SIMT sweeps
    int kb = 0;
    bool rmaj = (nrhs + 127) / 128 <= 65535;
    for (const BStage& m : b->stages) {
        if (m.kind != H2_STAGE_UP && m.kind != H2_STAGE_DOWN) continue;
        for (const MvOut& o : m.outs) {
            rmaj = rmaj && o.end - o.beg <= 2;
            kb = std::max(kb, o.rows);
        }
        for (const MvItem& it : m.items) kb = std::max({kb, it.rows, it.cols});
    }
    rmaj = rmaj && kb <= 64;
    // the handles' phase launches are independent (own operand buffers and workspaces): spread
    // them over the side streams so that the small grids of different Hessians run together
    auto phase = [&](int ph) {
        H2_CUDA(cudaEventRecord(b->fork_ev, s));
        for (int k = 0; k < kSide; ++k) H2_CUDA(cudaStreamWaitEvent(b->side[k], b->fork_ev, 0));
        for (size_t i = 0; i < b->hs.size(); ++i) {
            h2_handle_s* h = b->hs[i];
            tc_phase(h, mode, ph, X[i], ldx[i], (float*)Y[i], ldy[i], nrhs, h->ws.f32.p,
                     rmaj ? (int64_t)nrhs : h->plan.ws_rows, rmaj ? 1 : 0, b->side[i % kSide]);
        }
        for (int k = 0; k < kSide; ++k) {
            H2_CUDA(cudaEventRecord(b->side_ev[k], b->side[k]));
            H2_CUDA(cudaStreamWaitEvent(s, b->side_ev[k], 0));
        }
    };
    auto sweeps = [&](int kind) {
        for (BStage& m : b->stages) {
            if (m.outs.empty() || m.kind != kind) continue;
            if (rmaj)
                launch_batch_transfer_rm(md, kb, m.accumulate, m.d_outs.p, (int)m.outs.size(), m.d_items.p,
                                         b->d_bases.p, nrhs, s);
            else
                launch_batch_stage(md, rt, m.out_y, m.accumulate, m.d_outs.p, (int)m.outs.size(), m.d_items.p,
                                   b->d_bases.p, nrhs, s);
        }
    };
    phase(0);
    sweeps(H2_STAGE_UP);
    phase(1);
    sweeps(H2_STAGE_DOWN);
    phase(2);
}

}  // namespace

int build_batched(int count, const h2_op_fn* ops, void* const* ctxs, const h2_tree_t* trees, double tol,
                  const h2_build_opts& o, h2_handle_t* outs) {
    for (int i = 0; i < count; ++i) outs[i] = nullptr;
    const int nw = std::max(1, std::min(count, o.batch_workers > 0 ? o.batch_workers : 8));
    int worst = H2_OK;
    std::mutex mu;
    std::string first_err;
    int first_status = H2_OK;
    int next = 0;
    auto worker = [&]() {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lock(mu);
            if (first_status == H2_OK) { first_status = H2_ERR_CUDA; first_err = "stream creation failed"; }
            return;
        }
        {
            AllocScope scope(s);   // workspace blocks are reused across this worker's Hessians
            while (true) {
                int i;
                {
                    std::lock_guard<std::mutex> lock(mu);
                    if (next >= count || first_status != H2_OK) break;
                    i = next++;
                }
                auto* h = new h2_handle_s();
                try {
                    h2_build_opts oi = o;
                    oi.stream = (h2_stream_t)s;
                    if (o.q_level) oi.q_level = o.q_level + (int64_t)i * o.q_level_stride;
                    const int st = build_handle(ops[i], ctxs ? ctxs[i] : nullptr, trees[i], tol, oi, h);
                    finish_handle(h, oi, s);
                    std::lock_guard<std::mutex> lock(mu);
                    outs[i] = h;
                    worst = std::max(worst, st);
                } catch (const Error& e) {
                    delete h;
                    std::lock_guard<std::mutex> lock(mu);
                    if (first_status == H2_OK) { first_status = e.status; first_err = e.what(); }
                } catch (...) {
                    delete h;
                    std::lock_guard<std::mutex> lock(mu);
                    if (first_status == H2_OK) { first_status = H2_ERR_CUDA; first_err = "unknown failure"; }
                }
            }
        }
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    };
    std::vector<std::thread> pool;
    for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
    for (auto& t : pool) t.join();
    if (first_status != H2_OK) {
        for (int i = 0; i < count; ++i) {
            delete outs[i];
            outs[i] = nullptr;
        }
        fail(first_status, "h2_build_batched: " + first_err);
    }
    return worst;
}

h2_batch_s* batch_create(int count, const h2_handle_t* hs) {
    auto* b = new h2_batch_s();
    try {
        for (int i = 0; i < count; ++i) b->hs.push_back(hs[i]);
        merge(b);
        H2_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    } catch (...) {
        delete b;
        throw;
    }
    return b;
}

void batch_matvec(h2_batch_s* b, const void* const* X, const int64_t* ldx, void* const* Y, const int64_t* ldy,
                  int64_t nrhs, int mode, cudaStream_t s) {
    const int n = (int)b->hs.size();
    std::vector<BatchBase> bases(n);
    for (int i = 0; i < n; ++i) {
        h2_handle_s* h = b->hs[i];
        const int64_t need = h->plan.ws_rows * nrhs;
        BatchBase& x = bases[i];
        switch (mode) {
            case H2_FP64:
                h->ws.f64.reserve((size_t)need);
                x.fac = h->fac64.p;
                x.ws = h->ws.f64.p;
                break;
            case H2_FP32:
            case H2_TF32:
            case H2_TF32X3:
                if (!h->fac32.p) fail(H2_ERR_INVALID_ARG, "h2_batch_matvec: FP32 copy of the factors was not kept");
                h->ws.f32.reserve((size_t)need);
                x.fac = h->fac32.p;
                x.ws = h->ws.f32.p;
                break;
            case H2_BF16:
                if (!h->fac16.p) fail(H2_ERR_INVALID_ARG, "h2_batch_matvec: BF16 copy of the factors was not kept");
                h->ws.f32.reserve((size_t)need);
                x.fac = h->fac16.p;
                x.ws = h->ws.f32.p;
                break;
            default:
                fail(H2_ERR_INVALID_ARG, "h2_batch_matvec: unknown mode");
        }
        if (!X[i] || !Y[i] || ldx[i] < h->N || ldy[i] < h->N) fail(H2_ERR_INVALID_ARG, "h2_batch_matvec: bad X/Y");
        x.ws_ld = h->plan.ws_rows;
        x.perm = h->d_perm.p;
        x.X = X[i];
        x.ldx = ldx[i];
        x.Y = Y[i];
        x.ldy = ldy[i];
    }
    upload(b->d_bases, bases, s, b->st_bases);
    // SIMT arithmetic type of the merged stages (TF32 factors are the FP32 copy)
    const int md = (mode == H2_TF32 || mode == H2_TF32X3) ? H2_FP32 : mode;
    bool tc = (mode == H2_TF32 || mode == H2_TF32X3 || mode == H2_BF16) && nrhs >= kBatchTcMinNrhs;
    for (auto* h : b->hs) tc = tc && tc_supported(h) && ((mode == H2_BF16) ? h->tc.W16.p : h->tc.W32.p);
    uint64_t io = 0;
    if (tc) {
        for (int i = 0; i < n; ++i) {
            tc_reserve(b->hs[i], mode, (int)nrhs);
            // buffers the per-handle launches take as arguments (the captured graph holds them)
            for (uint64_t v : {(uint64_t)(uintptr_t)X[i], (uint64_t)ldx[i], (uint64_t)(uintptr_t)Y[i], (uint64_t)ldy[i],
                               (uint64_t)(uintptr_t)b->hs[i]->ws.f32.p, (uint64_t)(uintptr_t)b->hs[i]->tc.opnd.p})
                io = mix64(io ^ v);
        }
    }
    auto seq = [&](int rt, cudaStream_t st) {
        if (tc) launch_tc(b, mode, md, rt, (int)nrhs, X, ldx, Y, ldy, st);
        else launch_all(b, md, rt, (int)nrhs, st);
    };
    const TuneKey key{nrhs, tc ? mode : md, io};
    auto it = b->tuned.find(key);
    if (it == b->tuned.end()) {
        // autotune the right-hand-side tile of the SIMT stages on this call's data, then capture
        H2_CUDA(cudaStreamSynchronize(s));
        Tuned t;
        float best = 1e30f;
        cudaEvent_t e0, e1;
        H2_CUDA(cudaEventCreate(&e0));
        H2_CUDA(cudaEventCreate(&e1));
        for (int rt : {8, 16, 32}) {
            seq(rt, s);   // warm-up
            H2_CUDA(cudaEventRecord(e0, s));
            seq(rt, s);
            H2_CUDA(cudaEventRecord(e1, s));
            H2_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; t.rt = rt; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        const int64_t l0 = g_launches.load();
        H2_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        try {
            seq(t.rt, b->cap);
        } catch (...) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(b->cap, &junk);
            if (junk) cudaGraphDestroy(junk);
            throw;
        }
        H2_CUDA(cudaStreamEndCapture(b->cap, &t.graph));
        H2_CUDA(cudaGraphInstantiate(&t.exec, t.graph, 0));
        t.launches = g_launches.load() - l0;
        g_launches.fetch_sub(t.launches);   // counted at every replay
        it = b->tuned.emplace(key, t).first;
    }
    H2_CUDA(cudaGraphLaunch(it->second.exec, s));
    g_launches.fetch_add(it->second.launches, std::memory_order_relaxed);
}

int batch_tuned(h2_batch_s* b, int64_t nrhs, int mode) {
    const int md = (mode == H2_TF32 || mode == H2_TF32X3) ? H2_FP32 : mode;
    for (const auto& kv : b->tuned)
        if (kv.first.nrhs == nrhs && (kv.first.mode == mode || kv.first.mode == md)) return kv.second.rt;
    return 0;
}

}  // namespace h2
