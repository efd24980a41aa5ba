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

#include "handle.h"

namespace h2 {

int build_handle(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o,
                 h2_handle_s* h);
void finish_handle(h2_handle_s* h, const h2_build_opts& o, cudaStream_t s);

namespace {

constexpr int NT = 256;
constexpr int RMAX = 96;

struct BStage {
    int kind = 0, out_y = 0, accumulate = 0;
    std::vector<MvOut> outs;
    std::vector<MvItem> items;
    DevBuf<MvOut> d_outs;
    DevBuf<MvItem> d_items;
};

struct Tuned {
    int rt = 32;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

}  // namespace
}  // namespace h2

struct h2_batch_s {
    std::vector<h2_handle_s*> hs;
    std::vector<h2::BStage> stages;
    h2::DevBuf<h2::BatchBase> d_bases;
    h2::Stager st_bases;
    std::map<std::pair<int64_t, int>, h2::Tuned> tuned;
    cudaStream_t cap = nullptr;
    ~h2_batch_s() {
        for (auto& kv : tuned) {
            if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
            if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        }
        if (cap) cudaStreamDestroy(cap);
    }
};

namespace h2 {

// defined in matvec.cu (the batched stage kernel lives next to the stage body)
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

}  // namespace

int build_batched(int count, const h2_op_fn* ops, void* const* ctxs, const h2_tree_t* trees, double tol,
                  const h2_build_opts& o, h2_handle_t* outs) {
    for (int i = 0; i < count; ++i) outs[i] = nullptr;
    const int nw = std::max(1, std::min(count, 8));
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
    const int md = (mode == H2_TF32) ? H2_FP32 : mode;
    auto key = std::make_pair(nrhs, md);
    auto it = b->tuned.find(key);
    if (it == b->tuned.end()) {
        // autotune the right-hand-side tile on this call's data, then capture the sequence
        H2_CUDA(cudaStreamSynchronize(s));
        Tuned t;
        float best = 1e30f;
        cudaEvent_t e0, e1;
        H2_CUDA(cudaEventCreate(&e0));
        H2_CUDA(cudaEventCreate(&e1));
        for (int rt : {8, 16, 32}) {
            launch_all(b, md, rt, (int)nrhs, s);   // warm-up
            H2_CUDA(cudaEventRecord(e0, s));
            launch_all(b, md, rt, (int)nrhs, s);
            H2_CUDA(cudaEventRecord(e1, s));
            H2_CUDA(cudaEventSynchronize(e1));
            float ms = 0.f;
            H2_CUDA(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; t.rt = rt; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        H2_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        launch_all(b, md, t.rt, (int)nrhs, b->cap);
        H2_CUDA(cudaStreamEndCapture(b->cap, &t.graph));
        H2_CUDA(cudaGraphInstantiate(&t.exec, t.graph, 0));
        it = b->tuned.emplace(key, t).first;
    }
    H2_CUDA(cudaGraphLaunch(it->second.exec, s));
    int64_t nk = 0;
    for (const BStage& m : b->stages) nk += m.outs.empty() ? 0 : 1;
    g_launches.fetch_add(nk, std::memory_order_relaxed);
}

int batch_tuned(h2_batch_s* b, int64_t nrhs, int mode) {
    const int md = (mode == H2_TF32) ? H2_FP32 : mode;
    auto it = b->tuned.find(std::make_pair(nrhs, md));
    return it == b->tuned.end() ? 0 : it->second.rt;
}

}  // namespace h2
