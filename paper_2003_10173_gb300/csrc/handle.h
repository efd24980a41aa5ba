// Built H^2 matrix: factor storage, offsets and the matvec plan.
#pragma once

#include <cuda_bf16.h>

#include <functional>
#include <memory>

#include "common.h"
#include "tree.h"

namespace h2 {

// One product of a matvec stage: out_block += op(M) * in_block.
// op(M) is rows x cols; M at factor offset m_off with leading dimension ldm,
// transposed if trans.  The input block starts at row in_off of the input buffer.
struct MvItem {
    int64_t m_off;
    int64_t in_off;
    int ldm;
    int rows, cols;
    int trans;
    int in_ld;
};

// One output block of a stage with its list of items [beg, end).
struct MvOut {
    int64_t out_off;
    int out_ld;
    int rows;
    int beg, end;
    int h = 0;          // handle index in a batch (0 for single-handle plans)
};

// Per-handle bases of a batched matvec launch.
struct BatchBase {
    const void* fac;
    void* ws;
    int64_t ws_ld;
    const int32_t* perm;
    const void* X;
    int64_t ldx;
    void* Y;
    int64_t ldy;
};

// A stage: its outputs write internal coefficient buffers, or the caller's Y via
// the tree permutation; its inputs read internal buffers, or the caller's X.
struct MvStage {
    int kind = 0;           // H2_STAGE_* of this stage
    std::vector<MvOut> outs;
    std::vector<MvItem> items;
    int out_to_y = 0;       // outputs are rows of Y (tree positions, scattered by perm)
    int in_from_x = 0;      // bit 0: items with in_ld < 0 read X through perm
    int accumulate = 0;     // add to the existing output instead of overwriting
    DevBuf<MvOut> d_outs;
    DevBuf<MvItem> d_items;
    int max_rows = 0, max_cols = 0;
};

// A stored (lower-triangle or diagonal) block used in both orientations by the
// small-nrhs scatter path: out_t += M in_s and, unless diag, out_s += M^T in_t.
struct SymItem {
    int64_t m_off;
    int64_t in_s, out_t, in_t, out_s;
    int ldm, rows, cols, diag;
};

struct SymStage {
    int kind = 0;
    int via_perm = 0;       // inputs/outputs are X/Y rows (tree positions, through perm)
    std::vector<SymItem> items;
    DevBuf<SymItem> d_items;
};

struct MatvecPlan {
    std::vector<MvStage> stages;       // gather path (any nrhs)
    int64_t ws_rows = 0;     // rows of the internal coefficient workspace (per right-hand side)
    int64_t yh_row0 = 0;     // first row of the yh part of the workspace
    // small-nrhs path: gather stages for the tree sweeps, scatter stages for couplings and near field
    std::vector<MvStage> small_up, small_down;   // leaf upsweep + upsweep; downsweep
    MvStage small_expand;                        // Y += U_t yh_t (accumulate)
    SymStage couple, near;
};

// Tensor-core products (tcgen05): output blocks with lists of items; an item multiplies rows
// [a_row, a_row + k) of the padded operand buffer by a pre-laid-out n x k B tile.
struct TcOut {
    int64_t out_off;   // tree row (to_y) or workspace row of the output block
    int rows;          // rows written
    int n;             // MMA N (rows padded to 16)
    int beg, end;      // item range
    int to_y;          // 1: write Y through the permutation, 0: write the coefficient workspace
};
struct TcItem {
    int64_t a_row;     // first operand row
    int k;             // MMA K extent (padded to 16)
    int64_t b_off;     // byte offset of the B tile in the tile pool of the precision
};
struct TcGroup {       // consecutive outputs computed by one CTA, side by side in tensor memory
    int obeg, oend;    // output range
    int ibeg, iend;    // their items (split TF32: the tripled list has its own groups)
};
struct TcTileSrc {     // how a B tile is made from the FP64 factors
    int64_t m_off, dst;
    int ldm, trans, rows, cols, n, k;
};
struct TcStage {
    std::vector<TcOut> outs;
    std::vector<TcItem> items;     // b_off holds the tile index until packing
    std::vector<TcGroup> groups;
    DevBuf<TcGroup> d_groups, d_groups32x3;
    int tmem_cols = 32;            // tensor-memory columns per CTA (power of two >= the widest group)
    int kmax_item = 0, nmax_out = 0;   // largest item K and output N (choose the operand ring's tiles)
    DevBuf<TcOut> d_outs, d_outs32x3;
    DevBuf<TcItem> d_items16, d_items32, d_items32x3;   // split TF32: three items per product
};
struct TcPlan {
    int LP = 0;              // padded leaf rows
    int nleaf = 0;           // 0: tensor-core path unavailable
    int64_t op_rows = 0;     // rows of the operand buffer (X of leaves, xh and yh of boxes)
    int64_t w_elems = 0;     // elements of a tile pool
    int cur_eb = 0;
    TcStage leaf_up, couple, near;
    std::vector<int4> xh_boxes, yh_boxes;    // (operand row, k, padded k)
    std::vector<int64_t> xh_src, yh_src;     // workspace rows
    DevBuf<int4> d_xh_boxes, d_yh_boxes;
    DevBuf<int64_t> d_xh_src, d_yh_src, d_leaf_start;
    DevBuf<int> d_leaf_size, d_err;
    DevBuf<unsigned char> W16, W32, opnd;
};

struct Workspace {
    DevBuf<double> f64;
    DevBuf<float> f32;
    int64_t nrhs_cap = 0;
};

}  // namespace h2

// A captured h2_matvec launch sequence and what it was captured for.
struct MvGraph {
    const void* X = nullptr;
    const void* Y = nullptr;
    const void* ws = nullptr;
    const void* opnd = nullptr;
    int64_t ldx = 0, ldy = 0, nrhs = 0;
    int mode = 0;
    int uses = 0;                      // calls seen with this key (captured on the second)
    int64_t launches = 0;              // kernels in the graph
    uint64_t stamp = 0;                // last use (replacement order)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

struct h2_handle_s {
    std::shared_ptr<h2_tree_s> tree;
    int L = 0;
    int64_t N = 0;
    // ranks of every box: k[koff[l] + box]
    std::vector<int> k;
    std::vector<int64_t> koff;
    // factor offsets into fac (entries)
    std::vector<int64_t> u_off;              // per leaf: |t| x k_t, ld |t|
    std::vector<int64_t> uh_off;             // per box at levels 0..L-1 with children: (k_c1+k_c2) x k_p, ld k_c1+k_c2
    std::vector<std::vector<std::pair<int, int>>> far_lower;  // [level] (t, s), t > s
    std::vector<std::vector<int64_t>> s_off;                  // [level][i]: k_t x k_s, ld k_t
    std::vector<std::pair<int, int>> near_lower;              // (t, s), t >= s
    std::vector<int64_t> d_off;                                // |t| x |s|, ld |t|
    int64_t fac_entries = 0;
    h2::DevBuf<double> fac64;
    h2::DevBuf<float> fac32;
    h2::DevBuf<__nv_bfloat16> fac16;
    h2::DevBuf<int32_t> d_perm;
    h2::MatvecPlan plan;
    h2::TcPlan tc;
    h2::Workspace ws;
    // device staging of X and Y for h2_matvec_host (grown to the largest call)
    h2::DevBuf<unsigned char> host_x, host_y;
    h2_stats stats{};
    // per-stage timing (h2_profile)
    int prof = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    double prof_ms[H2_STAGE_COUNT] = {0};
    int64_t prof_n[H2_STAGE_COUNT] = {0};
    // CUDA graphs of repeated h2_matvec calls (a few keys, least recently used replaced)
    std::vector<MvGraph> graphs;
    uint64_t graph_clock = 0;
    cudaStream_t cap = nullptr;
    // second stream of the small-nrhs matvec (near field beside the tree sweeps) and its events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~h2_handle_s() {
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (auto& g : graphs) {
            if (g.exec) cudaGraphExecDestroy(g.exec);
            if (g.graph) cudaGraphDestroy(g.graph);
        }
        if (cap) cudaStreamDestroy(cap);
        for (auto e : ev_pool) cudaEventDestroy(e);
        for (auto& u : ev_used) {
            cudaEventDestroy(u.second.first);
            cudaEventDestroy(u.second.second);
        }
    }
    int64_t entries_U = 0, entries_E = 0, entries_S = 0, entries_D = 0;
};

namespace h2 {
// Computes factor offsets from k (and the tree), allocates fac64.
void layout_factors(h2_handle_s* h);
// Builds and uploads the matvec plan from the factor layout.
void build_plan(h2_handle_s* h, cudaStream_t s);
// Creates the requested reduced-precision copies of the factors.
void make_copies(h2_handle_s* h, int keep_fp32, int keep_bf16, cudaStream_t s);
void run_matvec(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs,
                int mode, cudaStream_t s);
void profile_read(h2_handle_s* h, double* ms, int64_t* n);
void run_matvec_noalloc(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs,
                        int mode, cudaStream_t s);
// X, Y in host memory: copy in, run_matvec on device staging buffers, copy out, synchronise.
void run_matvec_host(h2_handle_s* h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs, int mode,
                     cudaStream_t s);
bool tc_supported(const h2_handle_s* h);
void tc_reserve(h2_handle_s* h, int mode, int nrhs);
// ws_rmaj: the coefficient workspace is right-hand-side-major (ws[row * ws_ld + rhs]) instead of
// coefficient-major (ws[row + rhs * ws_ld]).
void tc_phase(h2_handle_s* h, int mode, int phase, const void* X, int64_t ldx, float* Y, int64_t ldy, int nrhs,
              float* ws, int64_t ws_ld, int ws_rmaj, cudaStream_t s);
void tc_prepare(h2_handle_s* h, int want_bf16, int want_tf32, cudaStream_t s);
void tc_matvec(h2_handle_s* h, int mode, const void* X, int64_t ldx, float* Y, int64_t ldy, int nrhs, float* ws,
               int64_t ws_ld, int ws_rmaj, cudaStream_t s, const std::function<void(int)>& sweeps,
               const std::function<void(int, std::function<void()>)>& timed);
int tc_device_error(h2_handle_s* h);
}  // namespace h2
