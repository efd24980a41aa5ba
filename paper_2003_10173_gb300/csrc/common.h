// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/h2.h"

namespace h2 {

// Error carried through the host code as an exception and converted to a
// status code at the C ABI.
struct Error : std::runtime_error {
    int status;
    Error(int s, const std::string& m) : std::runtime_error(m), status(s) {}
};

[[noreturn]] void fail(int status, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);
#define H2_CUDA(call) ::h2::check_cuda((call), #call)

// SplitMix64 (Steele, Lea, Flood 2014): output finaliser and the i-th output of
// a generator seeded with `key`.
__host__ __device__ inline uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

__host__ __device__ inline uint64_t splitmix_at(uint64_t key, uint64_t idx) {
    return mix64(key + (idx + 1ull) * 0x9E3779B97F4A7C15ull);
}

extern std::atomic<int64_t> g_launches;
// Call after every kernel launch: counts it and turns a launch error into an Error.
void after_launch(const char* name);

// ---- device memory ---------------------------------------------------------
// Device blocks come from dev_alloc_bytes and go back through dev_free; pinned host
// blocks from host_alloc_bytes / host_free.  Outside an AllocScope these are plain
// cudaMalloc / cudaFree and cudaMallocHost / cudaFreeHost (each free waits for the
// whole device).  Allocation failure -> H2_ERR_OOM.
void* dev_alloc_bytes(size_t bytes);
void dev_free(void* p);
void* host_alloc_bytes(size_t bytes);
void host_free(void* p);
// Device bytes the library holds (kept scope blocks included), and an optional cap (<= 0: none)
// above which allocations fail with H2_ERR_OOM.
int64_t dev_live_bytes();
void dev_alloc_limit(int64_t bytes);

// While an AllocScope is alive on a thread, the blocks that this thread allocated inside
// the scope and then frees are kept on per-thread free lists and handed out again to the
// thread's later allocations (best fit, sizes rounded up by at most a quarter) instead of
// being returned to the driver: no device-wide wait per free, which lets several threads
// build on their own streams without serialising one another.  Requirement: all device
// work that the thread issues on scope blocks runs on the scope's stream (then a reused
// device block is stream-ordered after its last use), and a pinned block is freed only
// after the copies from or to it have completed.  The scope's end synchronises the stream
// and returns the kept blocks.  A scope opened while another is alive on the thread does
// nothing.
class AllocScope {
  public:
    explicit AllocScope(cudaStream_t s);
    ~AllocScope();
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;

  private:
    bool owner_ = false;
};

// Owning device buffer on dev_alloc_bytes / dev_free.
template <class T>
struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    DevBuf() = default;
    explicit DevBuf(size_t count) { alloc(count); }
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
    DevBuf& operator=(DevBuf&& o) noexcept {
        if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
        return *this;
    }
    ~DevBuf() { release(); }
    void alloc(size_t count);
    void release() {
        if (p) dev_free(p);
        p = nullptr;
        n = 0;
    }
    // grow to at least count elements (contents are not preserved)
    void reserve(size_t count) {
        if (count > n) { release(); alloc(count); }
    }
};

template <class T>
void DevBuf<T>::alloc(size_t count) {
    n = count;
    p = count ? static_cast<T*>(dev_alloc_bytes(count * sizeof(T))) : nullptr;
}

// Pinned host staging area for asynchronous uploads of small host tables (a
// pageable cudaMemcpyAsync would synchronise the stream).  The buffer is reused
// only after the previous copy from it has completed.
struct Stager {
    void* host = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
    Stager() = default;
    Stager(const Stager&) = delete;
    Stager& operator=(const Stager&) = delete;
    ~Stager();
    void copy(void* dst, const void* src, size_t bytes, cudaStream_t s);
};

// Pinned host scratch for small synchronous reads and writes of device scalars (grown on demand).
struct Pinned {
    void* p = nullptr;
    size_t cap = 0;
    ~Pinned() { host_free(p); }
    template <class T>
    T* get(size_t n) {
        if (n * sizeof(T) > cap) {
            host_free(p);
            p = nullptr;
            cap = 0;
            p = host_alloc_bytes(n * sizeof(T) + 64);
            cap = n * sizeof(T) + 64;
        }
        return static_cast<T*>(p);
    }
};

template <class T>
void upload(DevBuf<T>& d, const std::vector<T>& h, cudaStream_t s, Stager& st) {
    d.reserve(h.size());
    if (!h.empty()) st.copy(d.p, h.data(), h.size() * sizeof(T), s);
}

// ---- batched FP64 GEMM (gemm.cu) -------------------------------------------
// C = alpha * op(A) * op(B) + beta * C, column-major, op = transpose if t* != 0.
struct GemmProb {
    const double* A;
    const double* B;
    double* C;
    int m, n, k;
    int lda, ldb, ldc;
    int ta, tb;
    double alpha, beta;
    int tm = 64;   // tile rows (64, 32 or 16), chosen by GemmBatch::run
    int tc = 0;    // 1: the problem is computed transposed (C^T = op(B)^T op(A)^T), stored back as C
};

// Runs a list of independent problems (their C regions must not overlap) in
// as few launches as possible; long reductions are split deterministically.
class GemmBatch {
  public:
    void add(const GemmProb& p) {
        if (p.m > 0 && p.n > 0) probs_.push_back(p);
    }
    void add(const double* A, int lda, int ta, const double* B, int ldb, int tb, double* C, int ldc,
             int m, int n, int k, double alpha, double beta) {
        add(GemmProb{A, B, C, m, n, k, lda, ldb, ldc, ta, tb, alpha, beta});
    }
    size_t size() const { return probs_.size(); }
    void clear() { probs_.clear(); }
    void run(cudaStream_t s);

  private:
    std::vector<GemmProb> probs_;
    Stager st_probs_, st_tiles_;
    DevBuf<GemmProb> d_probs_;
    DevBuf<int4> d_tiles_;
    DevBuf<double> d_work_;
    DevBuf<int4> d_red_;
};

void gemm_profile_enable(int on);
void gemm_profile_read(double* ms, double* flops, int64_t* launches, double* bytes);
int gemm_profile_on();
// The same switch times the stacked QR (which 0) and truncated-SVD (which 1) launches: device
// milliseconds, algorithmic flops of their Householder QRs (2 m n^2 - 2 n^3 / 3 for an m x n stack,
// m >= n; plus 4 c^3 / 3 for the pivoted QR of the SVD's triangle; the Jacobi rotations are not
// counted) and launches since the last read.
void stack_profile_read(int which, double* ms, double* flops, int64_t* launches);

// ---- dense linear-algebra kernels (la.cu) ----------------------------------
// Householder QR of panels in place with explicit orthonormal factor written to Q.
// Panel i: m_i x c rows/cols at Y + y_off[i] (ld ldy), Q at Q + q_off[i] (ld ldq).
void panel_qr(int count, const int64_t* d_y_off, const int64_t* d_q_off, const int* d_m, int c,
              double* Y, int ldy, double* Q, int ldq, cudaStream_t s);
// Shared-memory TSQR of panels (m_i > c rows, c <= 16 columns): explicit orthonormal factor
// of Y_i written to Q (Y_i is used as scratch).  Host arrays y_off, q_off, m.
struct TsqrChunk {
    int64_t y_off;   // first row of the chunk in Y
    int64_t q_off;   // first row of the chunk in Q
    int rows;
    int64_t r_off;   // offset of the chunk's R in the R buffer, -1 for single-chunk panels
    int64_t qs_off;  // offset of the chunk's c x c block in the stacked factor buffer
    int ldqs;
};
constexpr int kTsqrChunk = 512;      // target rows per chunk
constexpr int kTsqrMaxChunks = 96;   // chunks per panel (stacked R: <= 1536 x 16)
constexpr int kTsqrMaxRows = 1536;   // shared-memory rows of one CTA
struct TsqrWork {
    DevBuf<TsqrChunk> d_chunks, d_multi, d_multi2;
    DevBuf<int4> d_roots, d_roots2;
    DevBuf<double> Rbuf, Qs, R2, Qs2;
    Stager st_chunks, st_multi, st_roots, st_multi2, st_roots2;
};
void tsqr_panels(int count, const int64_t* y_off, const int64_t* q_off, const int* m, int c, double* Y, int ldy,
                 double* Q, int ldq, TsqrWork& w, cudaStream_t s);
// Sign convention of orthonormal bases: for every item, the column of `rows` entries at Q + q_off
// is negated when its dot product with the column at Y + y_off is negative, so that the basis
// is the Q factor of Y = QR with a non-negative diagonal of R.
struct SignItem {
    int64_t q_off, y_off;
    int rows;
};
void align_signs(int count, const SignItem* d_items, double* Q, const double* Y, cudaStream_t s);
// Maximum column 2-norm of each panel: out[i] = max_j ||Y_i[:, j]||.
void panel_colnorm_max(int count, const int64_t* d_y_off, const int* d_m, int c, const double* Y,
                       int ldy, double* out, cudaStream_t s);

// ---- stacked QR and truncated SVD (svd.cu) ----------------------------------
// One row block of a stacked matrix: rows x c at p (column-major, leading dimension ld).
// tri = 1: the block is upper triangular (its row i is zero in the columns before i), which the
// stacked QR uses to skip the zero part of every reflector.
struct RowSeg {
    const double* p;
    int rows;
    int ld;
    int tri = 0;
};
// A matrix given as the stack of segments [seg_begin, seg_end), each with c columns.
struct StackJob {
    int seg_begin, seg_end;
    int c;
    double* out;      // stacked_r: R (c x c, upper, zeros below); stacked_svd_trunc: U (c x k)
    int ldo;          // leading dimension of out
    int* k_out;       // stacked_svd_trunc: number of kept singular vectors
    double* sv_out;   // stacked_svd_trunc: all c singular values, descending (may be null)
};
struct CholItem;
struct StackWork {
    DevBuf<unsigned char> d_chol;
    Stager st_chol;
    DevBuf<StackJob> d_jobs, d_jobs2;
    DevBuf<RowSeg> d_segs, d_segs2;
    DevBuf<double> parts;
    Stager st_jobs, st_jobs2, st_segs, st_segs2;
    // side streams of the width classes of one stacked_r pass (created on first use), so that
    // the classes' launches overlap instead of each waiting for the previous one's tail
    static constexpr int kClasses = 6;
    cudaStream_t side[kClasses] = {};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[kClasses] = {};
    StackWork() = default;
    StackWork(const StackWork&) = delete;
    StackWork& operator=(const StackWork&) = delete;
    ~StackWork();
};
// R factors (Householder) of every job's stacked matrix (c <= 144 columns; any row count:
// matrices above a few thousand rows are split over several CTAs).  The stacked matrices must
// not overlap the outputs.  Host vectors; device pointers inside.
void stacked_r(const std::vector<StackJob>& jobs, const std::vector<RowSeg>& segs, StackWork& w, cudaStream_t s);
// For every job, W^T is the stacked matrix (W is c x rows, c <= 96): the left singular vectors
// of W with singular value > thr (at most kmax; *cap_flag = 1 if the cap removed one), sorted by
// descending singular value, written to out (c x k); k to *k_out.  QR of W^T, then one-sided
// Jacobi on the c x c triangle.
void stacked_svd_trunc(const std::vector<StackJob>& jobs, const std::vector<RowSeg>& segs, StackWork& w, double thr,
                       int kmax, int* d_cap_flag, cudaStream_t s);
int svd_max_order();
// Widest matrix (columns) that stacked_r factors in shared memory; wider groups of the
// recompression use Gram matrices instead.
int stacked_r_max_columns();
// Factors of small symmetric positive semidefinite m x m matrices (m <= 96) by Cholesky with
// symmetric pivoting: for every item, out (m x m, leading dimension ldo) receives F^T with
// F F^T = G (G: leading dimension ldg, lower triangle used); the factorisation stops once the
// largest remaining pivot is at or below m 2^-52 max(diag G) (those rows of out are zero).
struct CholItem {
    const double* G;
    double* out;
    int m, ldg, ldo;
};
void psd_chol_small(const std::vector<CholItem>& items, StackWork& w, cudaStream_t s);

// ---- small helper kernels (misc.cu) ------------------------------------------
void fill_zero(double* p, size_t count, cudaStream_t s);
// Omega (original order, N x ncols, ld N): Gaussian at rows whose tree position is in a
// child-0 box of `level`, else 0; tree-order copy in Om_tree (may be null).
void probe_fill(int64_t N, int ncols, int col0, const int32_t* d_perm, const int32_t* d_row_box,
                int level_shift, uint64_t seed, int stream_id, int level, double* Om_orig,
                double* Om_tree, cudaStream_t s);
// Coloured probes (original order, N x q*ncolors, ld N; tree-order copy in Om_tree if not null):
// column block c is Gaussian on the rows whose box at `level` (row_box >> level_shift) has
// colour c in d_color (-1: no probes), zero elsewhere.
void probe_fill_colored(int64_t N, int q, int ncolors, const int32_t* d_perm, const int32_t* d_row_box,
                        int level_shift, const int32_t* d_color, uint64_t seed, int stream_id, int level,
                        double* Om_orig, double* Om_tree, cudaStream_t s);
// power-iteration start vector (tree-order Gaussian) scattered to original order
void gaussian_vector(int64_t N, const int32_t* d_perm, uint64_t seed, int stream_id, double* x_orig,
                     cudaStream_t s);
// dst_tree[i, j] = src_orig[perm[i], j]
void gather_rows(int64_t N, int ncols, const int32_t* d_perm, const double* src, int64_t lds,
                 double* dst, int64_t ldd, cudaStream_t s);
// dst_orig[perm[i], j] = src_tree[i, j]
void scatter_rows(int64_t N, int ncols, const int32_t* d_perm, const double* src, int64_t lds,
                  double* dst, int64_t ldd, cudaStream_t s);
// sum over blocks of |x|^2 and a flag for non-finite values: out[0] += ..., out[1] = 1 if nan
void scan_finite(int64_t N, int ncols, const double* x, int64_t ld, int* d_flag, cudaStream_t s);
// out[i] = sum_{j in list i} in[j] for count matrices of size len_i (in and out may be one buffer
// when no output is also an input)
void sum_lists(int count, const int64_t* d_out_off, const int* d_len, const int* d_begin,
               const int* d_end, const int64_t* d_in_off, const double* in, double* out,
               int accumulate, cudaStream_t s);
// norms of vectors: out[j] = ||x[:, j]||^2
void col_sqnorms(int64_t N, int ncols, const double* x, int64_t ld, double* out, cudaStream_t s);
void scale_cols(int64_t N, int ncols, double* x, int64_t ld, const double* d_scale, cudaStream_t s);

// Block descriptors for copies between matrices with explicit offsets and leading dimensions.
struct BlkDesc {
    int64_t src_off;
    int64_t dst_off;
    int rows, cols;
    int lds, ldd;
};
enum { BLK_COPY = 0, BLK_IDENTITY = 1, BLK_SYMMETRIZE = 2 };
// COPY: dst = src; IDENTITY: dst = I (src unused); SYMMETRIZE: dst = (src + src^T)/2 (square)
void block_op(int kind, int count, const BlkDesc* d_desc, const double* src, double* dst, cudaStream_t s);
// Copies of more than kSplitEntries entries split into row chunks, so that one CTA per descriptor
// copies a bounded piece (identity and symmetrisation blocks are left whole).
constexpr int kSplitEntries = 1 << 16;
inline std::vector<BlkDesc> split_copies(const std::vector<BlkDesc>& d) {
    std::vector<BlkDesc> out;
    out.reserve(d.size());
    for (const BlkDesc& b : d) {
        if ((int64_t)b.rows * b.cols <= kSplitEntries || b.rows < 2) {
            out.push_back(b);
            continue;
        }
        const int chunk = std::max(1, kSplitEntries / std::max(b.cols, 1));
        for (int r = 0; r < b.rows; r += chunk)
            out.push_back(BlkDesc{b.src_off + r, b.dst_off + r, std::min(chunk, b.rows - r), b.cols, b.lds, b.ldd});
    }
    return out;
}
uint64_t rng_key(uint64_t seed, int stream_id, int level);
// C (n x n, lower, ld n) with C C^T = A for a symmetric positive semidefinite A (ld n, lower
// triangle used and overwritten); pivots at rounding level leave their column of C zero.
void psd_cholesky(double* A, int n, double* C, cudaStream_t s);

}  // namespace h2
