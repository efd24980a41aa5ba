/*
 * h2.h - C ABI of the GB300 H^2 Hessian library.
 *
 * Builds a hierarchical (H^2) approximation of a symmetric PDE-constrained
 * Hessian using only Hessian-vector products (randomized peeling, Section 3.3
 * of Ambartsumyan et al., "Hierarchical matrix approximations of Hessians
 * arising in inverse problems governed by PDEs", arXiv 2003.10173) and applies
 * it to many vectors at once (four-stage matvec, Section 3.2, Eq. (3.2)).
 *
 * Conventions for every entry point:
 *   - Return value: H2_OK (0) on success, a negative H2_ERR_* code on error, a
 *     positive H2_WARN_* code when the call completed with a caveat.  No C++
 *     exception crosses this boundary.  h2_error_string() names a code and
 *     h2_last_error() gives the calling thread's last detailed message.
 *   - Matrices are column-major with an explicit leading dimension.  Vectors and
 *     right-hand sides are in the caller's (original) node order; the library
 *     reorders internally.
 *   - "device" pointers are CUDA global-memory pointers on the current device;
 *     "host" pointers are ordinary CPU memory.
 *   - The caller owns every buffer it passes; the library owns trees, handles and
 *     operator contexts it creates and frees them in the matching *_free/destroy.
 *     Freeing NULL is a no-op.
 *   - A handle is not thread-safe; distinct handles may be used concurrently on
 *     distinct streams.
 *   - Streams are passed as h2_stream_t (a cudaStream_t cast to void*; NULL is the
 *     legacy default stream).  Calls that launch work are asynchronous with
 *     respect to the host unless stated otherwise.
 */
#ifndef H2_H
#define H2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void* h2_stream_t;
typedef struct h2_tree_s* h2_tree_t;
typedef struct h2_handle_s* h2_handle_t;
typedef struct h2_batch_s* h2_batch_t;

/* ---- status codes ------------------------------------------------------- */
enum {
    H2_OK = 0,
    H2_ERR_INVALID_ARG = -1,   /* bad size, pointer, option or unsupported mode */
    H2_ERR_CUDA = -2,          /* a CUDA runtime call or kernel launch failed */
    H2_ERR_OP_FAILED = -3,     /* the user's Hessian operator returned nonzero */
    H2_ERR_NAN = -4,           /* NaN or Inf found in operator samples */
    H2_ERR_OOM = -5,           /* device allocation failed */
    H2_ERR_DEVICE_CHECK = -6,  /* a kernel reported an out-of-range index or a bounded wait ran out */
    H2_WARN_TOL_NOT_MET = 1    /* the rank cap or the probe cap limited a truncation */
};

/* ---- admissibility (Section 3.1, Table 1) -------------------------------- */
enum {
    H2_ADM_WEAK = 0,    /* every off-diagonal sibling block is low rank (HSS partition) */
    H2_ADM_STRONG = 1   /* (t,s) low rank iff max(diam t, diam s) <= eta * dist(t, s) */
};

/* ---- matvec arithmetic modes ---------------------------------------------- */
enum {
    H2_FP64 = 0,   /* X, Y double; FP64 storage and arithmetic */
    H2_FP32 = 1,   /* X, Y float; FP32 storage and arithmetic */
    H2_TF32 = 2,   /* X float, Y float; FP32 storage, TF32 tensor-core products, FP32 accumulation */
    H2_BF16 = 3,   /* X bf16 (uint16 storage), Y float; BF16 storage, tensor-core products, FP32 accumulation */
    H2_TF32X3 = 4, /* X float, Y float; FP32 storage, split-TF32 tensor-core products (hi*hi + hi*lo + lo*hi,
                      about 22 significant bits, FP32-grade) from nrhs >= 64, FP32 arithmetic below */
    H2_FP32C = 5   /* X, Y double; FP32 storage (the FP32 copy: keep_fp32), compensated FP32 arithmetic on
                      the FP32 pipe: every value a pair hi + lo of floats (about 48 significant bits), products
                      and sums by error-free transformations, so that the FP32 rounding of the stored factors
                      (2^-24 relative per entry) is the only reduced-precision step; SIMT gather kernels at
                      every nrhs.  Not available in h2_matvec_noalloc and the batch API. */
};

#define H2_MAX_LEVELS 32

/*
 * Hessian-vector product callback (the only place where the library leaves its
 * own code; Section 3.3: the Hessian is available only through products).
 * Computes Y = H X for nrhs columns; X is n x nrhs (device, leading dimension
 * ldx), Y is n x nrhs (device, ldy), both in original node order, FP64.  Work
 * must be enqueued on `stream` (asynchronous is fine).  X and Y are library
 * scratch: the callback must not keep them after returning.  Return 0 on
 * success; any other value aborts the build with H2_ERR_OP_FAILED.
 */
typedef int (*h2_op_fn)(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx,
                        double* Y, int64_t ldy, h2_stream_t stream);

/* ---- construction options ------------------------------------------------ */
typedef struct {
    int kmax;            /* cap on basis ranks (default 32) */
    int q0;              /* initial probes per level, or the fixed count if adaptive == 0 (default 32) */
    int b_inc;           /* probe increment of the adaptive range finder, 1..16 (default 16) */
    int q_max;           /* probe cap per level (default 256) */
    int adaptive;        /* 1: grow probes until the a-posteriori range test passes (default 1) */
    uint64_t seed;       /* seed of the counter-based probe generator (default 7) */
    double norm_est;     /* > 0: use this value of ||H||_2 instead of estimating it (default 0) */
    int norm_maxit;      /* power-iteration cap for ||H||_2 (default 50) */
    double norm_rtol;    /* power-iteration stop: relative change (default 1e-3) */
    int keep_fp32;       /* also keep an FP32 copy of the factors (enables H2_FP32/H2_TF32), default 0 */
    int keep_bf16;       /* also keep a BF16 copy of the factors (enables H2_BF16), default 0 */
    h2_stream_t stream;  /* stream for all build work and operator calls (default NULL) */
    /* Predicted start counts (learned ranks): optional host array with at least L+1 entries,
     * indexed by level; entry l > 0 replaces q0 at level l (identity range when it is at
     * least the largest child-1 box of the level), entries <= 0 keep q0.  The first range
     * test after such a start uses q_test columns; later growth uses b_inc.  The array is
     * read during the call only.  Typically filled by h2_rankmodel_q_levels.  Default NULL. */
    const int32_t* q_level;
    int q_level_stride;  /* h2_build_batched: Hessian i reads q_level + i * q_level_stride (0: all share) */
    int q_test;          /* columns of the first range test after a q_level start, 1..16 (default 8) */
    /* Hybrid construction (Section 3.3, end: a global low-rank approximation B B^T first, the
     * hierarchical construction on the residual H - B B^T, B B^T added back as a low-rank
     * update with recompression).  global_rank > 0 is the budget of the global piece: an
     * adaptive randomized range finder on the whole matrix (start q0, growth b_inc, the levels'
     * a-posteriori test) gives an orthonormal Q with at most global_rank columns, one more
     * product gives M = Q^T H Q, and B = Q C with C C^T = M (semidefinite Cholesky; H must be
     * symmetric positive semidefinite).  If the range test passes within the budget the
     * residual is not sampled at all (every level reports range_passed = 2).  0 (default):
     * plain construction.  Requires 0 <= global_rank < n and, when > 0, n <= 14,155,776 (the
     * two-level tall-skinny QR of the whole matrix); ignored for a single leaf. */
    int global_rank;
    /* Sampling structure (Section 3.3: which blocks one probe block samples at once).
     * H2_SAMPLING_WEAK (default): the sibling blocks of every level, the paper's own choice.
     * H2_SAMPLING_COLORED: the strong-admissibility far blocks of every level themselves; the
     * column boxes are coloured so that no row box sees two boxes of one colour among its
     * remaining blocks, and each colour (range pass) and each probe slot of the projection pass
     * takes q0 probe columns; the near blocks come from identity probes on coloured leaves.  A
     * comparison mode (it needs far more products): q0 <= 16 fixed probes (adaptive, q_level and
     * global_rank are not used; global_rank must be 0), q0 below every box size with far blocks. */
    int sampling;
    /* h2_build_batched only: host worker threads, each with its own stream (0: min(count, 8)); the
     * per-level launches of different Hessians overlap on the GPU across workers. */
    int batch_workers;
    /* Certified range bases (weak sampling structure; Section 3.3's adaptive range finder in the
     * textbook form of Halko, Martinsson and Tropp, Algorithm 4.2): 1 keeps the columns of the
     * range test that passes out of the level's bases, since that test certifies the basis it
     * was run against; the projection pass and the recompression then work with need columns
     * (h2_build_stats.range_need) instead of every range probe drawn.  0 (default): the bases
     * span every range probe, the passing test's columns included.  Only 0 or 1. */
    int certified;
} h2_build_opts;

enum { H2_SAMPLING_WEAK = 0, H2_SAMPLING_COLORED = 1 };

/* Fill *opts with the defaults above.  Returns H2_ERR_INVALID_ARG if opts is NULL. */
int h2_build_opts_default(h2_build_opts* opts);

/* ---- statistics (host struct) -------------------------------------------- */
typedef struct {
    int64_t n;                              /* matrix size */
    int levels;                             /* tree depth L (leaves at level L) */
    int leaf_max;                           /* largest leaf */
    int64_t samples;                        /* Hessian-vector products of the peeling (excl. norm estimate) */
    int64_t norm_products;                  /* products spent on the ||H||_2 estimate */
    /* Per-level arrays are indexed by level; index 0 (the root, never sampled by the levels)
     * describes the global piece of a hybrid construction: range_probes[0] = columns of Q,
     * proj_probes[0] = products of its projection, range_calls[0] / range_need[0] /
     * range_passed[0] as for the levels (all 0 without a global piece). */
    int range_probes[H2_MAX_LEVELS];        /* range-pass probes per level (index = level) */
    int proj_probes[H2_MAX_LEVELS];         /* projection-pass probes per level */
    int max_rank[H2_MAX_LEVELS];            /* largest basis rank per level */
    int64_t far_lower;                      /* stored (lower-triangle) far blocks */
    int64_t near_lower;                     /* stored (lower-triangle + diagonal) near blocks */
    int64_t entries_D, entries_S, entries_U, entries_E;  /* stored floating-point entries */
    double norm_est;                        /* ||H||_2 estimate used */
    double tau_basis;                       /* absolute truncation threshold of the bases */
    double tau_test;                        /* threshold of the range test */
    int tol_met;                            /* 0 if a cap limited a truncation */
    double t_total, t_norm, t_op, t_peel, t_assemble;   /* seconds (host wall clock, synchronised) */
    int64_t op_calls;                       /* operator calls of the peeling (excl. norm estimate) */
    int range_calls[H2_MAX_LEVELS];         /* operator calls of the range pass per level */
    int range_need[H2_MAX_LEVELS];          /* probes of the range basis that passed the test; range_probes
                                               when no test passed; largest child-1 box for identity levels */
    int range_passed[H2_MAX_LEVELS];        /* 1 a range test passed, 0 none passed (cap or fixed count),
                                               -1 identity range (no range pass), 2 not sampled: the
                                               global piece already met the threshold */
} h2_stats;

/* ---- cluster tree and partition (host only; no CUDA calls) --------------- */

/*
 * Build the KD cluster tree (Section 4.2, Section 4.4: binary space partition,
 * spatial ordering) and the block partition (Section 3.1) for n points of
 * dimension dim (1..3), coordinates coords_host[i*dim + d] (host, row-major).
 * Every box of a level is split while the largest box of that level exceeds
 * leaf_size (>= 2), so all leaves share one depth; the split coordinate is the
 * longer bounding-box side (ties to the first); points are ordered by
 * (coordinate, original index) and the first floor(|t|/2) go to child 0.
 * adm is H2_ADM_WEAK or H2_ADM_STRONG with parameter eta > 0.
 * Errors: H2_ERR_INVALID_ARG for n < 1, bad dim, leaf_size < 2, bad adm or eta,
 * NULL pointers, non-finite coordinates or depth above H2_MAX_LEVELS - 1.
 */
int h2_tree_create(const double* coords_host, int64_t n, int dim, int leaf_size, int adm,
                   double eta, h2_tree_t* out);
void h2_tree_free(h2_tree_t tree);

/* Tree depth L, number of points, number of far blocks (both triangles, all
 * levels) and near blocks (both triangles).  Any output pointer may be NULL. */
int h2_tree_info(h2_tree_t tree, int* levels, int64_t* n, int64_t* n_far, int64_t* n_near);

/* Tree-order permutation: perm_host[i] = original index of tree position i (n entries). */
int h2_tree_perm(h2_tree_t tree, int64_t* perm_host);

/* Box ranges of one level: starts_host/sizes_host get 2^level entries (tree order). */
int h2_tree_boxes(h2_tree_t tree, int level, int64_t* starts_host, int64_t* sizes_host);

/* Far blocks of one level (both triangles, sorted by (t, s)): pairs_host[2*i], pairs_host[2*i+1].
 * *count receives the number of blocks; pairs_host may be NULL to query the count. */
int h2_tree_far(h2_tree_t tree, int level, int64_t* count, int32_t* pairs_host);

/* Near (leaf-level dense) blocks, both triangles, sorted by (t, s). */
int h2_tree_near(h2_tree_t tree, int64_t* count, int32_t* pairs_host);

/* ---- construction --------------------------------------------------------- */

/*
 * Construct the H^2 approximation of the symmetric operator `op` on `tree` to
 * relative accuracy tol (> 0) by randomized peeling (Section 3.3, Figure 2):
 * ||H||_2 estimate by power iteration (Section 3.2); per level, Gaussian probes on
 * child-0 boxes, removal of the coarser pieces, orthonormal range of every
 * child-1 sample block with an adaptive a-posteriori test, projection pass;
 * identity probes for the dense diagonal leaf blocks; then recompression into
 * nested orthonormal bases, couplings and dense near blocks (Section 3.2).
 * The tree may be freed after this call.  opts may be NULL (defaults).
 * Synchronises the stream before returning.  Errors: INVALID_ARG, CUDA, OOM,
 * OP_FAILED, NAN, DEVICE_CHECK; H2_WARN_TOL_NOT_MET leaves a valid handle.
 */
int h2_build(h2_op_fn op, void* ctx, h2_tree_t tree, double tol, const h2_build_opts* opts,
             h2_handle_t* out);

/*
 * Create a handle from explicit H^2 factors given in host memory (checkpoint
 * load, and test input).  Layout, all column-major FP64 and in tree order:
 *   ranks_host: k of every box, levels 0..L in order, 2^l boxes per level;
 *   U_host: leaf bases, leaf 0..2^L-1 in order, |t| x k_t each;
 *   E_host: transfer matrices of every box c at levels 1..L (in order), k_c x k_parent(c);
 *   S_host: couplings of the lower far blocks (t > s), levels 1..L, each level in
 *           h2_tree_far order, k_t x k_s each;
 *   D_host: near blocks with t >= s in h2_tree_near order, |t| x |s| each.
 * The representation is A = D + U S U^T with the upper blocks the transposes of the
 * lower ones (symmetric).  Errors: INVALID_ARG (sizes inconsistent with the tree),
 * CUDA, OOM.
 */
int h2_import(h2_tree_t tree, const int32_t* ranks_host, const double* U_host, const double* E_host,
              const double* S_host, const double* D_host, int keep_fp32, int keep_bf16,
              h2_handle_t* out);

/* Sizes of the arrays of h2_import/h2_export for handle h (entries, not bytes). */
int h2_factor_sizes(h2_handle_t h, int64_t* n_ranks, int64_t* n_U, int64_t* n_E, int64_t* n_S,
                    int64_t* n_D);

/* Copy the FP64 factors of h to host arrays in the h2_import layout (checkpoint save).
 * Any pointer may be NULL to skip that array.  Synchronous. */
int h2_export(h2_handle_t h, int32_t* ranks_host, double* U_host, double* E_host, double* S_host,
              double* D_host);

/*
 * Construct count H^2 approximations (uneven sizes allowed) in one call: Hessian i uses
 * ops[i], ctxs[i] (ctxs may be NULL), trees[i], the common tol and opts.  The builds run on
 * a pool of up to 8 host workers with their own CUDA streams, so that the many small
 * launches of different Hessians overlap on the GPU; each Hessian's arithmetic is exactly
 * that of h2_build (its operator is called on the worker's stream, so callbacks must be
 * callable from several threads for different contexts).  opts->stream is ignored; all work
 * is complete when the call returns.  outs[i] receive the handles.  On error every handle
 * is freed, outs are NULL, and the first error is returned; otherwise the largest warning.
 */
int h2_build_batched(int count, const h2_op_fn* ops, void* const* ctxs, const h2_tree_t* trees, double tol,
                     const h2_build_opts* opts, h2_handle_t* outs);

/* ---- application ----------------------------------------------------------- */

/*
 * Y = A X for nrhs right-hand sides by the four stages of Section 3.2, Eq. (3.2):
 * leaf bases and transfer matrices up the tree, couplings per level, transfer
 * matrices and leaf bases down the tree, plus the dense near blocks.  X (n x nrhs,
 * leading dimension ldx >= n) and Y (n x nrhs, ldy >= n) are device buffers in
 * original node order; their element types follow `mode` (see H2_FP64..H2_BF16).
 * X and Y must not overlap.  Enqueued on `stream`; returns before completion.
 * The coefficient workspace belongs to the handle: FP64 calls with up to 32 right-hand
 * sides use the part reserved at the handle's creation; wider calls and the reduced-
 * precision modes grow it once (an allocation) and keep it.  A call repeated with the same
 * buffers, sizes and mode is captured in a CUDA graph on its second occurrence and
 * replayed afterwards.  Errors: INVALID_ARG (sizes, NULL pointers, a mode whose storage
 * copy was not kept), CUDA, OOM.
 */
int h2_matvec(h2_handle_t h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs,
              int mode, h2_stream_t stream);

/*
 * Y = A X as h2_matvec, with X and Y in host memory (X: n x nrhs, leading dimension ldx >= n;
 * Y: n x nrhs, ldy >= n; element types as h2_matvec for `mode`).  The library copies X into a
 * device staging buffer owned by the handle, applies h2_matvec to it on `stream` and copies Y
 * back; the call returns when Y is complete on the host (it synchronises the stream).  Page-
 * locked host buffers (cudaHostAlloc, cudaHostRegister) give asynchronous copies at full bus
 * speed; pageable buffers work too.  The staging buffers grow to the largest call and are
 * released with the handle.  Errors: INVALID_ARG, CUDA, OOM.
 */
int h2_matvec_host(h2_handle_t h, const void* X_host, int64_t ldx, void* Y_host, int64_t ldy, int64_t nrhs, int mode,
                   h2_stream_t stream);

/*
 * The product of h2_matvec, for callers that cannot allocate device memory: for
 * example code whose device memory is entirely managed by another allocator (a
 * framework's caching pool that has already reserved the free memory), or
 * latency-critical loops that must not pay the implicit device-wide
 * synchronisation of cudaMalloc/cudaFree.  This entry point calls no allocation
 * routine.  Its coefficient scratch is one fixed array of 32 MiB inside the
 * library's device image, which every GPU that loads the library holds until the
 * process exits; calls needing more (coefficient rows of the handle x nrhs x 8 bytes
 * in H2_FP64, x 4 bytes otherwise) fail with H2_ERR_INVALID_ARG and a message giving
 * the size.  The array's device address is looked up, with the device current, when
 * a handle is created on that device (h2_build, h2_import and every other call that
 * returns a handle do it), which also loads the part of the library's device image
 * that holds the array while allocating is still allowed; a call with a handle of a
 * device whose address was never looked up does the lookup itself, so it should come
 * before any stream capture.  All calls share the array and it keeps the contents of
 * the last call (no element needs to start at zero: every element a call reads it
 * has written before), so calls whose executions overlap on the GPU, on any handle
 * or stream, race on it: serialise them.
 * Arithmetic: always the non-tensor-core kernels.  H2_FP64 and H2_FP32 run the
 * kernels h2_matvec runs in those modes (at nrhs <= 4 they add with atomics, so the
 * last bits can differ from call to call); H2_BF16 (BF16 storage and inputs, FP32
 * arithmetic) equals h2_matvec up to FP32 summation order, which differs from
 * h2_matvec's tensor-core path at nrhs >= 64.  H2_TF32 and H2_TF32X3 need the
 * tensor-core path's operand workspace and are rejected with H2_ERR_INVALID_ARG.
 * Other arguments and errors as h2_matvec.  The paper has no counterpart of this
 * entry point.
 */
int h2_matvec_noalloc(h2_handle_t h, const void* X, int64_t ldx, void* Y, int64_t ldy, int64_t nrhs,
                      int mode, h2_stream_t stream);

/* Stage kinds of the matvec, for h2_profile_read. */
enum {
    H2_STAGE_LEAF_UP = 0,   /* xh_t = U_t^T X_t */
    H2_STAGE_UP = 1,        /* transfer upsweep, all levels */
    H2_STAGE_COUPLE = 2,    /* couplings, all levels */
    H2_STAGE_DOWN = 3,      /* transfer downsweep, all levels */
    H2_STAGE_LEAF_NEAR = 4, /* Y_t = U_t yh_t (+ sum_s D_ts X_s when the near field is gathered per leaf) */
    H2_STAGE_NEAR = 5,      /* near field scattered per stored block (small nrhs): Y += D X */
    H2_STAGE_COUNT = 6
};

/* Enable (1) or disable (0) per-stage timing of h2_matvec on handle h: CUDA events
 * are recorded on the caller's stream around every stage launch.  Diagnostics only. */
int h2_profile(h2_handle_t h, int enable);

/* Synchronise the device, then return and reset the accumulated per-kind stage times
 * (milliseconds, ms_out[H2_STAGE_COUNT]) and launch counts (launches_out[H2_STAGE_COUNT]).
 * Either pointer may be NULL. */
int h2_profile_read(h2_handle_t h, double* ms_out, int64_t* launches_out);

/* Process-wide timing of the batched FP64 GEMM kernel used by the construction and
 * by the shipped operators: when enabled (1), CUDA events are recorded around every
 * GEMM launch on its stream.  h2_gemm_profile_read synchronises the device, returns the
 * accumulated milliseconds, algorithmic flops (sum of 2 m n k), algorithmic bytes (sum of
 * 8 (m k + k n + m n), plus 8 m n for C read when beta != 0) and launches, and resets.
 * Any output pointer may be NULL. */
int h2_gemm_profile(int enable);
int h2_gemm_profile_read(double* ms_out, double* flops_out, int64_t* launches_out, double* bytes_out);

/* Timing of the recompression's stacked Householder QR (which = 0) and truncated-SVD (which = 1)
 * launches, switched on and off with h2_gemm_profile: device milliseconds, algorithmic flops of
 * their QR factorisations (2 m n^2 - 2 n^3 / 3 per m x n stack with m >= n; the SVD adds 4 c^3 / 3
 * for the pivoted QR of its c x c triangle and does not count its Jacobi rotations) and launches
 * since the last read; reading resets them.  Any pointer may be NULL. */
int h2_stack_profile_read(int which, double* ms, double* flops, int64_t* launches);

/* Synchronise the device and report whether a kernel of handle h recorded a failed bounded
 * wait (H2_ERR_DEVICE_CHECK) since h was created; H2_OK otherwise. */
int h2_device_status(h2_handle_t h);

/*
 * Batched application (the batching pattern): the matvec stages of count handles are merged
 * into one launch per stage and tree level, the per-handle pointers are read from a device
 * table, and for every (nrhs, mode) the launch sequence is autotuned (right-hand-side tile 8,
 * 16 or 32, timed once on the first call) and captured in a CUDA graph that later calls replay.
 * The handles must stay alive while the batch exists.  h2_batch_matvec computes
 * Y[i] = A_i X[i] for every handle (device buffers, leading dimensions ldx[i], ldy[i], element
 * types as h2_matvec for `mode`; H2_TF32 runs in FP32 here).  Errors: INVALID_ARG, CUDA, OOM.
 */
int h2_batch_create(int count, const h2_handle_t* hs, h2_batch_t* out);
int h2_batch_matvec(h2_batch_t b, const void* const* X, const int64_t* ldx, void* const* Y, const int64_t* ldy,
                    int64_t nrhs, int mode, h2_stream_t stream);
/* Right-hand-side tile the autotuner chose for (nrhs, mode), 0 if that key was not run yet. */
int h2_batch_tuned(h2_batch_t b, int64_t nrhs, int mode, int* rhs_tile);
void h2_batch_free(h2_batch_t b);

/* One-shot batched application: h2_batch_create, h2_batch_matvec and h2_batch_free in one
 * call (the autotuning and capture run on this call and are not kept; callers that apply the
 * same handles repeatedly should keep an h2_batch_t).  Returns after the products are complete
 * (the device is synchronised).  Arguments and errors as h2_batch_create / h2_batch_matvec. */
int h2_matvec_batched(int count, const h2_handle_t* hs, const void* const* X, const int64_t* ldx, void* const* Y,
                      const int64_t* ldy, int64_t nrhs, int mode, h2_stream_t stream);

/* Statistics of the construction of h (host struct). */
int h2_get_stats(h2_handle_t h, h2_stats* out);

/* Release a handle and its device memory.  NULL is a no-op. */
void h2_free(h2_handle_t h);

/* ---- iterative inversion --------------------------------------------------------- */

/*
 * Approximate inverse of A = H + shift I (H an H^2 handle, symmetric positive definite with the
 * shift) by the hierarchical hyperpower iteration of Appendix A: X_{k+1} = X_k sum_{i<l} R_k^i,
 * R_k = I - A X_k (order l = 2: Newton-Schulz, Algorithm 1), every iterate constructed by peeling
 * (h2_build's method, Section 3.3) from a sampler that applies the iteration to probe blocks with
 * H^2 matvecs of A and X_k (Algorithms 2 and 4).  X_0 = I / ||A||_2 (power iteration).  Iterate k
 * is constructed to the relative threshold eps_k = max(eps / (||A|| ||X_k||), min(eps_loose,
 * theta E^2)) with E = ||A X_k - I||_2 (power iteration on (X A - I)(A X - I), stopped at
 * res_rtol relative change); eps_loose = eps gives the static threshold.  The iteration stops at
 * E <= eps, after max_iter iterates, or when an iterate stalls (E_{k+1} > 0.9 E_k while the exact
 * iteration would reach E_k^l < 0.5 E_{k+1}).  Not a construct of this library's paper beyond
 * Appendix A; the readings above are the library's.  With x0 the iteration starts from a given
 * iterate; with unroll it constructs one unrolled iterate (see the fields below).
 */
#define H2_MAX_INVERT_ITERS 64
typedef struct {
    int order;           /* hyperpower order l >= 2 (default 2: Newton-Schulz) */
    double eps;          /* target ||A X - I||_2 (default 1e-6) */
    double eps_loose;    /* loosest construction threshold (default 1e-6, i.e. static) */
    double theta;        /* factor of E^2 in the dynamic threshold (default 0.1) */
    int max_iter;        /* iterate cap, 0..H2_MAX_INVERT_ITERS (default 50) */
    double shift;        /* A = H + shift I (default 0) */
    int res_maxit;       /* power-iteration cap of the norm and residual estimates (default 50) */
    double res_rtol;     /* their stop: relative change (default 1e-2) */
    uint64_t seed;       /* seed of the power-iteration start vectors (default 9) */
    /* Warm start (Appendix A: a previous approximate inverse as the initial iterate): X_0 = x0
     * (an H^2 handle on A's tree, e.g. an earlier h2_invert result; it is only read and stays the
     * caller's) instead of alpha I.  Default NULL. */
    h2_handle_t x0;
    /* Unrolled iterations (Appendix A, "Unrolling iterations"): unroll = k >= 1 constructs the k-th
     * Newton-Schulz iterate of X_0 in one construction, X_k = X_0 sum_{i < 2^k} (I - A X_0)^i (the
     * product prod_{j<k} (I + R_0^{2^j}) of k Newton-Schulz steps written as one geometric sum;
     * Appendix A prints this identity garbled), evaluated on the probe blocks by Horner's rule with
     * 2^k - 1 products of A and X_0 per probe, and constructed to the final threshold
     * eps / (||A|| ||X_0||); the order, iterate count and threshold settings are then ignored.
     * k <= 6.  Default 0: ordinary iterations. */
    int unroll;
} h2_invert_opts;

typedef struct {
    int iterations;                              /* iterates constructed */
    int converged;                               /* 1 if the final E <= eps */
    double norm_A, alpha;                        /* ||A||_2 estimate; X_0 = alpha I */
    double err[H2_MAX_INVERT_ITERS + 1];         /* E before iterate k (k < iterations), then the final E */
    double eps_k[H2_MAX_INVERT_ITERS];           /* construction threshold of iterate k */
    int64_t samples[H2_MAX_INVERT_ITERS];        /* peeling products of iterate k */
    double t_build[H2_MAX_INVERT_ITERS];         /* seconds of iterate k's construction */
    double final_err, t_total;
} h2_invert_stats;

/* Fill *opts with the defaults above.  Returns H2_ERR_INVALID_ARG if opts is NULL. */
int h2_invert_opts_default(h2_invert_opts* opts);

/* X_out receives the last iterate (a new handle on A's tree; free with h2_free); build_opts (may
 * be NULL) configure every construction (their stream carries all work).  stats may be NULL.
 * Errors: INVALID_ARG, CUDA, OOM, NAN, OP_FAILED; the result of a run that stopped unconverged
 * is still returned with H2_WARN_TOL_NOT_MET. */
int h2_invert(h2_handle_t A, const h2_invert_opts* opts, const h2_build_opts* build_opts, h2_handle_t* X_out,
              h2_invert_stats* stats);

/* ---- coloured sampling plan ------------------------------------------------------ */

/* The probe counts of H2_SAMPLING_COLORED for a tree, without any product (Section 3.3: C_l, the
 * number of probe blocks that sample all blocks of level l without interference).  counts (host,
 * 3 (L + 1) + 1 ints): for level l, counts[3 l] = colours of the range pass, counts[3 l + 1] =
 * probe slots of the projection pass, counts[3 l + 2] = lower far pairs sampled; counts[3 (L + 1)] =
 * leaf colours of the near-block pass.  Level l then takes q (counts[3 l] + counts[3 l + 1])
 * products and the leaf pass leaf_max counts[3 (L + 1)].  Errors: INVALID_ARG (NULL, q outside
 * 1..16, q not below a box with far blocks). */
int h2_colored_plan(h2_tree_t tree, int q, int* counts);

/* ---- low-rank update with recompression --------------------------------------- */

/*
 * A~ = A + B M B^T as a new H^2 matrix on A's tree (Section 3.2, Eqs. 3.3-3.4: a global low-rank
 * update raises every block's rank by r; recompression then finds new nested bases by a QR
 * downsweep of the block rows and a truncated-SVD upsweep, and projects the couplings on them).
 * With M = I this is the paper's X Y^T for X = Y = B (the symmetric form that a Hessian keeps);
 * M = -I removes B B^T.  Nothing is sampled: the update works on A's factors alone.
 *   A      built or imported handle (only read; stays the caller's).
 *   B      device, n x r, original node order, column-major with leading dimension ldb >= n;
 *          may be NULL when r == 0 (then the call recompresses A alone).  Only read.
 *   r      update rank, 0 <= r and r + (largest rank of A) <= 144.
 *   M      host, r x r column-major; its symmetric part (M + M^T)/2 is used.  NULL: identity.
 *   tol    relative target: the new bases are truncated at 2 tol ||A~||_2 / sqrt(#leaves), the
 *          construction's basis threshold.
 *   opts   may be NULL.  Used fields: kmax (<= 48; rank cap of the new bases), norm_est (> 0:
 *          ||A~||_2 to use; else power iteration on products with A~ with seed, norm_maxit,
 *          norm_rtol as in h2_build), keep_fp32, keep_bf16, stream (carries all work).
 *   out    receives the new handle (free with h2_free); its stats give norm_est, tau_basis,
 *          max_rank, t_total.
 * Errors: INVALID_ARG (sizes, ranks above the limits), CUDA, OOM, NAN; H2_WARN_TOL_NOT_MET
 * (still a valid handle) when kmax cut a truncation.
 */
int h2_lowrank_update(h2_handle_t A, const double* B, int64_t ldb, int r, const double* M, double tol,
                      const h2_build_opts* opts, h2_handle_t* out);

/* ---- learned rank model ------------------------------------------------------ */

/*
 * A 3-layer perceptron that predicts, per tree level, the probe count the adaptive range
 * finder settles on, so that peeling can start there (Section 3.3: the per-level sample
 * count C_l k is the quantity being tuned; adaptive growth stays the fallback and decides
 * the error).  Not a construct of the paper: a learned replacement for its hand-tuned
 * sampling parameters.
 *   x (H2_RM_FEATURES) -> gelu(W1 x + b1) -> gelu(W2 h1 + b2) -> y = W3 h2 + b3, width 64,
 *   gelu(u) = u/2 (1 + tanh(sqrt(2/pi) (u + 0.044715 u^3))); target y = log2(1 + need).
 * Parameters (H2_RM_NPARAM floats, this order): W1 (64 x 8 row-major), b1 (64), W2 (64 x 64
 * row-major, W2[o][i]), b2 (64), W3 (64), b3 (1).  Master weights, Adam moments and all
 * arithmetic are FP32; with bf16 != 0 the forward and backward passes use the master
 * weights rounded to bfloat16 (nearest even).  Training: mean squared error, Adam
 * (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).  A model lives on the device that was
 * current at creation; it is not thread-safe.
 */
#define H2_RM_FEATURES 8
#define H2_RM_WIDTH 64
#define H2_RM_NPARAM (64 * 8 + 64 + 64 * 64 + 64 + 64 + 1)
typedef struct h2_rankmodel_s* h2_rankmodel_t;

/* Create a model with weights drawn U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from the counter-based
 * generator seeded with seed, zero biases, zero Adam state.  Errors: INVALID_ARG, CUDA, OOM. */
int h2_rankmodel_create(uint64_t seed, int bf16, h2_rankmodel_t* out);
void h2_rankmodel_free(h2_rankmodel_t m);

/* Host copies of the master parameters, Adam moments (H2_RM_NPARAM floats each) and the Adam
 * step count.  Any pointer may be NULL (get: skipped; set: that part is left unchanged, except
 * step < 0 which keeps the count).  Synchronous. */
int h2_rankmodel_get(h2_rankmodel_t m, float* params_host, float* adam_m_host, float* adam_v_host,
                     int64_t* step);
int h2_rankmodel_set(h2_rankmodel_t m, const float* params_host, const float* adam_m_host,
                     const float* adam_v_host, int64_t step);

/* Features of every level l = 0..L of tree (row l of out_host, (L+1) x H2_RM_FEATURES, row-major,
 * host): l/L, log2(mean box size)/20, mean box diameter / root diameter, log10(kappa_T)/4,
 * density, log10(tol)/10, log10(sqrt(kappa_T) / mean box diameter)/2, log2(n)/20, where
 * kappa_T is the diffusivity times the final time of the heat Hessian and density the
 * sensor fraction m/n.  Errors: INVALID_ARG (NULL, kappa_T <= 0, tol <= 0). */
int h2_rankmodel_features(h2_tree_t tree, double kappa_T, double density, double tol, double* out_host);

/* Mean squared error and its gradient with respect to the (effective) parameters over the n
 * rows of X (device, n x H2_RM_FEATURES row-major, FP32) and targets t (device, n).  Outputs
 * on the host (grad_host: H2_RM_NPARAM floats, may be NULL).  No update.  Synchronous. */
int h2_rankmodel_loss_grad(h2_rankmodel_t m, const float* X, const float* t, int64_t n, float* loss_host,
                           float* grad_host);

/* steps Adam steps on minibatches of `batch` rows (1..1024) of (X, t) (device, as above), all
 * in one launch on one CTA.  idx (device, steps x batch int32 in [0, n)) lists the rows of
 * every minibatch; NULL draws them from the model's counter-based generator.  loss_out
 * (device, steps floats, may be NULL) receives each minibatch's loss before its update.
 * Asynchronous on stream.  Errors: INVALID_ARG, CUDA. */
int h2_rankmodel_train(h2_rankmodel_t m, const float* X, const float* t, int64_t n, const int32_t* idx,
                       int steps, int batch, float lr, float* loss_out, h2_stream_t stream);

/* y (device, n floats) = model(X) (device, n x H2_RM_FEATURES).  Asynchronous on stream. */
int h2_rankmodel_predict(h2_rankmodel_t m, const float* X, int64_t n, float* y, h2_stream_t stream);

/* Save a model (bf16 flag, seed, Adam step, parameters and both Adam moments) to a binary file
 * (host path; native byte order, magic "H2RM0001"), and create a model on the current device from
 * such a file.  Synchronous.  Errors: INVALID_ARG (NULL arguments, file not writable/readable,
 * wrong magic or size), CUDA, OOM. */
int h2_rankmodel_save(h2_rankmodel_t m, const char* path);
int h2_rankmodel_load(const char* path, h2_rankmodel_t* out);

/* Start counts for h2_build_opts.q_level: q_host[l] (host, L+1 entries) = ceil(2^y_l) - 1 + pad
 * rounded up to a multiple of 8 and clamped to [8, q_max], y_l the prediction for level l of
 * h2_rankmodel_features(tree, kappa_T, density, tol); q_host[0] = 0.  y_host (L+1 floats,
 * may be NULL) receives the raw predictions.  Synchronous. */
int h2_rankmodel_q_levels(h2_rankmodel_t m, h2_tree_t tree, double kappa_T, double density, double tol,
                          int pad, int q_max, int32_t* q_host, float* y_host);

/* Training targets of the model from a finished construction h: for every sampled level l
 * (levels with an identity range are skipped), levels_host[i] = l and targets_host[i] =
 * log2(1 + need_l), need_l the probe count whose range basis passed the adaptive test
 * (h2_stats.range_need).  *count receives the number of entries (at most L); either array may
 * be NULL to query the count.  Host arrays.  Errors: INVALID_ARG. */
int h2_rankmodel_targets(h2_handle_t h, int32_t* levels_host, float* targets_host, int* count);

/* ---- synthetic Hessians shipped with the library ------------------------- */

/*
 * Misfit Hessian of 2-D heat-equation initial-condition inversion on the unit
 * square: H = F diag(mask) F / sigma^2, F = exp(T kappa Lap_h) with the 5-point
 * Dirichlet Laplacian on the n x n interior grid (node p = i*n + j at ((i+1)h,
 * (j+1)h), h = 1/(n+1)), applied through the orthonormal DST-I: F = F1 (x) F1 with
 * F1 = S diag(exp(-T kappa mu)) S, restricted to the sine modes whose factor is at least
 * 2^-60 times the largest (the rest is below FP64 resolution).  mask_host holds n*n
 * entries (1 at sensor nodes, 0 elsewhere).  Creates device state on the current device.
 * Errors: INVALID_ARG, CUDA, OOM.
 */
int h2_heat2d_create(int n, double kappa, double T, double sigma, const double* mask_host,
                     void** ctx_out);
/* h2_op_fn implementation for a context from h2_heat2d_create. */
int h2_heat2d_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y,
                    int64_t ldy, h2_stream_t stream);
void h2_heat2d_destroy(void* ctx);

/* Dense symmetric operator Y = A X with A an n x n device matrix (leading dimension
 * lda) that the caller keeps alive while the context is used. */
int h2_dense_op_create(const double* A_device, int64_t n, int64_t lda, void** ctx_out);
int h2_dense_op_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y,
                      int64_t ldy, h2_stream_t stream);
void h2_dense_op_destroy(void* ctx);

/* Factored symmetric positive semidefinite operator Y = scale Z (Z^T X), Z an n x r device
 * matrix (leading dimension ldz) that the caller keeps alive while the context is used; the
 * misfit Hessian of a linear inverse problem with r point observations has this form with
 * Z = A^-T O^T (one adjoint solve per observation) and scale = 1 / sigma^2 (Section 4.3's source
 * inversion).  Workspace r x nrhs is owned by the context.  Errors: INVALID_ARG, CUDA, OOM. */
int h2_lowrank_op_create(const double* Z_device, int64_t n, int64_t r, int64_t ldz, double scale, void** ctx_out);
int h2_lowrank_op_apply(void* ctx, int64_t n, int64_t nrhs, const double* X, int64_t ldx, double* Y,
                        int64_t ldy, h2_stream_t stream);
void h2_lowrank_op_destroy(void* ctx);

/* ---- diagnostics ------------------------------------------------------------ */

const char* h2_error_string(int status);
/* Detailed message of the calling thread's last failing call ("" if none). */
const char* h2_last_error(void);
/* Number of kernels the library has launched in this process. */
int64_t h2_launch_count(void);
/* Device bytes the library currently holds (all handles, trees, workspaces and cached blocks of
 * running constructions).  No CUDA call. */
int64_t h2_device_bytes(void);
/* Cap on the library's device bytes (<= 0 removes it): an allocation that would go above it
 * fails with H2_ERR_OOM as if the device were full, for testing allocation-failure paths.
 * Affects all threads; returns H2_OK. */
int h2_set_device_limit(int64_t bytes);
/* Library version string. */
const char* h2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* H2_H */
