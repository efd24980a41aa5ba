// Construction of the H^2 approximation from Hessian-vector products.
//
// Peeling (Section 3.3, Figure 2, weak-admissibility sampling structure):
//   for l = 1..L, all sibling pairs (a, b) of level l at once:
//     range pass   Omega: Gaussian on child-0 rows;  Y = H Omega - K Omega  (K: coarser pieces)
//                  Q_b: orthonormal range of Y[b], grown by b_inc probes until the new
//                  probes' residuals (I - Q Q^T) y are below tau / (10 sqrt(2/pi))
//     projection   Psi = [Q_b on child-1 rows];  Z = H Psi - K Psi;  piece H[b,a] ~ Q_b Z[a]^T
//   leaf pass      identity probes on every leaf -> dense diagonal blocks.
// Recompression into nested bases (Section 3.2): for every box t, the far block
// row (far blocks of t and of its ancestors restricted to t) is, grouped by the
// pair level lp of the sampled piece containing each block, sum_lp P_lp[t] C_lp^T.
// A QR downsweep gives the R factors R_lp(t) of the column sides C_lp(t), so that
// the block row has the left singular vectors and values of the compact factor
// W_t = [P_lp[t] R_lp(t)^T]_lp; its truncated SVD (QR of W_t^T, one-sided Jacobi)
// gives the leaf bases and, in the coordinates of the children's bases, the
// transfer matrices of every upper level (upsweep), keeping the directions above
// the truncation threshold.  No Gram matrix is formed, so the singular values are
// resolved to about eps * sigma_max.  Couplings S_ts are products of
// the projected pieces, near blocks products of the pieces.
//
// The host only orchestrates: every arithmetic step runs in the library's kernels.
#include <algorithm>
#include <chrono>
#include <tuple>
#include <cmath>
#include <cstring>
#include <map>

#include "handle.h"

namespace h2 {

namespace {

constexpr int STREAM_PROBE = 1;
constexpr int STREAM_POWER = 2;
constexpr int STREAM_GLOBAL = 5;   // probes of the global low-rank range finder
constexpr int64_t kGlobalMaxRows = (int64_t)96 * 96 * 1536;   // one two-level TSQR panel of the whole matrix
constexpr int PANEL = 16;

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

class Builder {
  public:
    Builder(const h2_tree_s& T, h2_op_fn op, void* ctx, double tol, const h2_build_opts& o)
        : T_(T), op_(op), ctx_(ctx), tol_(tol), o_(o), s_((cudaStream_t)o.stream) {
        N_ = T.N;
        L_ = T.L;
    }

    void run(h2_handle_s* h);

  private:
    const h2_tree_s& T_;
    h2_op_fn op_;
    void* ctx_;
    double tol_;
    h2_build_opts o_;
    cudaStream_t s_;
    int64_t N_;
    int L_;

    DevBuf<int32_t> d_perm_, d_row_leaf_;
    DevBuf<double> Om_, Yo_, Yt_, Ot_, Tw_, Cw_, Ysv_, Tp_;
    DevBuf<SignItem> d_sign_;
    DevBuf<double> Pcap_;
    std::vector<int64_t> pcol_;      // capacity column offset per level
    std::vector<int> qcap_, qw_;     // capacity and final piece width per level
    std::vector<std::vector<int>> kb_;  // per level, per pair: columns of Q_b
    DevBuf<double> Ddiag_;
    std::vector<int64_t> ddiag_off_;
    GemmBatch gb_;
    TsqrWork tsqr_;
    StackWork stk_;
    Stager stg_[4];
    DevBuf<int64_t> d_i64a_, d_i64b_;
    DevBuf<int> d_i32a_, d_i32b_, d_i32c_, d_flag_;
    DevBuf<double> d_red_;
    DevBuf<BlkDesc> d_blk_;
    Pinned pin_;
    int cmax_ = 0;
    int64_t samples_ = 0, norm_products_ = 0, op_calls_ = 0;
    double t_op_ = 0.0;
    double norm_ = 0.0, tau_basis_ = 0.0, tau_test_ = 0.0;
    bool cap_hit_ = false;
    std::vector<int> range_probes_, proj_probes_, range_calls_, range_need_, range_passed_;
    int kb0_ = 0;            // columns of the global range basis Q (level-0 slot of Pcap_)
    bool covered_ = false;   // the global piece met the threshold: the residual is not sampled

    void call_op(const double* X, double* Y, int ncols, bool count_sample);
    void check_flag(const char* where, int level);
    double norm_estimate();
    void subtract(const double* Omt, double* Yt, int c, int lmax, int lsel = -1, int in_par = 0);
    void project(int l, const std::vector<int>& pairs, int c, int c0, int passes);
    std::vector<double> colnorm(int l, const std::vector<int>& pairs, int c, int c0);
    void panel(int l, const std::vector<int>& pairs, int c0, int w);
    void identity(int l, const std::vector<int>& pairs);
    void blocks(int kind, const std::vector<BlkDesc>& d, const double* src, double* dst);
    void peel_level(int l);
    void copy_tall(const double* src, double* dst, int cols);
    void gproject(int c0, int c, int passes);
    void gpanel(int c0, int w);
    void global_pass();
    void leaf_pass();
    void add_global_diag(double beta);
    void assemble(h2_handle_s* h);
    template <class T>
    T* dev_list(DevBuf<T>& buf, const std::vector<T>& v, int which) {
        upload(buf, v, s_, stg_[which & 3]);
        return buf.p;
    }
    double* Pl(int l) { return Pcap_.p + pcol_[l] * N_; }
    // start count of the range pass at level l (predicted, else q0)
    bool predicted(int l) const { return o_.q_level && o_.q_level[l] > 0; }
    int q_start(int l) const { return predicted(l) ? o_.q_level[l] : o_.q0; }
    int64_t bstart(int l, int b) const { return T_.start[l][b]; }
    int bsize(int l, int b) const { return (int)T_.size[l][b]; }
};

void Builder::call_op(const double* X, double* Y, int ncols, bool count_sample) {
    if (ncols <= 0) return;
    const double t0 = now_s();
    const int r = op_(ctx_, N_, ncols, X, N_, Y, N_, (h2_stream_t)s_);
    if (r != 0) fail(H2_ERR_OP_FAILED, "Hessian operator returned " + std::to_string(r));
    t_op_ += now_s() - t0;
    scan_finite(N_, ncols, Y, N_, d_flag_.p, s_);
    if (count_sample) {
        samples_ += ncols;
        ++op_calls_;
    } else {
        norm_products_ += ncols;
    }
}

void Builder::check_flag(const char* where, int level) {
    int* f = pin_.get<int>(1);
    H2_CUDA(cudaMemcpyAsync(f, d_flag_.p, sizeof(int), cudaMemcpyDeviceToHost, s_));
    H2_CUDA(cudaStreamSynchronize(s_));
    if (*f)
        fail(H2_ERR_NAN, std::string("non-finite values in Hessian-vector products (") + where + ", level " +
                             std::to_string(level) + ")");
}

// ||H||_2 by power iteration (Section 3.2) from a Gaussian start vector.
double Builder::norm_estimate() {
    double* v = Om_.p;
    double* w = Yo_.p;
    gaussian_vector(N_, d_perm_.p, o_.seed, STREAM_POWER, v, s_);
    auto sqnorm = [&](const double* x) {
        col_sqnorms(N_, 1, x, N_, d_red_.p, s_);
        double* hp = pin_.get<double>(1);
        H2_CUDA(cudaMemcpyAsync(hp, d_red_.p, sizeof(double), cudaMemcpyDeviceToHost, s_));
        H2_CUDA(cudaStreamSynchronize(s_));
        return *hp;
    };
    auto scale = [&](double* x, double f) {
        double* hp = pin_.get<double>(1);
        *hp = f;
        H2_CUDA(cudaMemcpyAsync(d_red_.p + 1, hp, sizeof(double), cudaMemcpyHostToDevice, s_));
        scale_cols(N_, 1, x, N_, d_red_.p + 1, s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    };
    const double g = std::sqrt(sqnorm(v));
    if (!(g > 0.0)) fail(H2_ERR_CUDA, "power iteration: zero start vector");
    scale(v, 1.0 / g);
    double lam = 0.0, prev = 0.0;
    for (int it = 1; it <= o_.norm_maxit; ++it) {
        call_op(v, w, 1, false);
        check_flag("norm estimate", 0);
        lam = std::sqrt(sqnorm(w));
        if (lam == 0.0) break;
        scale(w, 1.0 / lam);
        std::swap(v, w);
        if (it > 1 && std::fabs(lam - prev) <= o_.norm_rtol * lam) break;
        prev = lam;
    }
    return lam;
}

void Builder::blocks(int kind, const std::vector<BlkDesc>& d, const double* src, double* dst) {
    if (d.empty()) return;
    if (kind == BLK_COPY) {
        const std::vector<BlkDesc> ds = split_copies(d);
        block_op(kind, (int)ds.size(), dev_list(d_blk_, ds, 0), src, dst, s_);
        return;
    }
    block_op(kind, (int)d.size(), dev_list(d_blk_, d, 0), src, dst, s_);
}

// Y -= K Omega for the pieces of levels 1..lmax (tree order, N x c, ld N).  With lsel > 0 the
// probe block is nonzero only on the rows of the level-lsel boxes whose child index is in_par, and
// only the rows of the other children are needed (the range pass reads child-1 rows of probes on
// child-0 rows; the projection pass the reverse): both products then run over those boxes only,
// the first as per-box partial products summed per level-lp box, so that each does half the work.
void Builder::subtract(const double* Omt, double* Yt, int c, int lmax, int lsel, int in_par) {
    if (qw_[0] > 0 && lmax >= 0) {
        // the global piece: Y -= B (B^T Om)
        const int q = qw_[0];
        gb_.add(Pl(0), (int)N_, 1, Omt, (int)N_, 0, Tw_.p, q, q, c, (int)N_, 1.0, 0.0);
        gb_.run(s_);
        gb_.add(Pl(0), (int)N_, 0, Tw_.p, q, 0, Yt, (int)N_, (int)N_, c, q, -1.0, 1.0);
        gb_.run(s_);
    }
    for (int lp = 1; lp <= lmax; ++lp) {
        const int q = qw_[lp];
        if (q == 0) continue;
        const double* P = Pl(lp);
        const int nb = 1 << lp;
        if (lsel > lp) {
            const int sh = lsel - lp;
            const int64_t blk = (int64_t)q * c;   // one q x c block (leading dimension q)
            Tp_.reserve((size_t)((int64_t)1 << (lsel - 1)) * blk);
            Tw_.reserve((size_t)nb * blk);
            for (int cb = in_par; cb < (1 << lsel); cb += 2)
                gb_.add(P + bstart(lsel, cb), (int)N_, 1, Omt + bstart(lsel, cb), (int)N_, 0, Tp_.p + (cb >> 1) * blk, q,
                        q, c, bsize(lsel, cb), 1.0, 0.0);
            gb_.run(s_);
            std::vector<int64_t> oo(nb), io;
            std::vector<int> len(nb, (int)blk), bg(nb), en(nb);
            for (int b = 0; b < nb; ++b) {
                oo[b] = b * blk;
                bg[b] = (int)io.size();
                for (int cb = (b << sh) + in_par; cb < ((b + 1) << sh); cb += 2) io.push_back((cb >> 1) * blk);
                en[b] = (int)io.size();
            }
            sum_lists(nb, dev_list(d_i64a_, oo, 0), dev_list(d_i32a_, len, 1), dev_list(d_i32b_, bg, 2),
                      dev_list(d_i32c_, en, 3), dev_list(d_i64b_, io, 0), Tp_.p, Tw_.p, 0, s_);
            for (int d = 1 - in_par; d < (1 << lsel); d += 2)
                gb_.add(P + bstart(lsel, d), (int)N_, 0, Tw_.p + ((d >> sh) ^ 1) * blk, q, 0, Yt + bstart(lsel, d),
                        (int)N_, bsize(lsel, d), c, q, -1.0, 1.0);
            gb_.run(s_);
            continue;
        }
        const int ldt = nb * q;
        for (int b = 0; b < nb; ++b)
            gb_.add(P + bstart(lp, b), (int)N_, 1, Omt + bstart(lp, b), (int)N_, 0, Tw_.p + (int64_t)b * q, ldt, q,
                    c, bsize(lp, b), 1.0, 0.0);
        gb_.run(s_);
        for (int i = 0; i < nb / 2; ++i) {
            const int a = 2 * i, b = 2 * i + 1;
            gb_.add(P + bstart(lp, b), (int)N_, 0, Tw_.p + (int64_t)a * q, ldt, 0, Yt + bstart(lp, b), (int)N_,
                    bsize(lp, b), c, q, -1.0, 1.0);
            gb_.add(P + bstart(lp, a), (int)N_, 0, Tw_.p + (int64_t)b * q, ldt, 0, Yt + bstart(lp, a), (int)N_,
                    bsize(lp, a), c, q, -1.0, 1.0);
        }
        gb_.run(s_);
    }
}

// Block Gram-Schmidt projection of columns [c0, c0+c) of Yt[b] against Q_b = P_l[b, 0:kb].
void Builder::project(int l, const std::vector<int>& pairs, int c, int c0, int passes) {
    double* P = Pl(l);
    const int ldc = std::max(qcap_[l], 1);
    for (int pass = 0; pass < passes; ++pass) {
        int n = 0;
        for (int i : pairs) {
            const int kb = kb_[l][i];
            if (!kb) { ++n; continue; }
            const int64_t st = bstart(l, 2 * i + 1);
            gb_.add(P + st, (int)N_, 1, Yt_.p + st + (int64_t)c0 * N_, (int)N_, 0, Cw_.p + (int64_t)n * ldc * c, ldc,
                    kb, c, bsize(l, 2 * i + 1), 1.0, 0.0);
            ++n;
        }
        gb_.run(s_);
        n = 0;
        for (int i : pairs) {
            const int kb = kb_[l][i];
            if (!kb) { ++n; continue; }
            const int64_t st = bstart(l, 2 * i + 1);
            gb_.add(P + st, (int)N_, 0, Cw_.p + (int64_t)n * ldc * c, ldc, 0, Yt_.p + st + (int64_t)c0 * N_, (int)N_,
                    bsize(l, 2 * i + 1), c, kb, -1.0, 1.0);
            ++n;
        }
        gb_.run(s_);
    }
}

std::vector<double> Builder::colnorm(int l, const std::vector<int>& pairs, int c, int c0) {
    std::vector<int64_t> off;
    std::vector<int> m;
    for (int i : pairs) {
        off.push_back(bstart(l, 2 * i + 1) + (int64_t)c0 * N_);
        m.push_back(bsize(l, 2 * i + 1));
    }
    std::vector<double> out(pairs.size(), 0.0);
    if (pairs.empty()) return out;
    panel_colnorm_max((int)pairs.size(), dev_list(d_i64a_, off, 1), dev_list(d_i32a_, m, 2), c, Yt_.p, (int)N_,
                      d_red_.p, s_);
    double* hp = pin_.get<double>(pairs.size());
    H2_CUDA(cudaMemcpyAsync(hp, d_red_.p, pairs.size() * sizeof(double), cudaMemcpyDeviceToHost, s_));
    H2_CUDA(cudaStreamSynchronize(s_));
    std::memcpy(out.data(), hp, pairs.size() * sizeof(double));
    return out;
}

// Appends the panel columns [c0, c0+w) of Yt[b] to Q_b = P_l[b, 0:kb] by block classical
// Gram-Schmidt with reorthogonalisation (BCGS2; Barlow and Smoktunowicz 2013): project and
// Householder-QR the panel, then project the orthonormal result once more and QR it again.
// The second round keeps the new columns orthogonal to Q_b also when the panel is
// numerically rank deficient (samples of a block whose range is already captured).  Finally
// every new column q_j is turned so that q_j^T y_j >= 0 for its sample column y_j: the basis
// is then the Q factor of the samples' thin QR with a non-negative diagonal of R, fixed by
// the samples and not by the orthogonalisation method (the projection pass applies all
// blocks' bases at once, so the basis itself, not only its span, reaches the pieces).
void Builder::panel(int l, const std::vector<int>& pairs, int c0, int w) {
    if (pairs.empty()) return;
    std::vector<int64_t> yoff, qoff;
    std::vector<int> m;
    std::vector<BlkDesc> back, save;
    std::vector<SignItem> signs;
    for (int i : pairs) {
        const int64_t st = bstart(l, 2 * i + 1);
        yoff.push_back(st + (int64_t)c0 * N_);
        qoff.push_back(st + (int64_t)kb_[l][i] * N_);
        m.push_back(bsize(l, 2 * i + 1));
        back.push_back(BlkDesc{st + (int64_t)kb_[l][i] * N_, st + (int64_t)c0 * N_, bsize(l, 2 * i + 1), w, (int)N_,
                               (int)N_});
        save.push_back(BlkDesc{st + (int64_t)c0 * N_, st, bsize(l, 2 * i + 1), w, (int)N_, (int)N_});
        for (int j = 0; j < w; ++j)
            signs.push_back(SignItem{st + (int64_t)(kb_[l][i] + j) * N_, st + (int64_t)j * N_, bsize(l, 2 * i + 1)});
    }
    Ysv_.reserve((size_t)N_ * PANEL);
    blocks(BLK_COPY, save, Yt_.p, Ysv_.p);
    for (int round = 0; round < 2; ++round) {
        project(l, pairs, w, c0, 1);
        tsqr_panels((int)pairs.size(), yoff.data(), qoff.data(), m.data(), w, Yt_.p, (int)N_, Pl(l), (int)N_, tsqr_,
                    s_);
        if (round == 0) blocks(BLK_COPY, back, Pl(l), Yt_.p);
    }
    align_signs((int)signs.size(), dev_list(d_sign_, signs, 3), Pl(l), Ysv_.p, s_);
    for (int i : pairs) kb_[l][i] += w;
}

// Q_b = I for the given pairs (their range is all of R^|b|).
void Builder::identity(int l, const std::vector<int>& pairs) {
    std::vector<BlkDesc> d;
    for (int i : pairs) {
        const int m = bsize(l, 2 * i + 1);
        d.push_back(BlkDesc{0, bstart(l, 2 * i + 1), m, m, 0, (int)N_});
        kb_[l][i] = m;
    }
    blocks(BLK_IDENTITY, d, nullptr, Pl(l));
}

void Builder::peel_level(int l) {
    const int npairs = 1 << (l - 1);
    int mb = 0;
    for (int i = 0; i < npairs; ++i) mb = std::max(mb, bsize(l, 2 * i + 1));
    kb_[l].assign(npairs, 0);
    std::vector<int> all(npairs);
    for (int i = 0; i < npairs; ++i) all[i] = i;
    const double thr = tau_test_;
    int range = 0;
    auto range_batch = [&](int col0, int c) {
        probe_fill(N_, c, col0, d_perm_.p, d_row_leaf_.p, L_ - l, o_.seed, STREAM_PROBE, l, Om_.p, Ot_.p, s_);
        call_op(Om_.p, Yo_.p, c, true);
        gather_rows(N_, c, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
        subtract(Ot_.p, Yt_.p, c, l - 1, l, 0);
    };
    // orthonormalise the c new columns [off, off + c) of Yt into the bases; returns the max
    // residual of the test
    auto orth_batch = [&](int c, bool test, int off) {
        std::vector<int> active, full;
        for (int i : all) {
            const int m = bsize(l, 2 * i + 1);
            if (kb_[l][i] >= m) continue;
            if (kb_[l][i] + c >= m) full.push_back(i);
            else active.push_back(i);
        }
        double err = 0.0;
        if (test) {
            std::vector<int> tp = active;
            tp.insert(tp.end(), full.begin(), full.end());
            project(l, tp, c, off, 2);
            for (double e : colnorm(l, tp, c, off)) err = std::max(err, e);
            // certified bases: a passing test's columns stay out of the basis it certified
            if (o_.certified && err <= thr) return err;
        }
        identity(l, full);
        for (int c0 = 0; c0 < c; c0 += PANEL) {
            const int w = std::min(PANEL, c - c0);
            panel(l, active, off + c0, w);
        }
        return err;
    };
    const int q1 = q_start(l);
    int calls = 0, need = 0, passed = 0;
    if (q1 >= mb) {
        identity(l, all);
        need = mb;
        passed = -1;
    } else {
        // after a predicted start the first test uses q_test columns, later growth b_inc
        int inc = predicted(l) ? o_.q_test : o_.b_inc;
        // the first test batch is drawn with the start block: one operator call for both
        const int c1 = (o_.adaptive && q1 < o_.q_max && q1 < mb) ? std::min(inc, o_.q_max - q1) : 0;
        range_batch(0, q1 + c1);
        ++calls;
        orth_batch(q1, false, 0);
        int q = q1;
        need = q;
        bool pending = c1 > 0;
        while (o_.adaptive && q < o_.q_max && q < mb) {
            const int c = std::min(inc, o_.q_max - q);
            inc = o_.b_inc;
            int off = 0;
            if (pending) {
                off = q1;          // columns [q1, q1 + c1) of the first call
                pending = false;
            } else {
                range_batch(q, c);
                ++calls;
            }
            const double err = orth_batch(c, true, off);
            need = q;
            q += c;
            if (err <= thr) {
                passed = 1;
                break;
            }
        }
        if (passed != 1) need = q;
        range = q;
        if (o_.adaptive && q >= o_.q_max && q < mb) cap_hit_ = true;
    }
    range_calls_[l] = calls;
    range_need_[l] = need;
    range_passed_[l] = passed;
    check_flag("range pass", l);
    int qp = 0;
    for (int i : all) qp = std::max(qp, kb_[l][i]);
    // projection pass: Psi (tree order) is P_l itself (Q_b on child-1 rows, zero elsewhere)
    double* P = Pl(l);
    scatter_rows(N_, qp, d_perm_.p, P, N_, Om_.p, N_, s_);
    call_op(Om_.p, Yo_.p, qp, true);
    gather_rows(N_, qp, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    subtract(P, Yt_.p, qp, l - 1, l, 1);
    std::vector<BlkDesc> d;
    for (int i : all) {
        const int64_t st = bstart(l, 2 * i);
        if (kb_[l][i]) d.push_back(BlkDesc{st, st, bsize(l, 2 * i), kb_[l][i], (int)N_, (int)N_});
    }
    blocks(BLK_COPY, d, Yt_.p, P);
    qw_[l] = qp;
    range_probes_[l] = range;
    proj_probes_[l] = qp;
    check_flag("projection pass", l);
}

// dst = src for N x cols tree-order blocks (ld N), in row chunks so that every CTA copies a
// bounded piece.
void Builder::copy_tall(const double* src, double* dst, int cols) {
    std::vector<BlkDesc> d;
    const int chunk = 2048;
    for (int64_t r = 0; r < N_; r += chunk)
        d.push_back(BlkDesc{r, r, (int)std::min<int64_t>(chunk, N_ - r), cols, (int)N_, (int)N_});
    blocks(BLK_COPY, d, src, dst);
}

// Block Gram-Schmidt projection of columns [c0, c0+c) of Yt against the global basis Q.
void Builder::gproject(int c0, int c, int passes) {
    if (!kb0_) return;
    for (int pass = 0; pass < passes; ++pass) {
        gb_.add(Pl(0), (int)N_, 1, Yt_.p + (int64_t)c0 * N_, (int)N_, 0, Cw_.p, kb0_, kb0_, c, (int)N_, 1.0, 0.0);
        gb_.run(s_);
        gb_.add(Pl(0), (int)N_, 0, Cw_.p, kb0_, 0, Yt_.p + (int64_t)c0 * N_, (int)N_, (int)N_, c, kb0_, -1.0, 1.0);
        gb_.run(s_);
    }
}

// Appends the panel columns [c0, c0+w) of Yt to the global basis Q (BCGS2 with TSQR, as for
// the sibling bases, on one panel of all N rows).
void Builder::gpanel(int c0, int w) {
    const int64_t yoff = (int64_t)c0 * N_, qoff = (int64_t)kb0_ * N_;
    const int m = (int)N_;
    for (int round = 0; round < 2; ++round) {
        gproject(c0, w, 1);
        tsqr_panels(1, &yoff, &qoff, &m, w, Yt_.p, (int)N_, Pl(0), (int)N_, tsqr_, s_);
        if (round == 0) copy_tall(Pl(0) + qoff, Yt_.p + yoff, w);
    }
    kb0_ += w;
}

// Global low-rank piece (Section 3.3, end): adaptive randomized range finder on the whole
// matrix (Gaussian probes on every row, start q0, growth b_inc up to global_rank, the levels'
// a-posteriori test with the first test batch drawn in the start call), M = Q^T H Q from one
// more product, semidefinite Cholesky M = C C^T, and B = Q C stored as the level-0 piece.
void Builder::global_pass() {
    const int rmax = o_.global_rank;
    const double thr = tau_test_;
    kb0_ = 0;
    auto batch = [&](int col0, int c) {
        // shift L: every row's leaf index >> L is 0, so every row gets a Gaussian
        probe_fill(N_, c, col0, d_perm_.p, d_row_leaf_.p, L_, o_.seed, STREAM_GLOBAL, 0, Om_.p, nullptr, s_);
        call_op(Om_.p, Yo_.p, c, true);
        gather_rows(N_, c, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    };
    auto orth = [&](int off, int c) {
        for (int c0 = 0; c0 < c; c0 += PANEL) gpanel(off + c0, std::min(PANEL, c - c0));
    };
    const int q1 = std::min(o_.q0, rmax);
    const int c1 = (o_.adaptive && q1 < rmax) ? std::min(o_.b_inc, rmax - q1) : 0;
    batch(0, q1 + c1);
    int calls = 1, passed = 0, q = q1, need = q1;
    orth(0, q1);
    bool pending = c1 > 0;
    while (o_.adaptive && q < rmax) {
        const int c = std::min(o_.b_inc, rmax - q);
        int off = 0;
        if (pending) {
            off = q1;
            pending = false;
        } else {
            batch(q, c);
            ++calls;
        }
        gproject(off, c, 2);
        double err = 0.0;
        {
            const int64_t yo = (int64_t)off * N_;
            const int m = (int)N_;
            panel_colnorm_max(1, dev_list(d_i64a_, std::vector<int64_t>{yo}, 1), dev_list(d_i32a_, std::vector<int>{m}, 2),
                              c, Yt_.p, (int)N_, d_red_.p, s_);
            double* hp = pin_.get<double>(1);
            H2_CUDA(cudaMemcpyAsync(hp, d_red_.p, sizeof(double), cudaMemcpyDeviceToHost, s_));
            H2_CUDA(cudaStreamSynchronize(s_));
            err = *hp;
        }
        orth(off, c);
        need = q;
        q += c;
        if (err <= thr) {
            passed = 1;
            break;
        }
    }
    if (passed != 1) need = q;
    check_flag("global range pass", 0);
    // projection: Z = H Q (tree order), M = Q^T Z, symmetrised, C C^T = M, B = Q C
    const int r = kb0_;
    scatter_rows(N_, r, d_perm_.p, Pl(0), N_, Om_.p, N_, s_);
    call_op(Om_.p, Yo_.p, r, true);
    gather_rows(N_, r, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    check_flag("global projection pass", 0);
    DevBuf<double> Mg((size_t)r * r * 3);
    double* M0 = Mg.p;
    double* M1 = Mg.p + (int64_t)r * r;
    double* Cc = Mg.p + 2 * (int64_t)r * r;
    gb_.add(Pl(0), (int)N_, 1, Yt_.p, (int)N_, 0, M0, r, r, r, (int)N_, 1.0, 0.0);
    gb_.run(s_);
    blocks(BLK_SYMMETRIZE, {BlkDesc{0, 0, r, r, r, r}}, M0, M1);
    psd_cholesky(M1, r, Cc, s_);
    gb_.add(Pl(0), (int)N_, 0, Cc, r, 0, Yt_.p, (int)N_, (int)N_, r, r, 1.0, 0.0);
    gb_.run(s_);
    copy_tall(Yt_.p, Pl(0), r);
    H2_CUDA(cudaStreamSynchronize(s_));
    qw_[0] = r;
    covered_ = passed == 1;
    range_probes_[0] = q;
    proj_probes_[0] = r;
    range_calls_[0] = calls;
    range_need_[0] = need;
    range_passed_[0] = passed;
}

// Identity probes on every leaf give the dense diagonal blocks once all pieces are removed.
void Builder::leaf_pass() {
    const int lm = T_.leaf_max;
    const int nleaf = 1 << L_;
    if (covered_) {
        // the global piece met the threshold: the diagonal blocks are those of B B^T
        ddiag_off_.assign(nleaf, 0);
        int64_t tot = 0;
        for (int t = 0; t < nleaf; ++t) {
            ddiag_off_[t] = tot;
            tot += (int64_t)bsize(L_, t) * bsize(L_, t);
        }
        Ddiag_.reserve((size_t)tot);
        add_global_diag(0.0);
        return;
    }
    fill_zero(Ot_.p, (size_t)N_ * lm, s_);
    std::vector<BlkDesc> d;
    for (int t = 0; t < nleaf; ++t) d.push_back(BlkDesc{0, bstart(L_, t), bsize(L_, t), bsize(L_, t), 0, (int)N_});
    blocks(BLK_IDENTITY, d, nullptr, Ot_.p);
    scatter_rows(N_, lm, d_perm_.p, Ot_.p, N_, Om_.p, N_, s_);
    call_op(Om_.p, Yo_.p, lm, true);
    gather_rows(N_, lm, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    subtract(Ot_.p, Yt_.p, lm, L_);
    ddiag_off_.assign(nleaf, 0);
    int64_t tot = 0;
    for (int t = 0; t < nleaf; ++t) {
        ddiag_off_[t] = tot;
        tot += (int64_t)bsize(L_, t) * bsize(L_, t);
    }
    Ddiag_.reserve((size_t)tot);
    d.clear();
    for (int t = 0; t < nleaf; ++t)
        d.push_back(BlkDesc{bstart(L_, t), ddiag_off_[t], bsize(L_, t), bsize(L_, t), (int)N_, bsize(L_, t)});
    blocks(BLK_SYMMETRIZE, d, Yt_.p, Ddiag_.p);
    check_flag("leaf pass", L_);
    if (qw_[0] > 0) add_global_diag(1.0);
}

// D_tt = B_t B_t^T + beta D_tt on every leaf (the global piece's diagonal blocks).
void Builder::add_global_diag(double beta) {
    const int q = qw_[0];
    for (int t = 0; t < (1 << L_); ++t)
        gb_.add(Pl(0) + bstart(L_, t), (int)N_, 0, Pl(0) + bstart(L_, t), (int)N_, 1, Ddiag_.p + ddiag_off_[t],
                bsize(L_, t), bsize(L_, t), bsize(L_, t), q, 1.0, beta);
    gb_.run(s_);
}

// Recompression of the sampled pieces into nested orthonormal bases, couplings and
// near blocks.
void Builder::assemble(h2_handle_s* h) {
    const int L = L_;
    h->koff.assign(L + 2, 0);
    for (int l = 0; l <= L + 1; ++l) h->koff[l] = (1LL << l) - 1;
    h->k.assign((size_t)h->koff[L + 1], 0);
    // piece columns: level 0 (the global piece of a hybrid construction) then levels 1..L
    std::vector<int64_t> qoff(L + 1, 0);
    int64_t Q = 0;
    for (int l = 0; l <= L; ++l) {
        qoff[l] = Q;
        Q += qw_[l];
    }
    DevBuf<double> Pall, Tall, Rb, Utmp, Uhtmp;
    std::vector<DevBuf<double>> Pi(L + 1);
    std::vector<std::vector<int64_t>> rowoff(L + 1);
    std::vector<int64_t> Krows(L + 1, 0);
    std::vector<int64_t> utmp_off(1 << L, 0), uhtmp_off(h->koff[L], 0);
    DevBuf<int> d_k, d_cap(1);
    H2_CUDA(cudaMemsetAsync(d_cap.p, 0, sizeof(int), s_));
    auto K = [&](int l, int b) -> int& { return h->k[h->koff[l] + b]; };
    auto read_ints = [&](const int* dsrc, int n) {
        std::vector<int> v(n);
        if (!n) return v;
        int* hp = pin_.get<int>(n);
        H2_CUDA(cudaMemcpyAsync(hp, dsrc, n * sizeof(int), cudaMemcpyDeviceToHost, s_));
        H2_CUDA(cudaStreamSynchronize(s_));
        std::memcpy(v.data(), hp, n * sizeof(int));
        return v;
    };
    if (L >= 1 && Q > 0) {
        // compact the pieces: Pall = [P_1 | P_2 | ... | P_L], N x Q
        Pall.reserve((size_t)N_ * Q);
        {
            std::vector<BlkDesc> d;
            const int chunk = 2048;
            for (int l = 0; l <= L; ++l)
                for (int64_t r = 0; r < N_; r += chunk)
                    d.push_back(BlkDesc{pcol_[l] * N_ + r, qoff[l] * N_ + r, (int)std::min<int64_t>(chunk, N_ - r),
                                        qw_[l], (int)N_, (int)N_});
            blocks(BLK_COPY, d, Pcap_.p, Pall.p);
        }
        H2_CUDA(cudaStreamSynchronize(s_));
        Pcap_.release();
        Tw_.release();
        Om_.release(); Yo_.release(); Yt_.release(); Ot_.release();
        auto Pp = [&](int l, int b, int lp) { return Pall.p + bstart(l, b) + qoff[lp] * N_; };

        // QR downsweep (Section 3.2).  Far block (r, s) of level l lies in the sibling piece of
        // its pair level lp (and in the global piece lp = 0), so the far block row of box t is
        // sum_lp P_lp[t] C_lp(t)^T, C_lp(t) the stacked P_lp[s] of the far blocks of t and of
        // its ancestors.  Rs(l, s, lp) = R of P_lp[s]; R(l, t, lp) = R of [R(l-1, parent, lp);
        // Rs(l, s, lp) for the far blocks (t, s) of t itself] (the parent's factor when t has
        // none).  Every factor is c x c (c = qw_[lp]) with reff <= c non-zero rows.
        using Key = std::tuple<int, int, int>;  // (level, box, lp)
        struct RInfo { int64_t off; int reff; };
        std::map<Key, RInfo> rs, rt;
        std::map<Key, std::vector<int>> own;   // (level, t, lp) -> far column boxes of t
        int64_t rtot = 0;
        auto c2 = [&](int lp) { return (int64_t)qw_[lp] * qw_[lp]; };
        const int wide_c = stacked_r_max_columns();
        auto wide = [&](int lp) { return qw_[lp] > wide_c; };
        for (int l = 1; l <= L; ++l)
            for (auto [r, sb] : T_.far[l])
                for (const int lp : {pair_level(l, r, sb), 0}) {
                    if (!qw_[lp] || wide(lp)) continue;
                    Key kb{l, sb, lp};
                    if (!rs.count(kb)) {
                        rs[kb] = RInfo{rtot, std::min(qw_[lp], bsize(l, sb))};
                        rtot += c2(lp);
                    }
                    own[Key{l, r, lp}].push_back(sb);
                }
        for (int l = 1; l <= L; ++l)
            for (int t = 0; t < (1 << l); ++t)
                for (int lp = 0; lp <= l; ++lp) {
                    if (!qw_[lp] || wide(lp)) continue;
                    auto par = rt.find(Key{l - 1, t >> 1, lp});
                    auto ow = own.find(Key{l, t, lp});
                    if (ow == own.end()) {
                        if (par != rt.end()) rt[Key{l, t, lp}] = par->second;   // alias
                        continue;
                    }
                    int rows = par != rt.end() ? par->second.reff : 0;
                    for (int sb : ow->second) rows += rs[Key{l, sb, lp}].reff;
                    rt[Key{l, t, lp}] = RInfo{rtot, std::min(qw_[lp], rows)};
                    rtot += c2(lp);
                }
        Rb.reserve((size_t)std::max<int64_t>(rtot, 1));
        {
            std::vector<StackJob> jobs;
            std::vector<RowSeg> segs;
            for (auto& [key, ri] : rs) {
                auto [l, sb, lp] = key;
                const int q = qw_[lp];
                jobs.push_back(StackJob{(int)segs.size(), (int)segs.size() + 1, q, Rb.p + ri.off, q, nullptr, nullptr});
                segs.push_back(RowSeg{Pp(l, sb, lp), bsize(l, sb), (int)N_});
            }
            stacked_r(jobs, segs, stk_, s_);
        }
        for (int l = 1; l <= L; ++l) {
            std::vector<StackJob> jobs;
            std::vector<RowSeg> segs;
            for (int t = 0; t < (1 << l); ++t)
                for (int lp = 0; lp <= l; ++lp) {
                    auto ow = own.find(Key{l, t, lp});
                    if (ow == own.end() || !qw_[lp]) continue;
                    const int q = qw_[lp];
                    const RInfo ri = rt[Key{l, t, lp}];
                    StackJob jb{(int)segs.size(), 0, q, Rb.p + ri.off, q, nullptr, nullptr};
                    auto par = rt.find(Key{l - 1, t >> 1, lp});
                    // a factor of a stack with at least q rows is upper triangular (tri)
                    if (par != rt.end() && par->second.reff)
                        segs.push_back(RowSeg{Rb.p + par->second.off, par->second.reff, q, par->second.reff == q});
                    for (int sb : ow->second) {
                        const RInfo& si = rs[Key{l, sb, lp}];
                        if (si.reff) segs.push_back(RowSeg{Rb.p + si.off, si.reff, q, si.reff == q});
                    }
                    jb.seg_end = (int)segs.size();
                    jobs.push_back(jb);
                }
            stacked_r(jobs, segs, stk_, s_);
        }

        // Groups wider than stacked_r takes (the global piece of a hybrid construction with a
        // budget above its limit, or levels with that many probes): Gram matrices M(l, t, lp) =
        // C_lp(t)^T C_lp(t) by a downsweep of per-box sums instead of R factors.  Such a group
        // enters a box's SVD through a semidefinite Cholesky factor of P_lp[t] M P_lp[t]^T (its
        // block of W W^T), which resolves its small singular values to sqrt(eps) sigma_max only.
        std::map<Key, int64_t> gcol, gm;
        std::map<Key, std::vector<int64_t>> gown;
        std::map<Key, bool> gm_own;
        int64_t gtot = 0;
        for (int l = 1; l <= L; ++l)
            for (auto [r, sb] : T_.far[l])
                for (const int lp : {pair_level(l, r, sb), 0}) {
                    if (!qw_[lp] || !wide(lp)) continue;
                    Key kb{l, sb, lp};
                    if (!gcol.count(kb)) { gcol[kb] = gtot; gtot += c2(lp); }
                    gown[Key{l, r, lp}].push_back(gcol[kb]);
                }
        for (int l = 1; l <= L; ++l)
            for (int t = 0; t < (1 << l); ++t)
                for (int lp = 0; lp <= l; ++lp) {
                    if (!qw_[lp] || !wide(lp)) continue;
                    auto par = gm.find(Key{l - 1, t >> 1, lp});
                    if (!gown.count(Key{l, t, lp})) {
                        if (par != gm.end()) gm[Key{l, t, lp}] = par->second;
                        continue;
                    }
                    gm[Key{l, t, lp}] = gtot;
                    gm_own[Key{l, t, lp}] = true;
                    gtot += c2(lp);
                }
        DevBuf<double> Gw((size_t)std::max<int64_t>(gtot, 1));
        if (!gcol.empty()) {
            for (auto& [key, off] : gcol) {
                auto [l, sb, lp] = key;
                const int q = qw_[lp];
                gb_.add(Pp(l, sb, lp), (int)N_, 1, Pp(l, sb, lp), (int)N_, 0, Gw.p + off, q, q, q, bsize(l, sb), 1.0, 0.0);
            }
            gb_.run(s_);
            for (int l = 1; l <= L; ++l) {
                std::vector<int64_t> oo, io;
                std::vector<int> len, bg, en;
                for (int t = 0; t < (1 << l); ++t)
                    for (int lp = 0; lp <= l; ++lp) {
                        if (!gm_own.count(Key{l, t, lp})) continue;
                        oo.push_back(gm[Key{l, t, lp}]);
                        len.push_back((int)c2(lp));
                        bg.push_back((int)io.size());
                        auto par = gm.find(Key{l - 1, t >> 1, lp});
                        if (par != gm.end()) io.push_back(par->second);
                        for (int64_t o : gown[Key{l, t, lp}]) io.push_back(o);
                        en.push_back((int)io.size());
                    }
                if (oo.empty()) continue;
                sum_lists((int)oo.size(), dev_list(d_i64a_, oo, 0), dev_list(d_i32a_, len, 1), dev_list(d_i32b_, bg, 2),
                          dev_list(d_i32c_, en, 3), dev_list(d_i64b_, io, 0), Gw.p, Gw.p, 0, s_);
                H2_CUDA(cudaStreamSynchronize(s_));
            }
        }
        // block of W W^T of a wide group for the rows V (rows x q, leading dimension ldv):
        // G = V M V^T into Gsm, then its Cholesky factor into the stack at out (leading dimension ldo)
        DevBuf<double> Vm, Gsm;
        struct WideItem { const double* V; int ldv; int rows; int lp; const double* M; double* out; int ldo; };
        auto wide_blocks = [&](const std::vector<WideItem>& items) {
            if (items.empty()) return;
            int64_t vt = 0, gt2 = 0;
            for (auto& it : items) { vt += (int64_t)it.rows * qw_[it.lp]; gt2 += (int64_t)it.rows * it.rows; }
            Vm.reserve((size_t)vt);
            Gsm.reserve((size_t)gt2);
            int64_t vo = 0, go = 0;
            std::vector<CholItem> ch;
            for (auto& it : items) {
                const int q = qw_[it.lp];
                gb_.add(it.V, it.ldv, 0, it.M, q, 0, Vm.p + vo, it.rows, it.rows, q, q, 1.0, 0.0);
                vo += (int64_t)it.rows * q;
            }
            gb_.run(s_);
            vo = 0;
            for (auto& it : items) {
                const int q = qw_[it.lp];
                gb_.add(Vm.p + vo, it.rows, 0, it.V, it.ldv, 1, Gsm.p + go, it.rows, it.rows, it.rows, q, 1.0, 0.0);
                ch.push_back(CholItem{Gsm.p + go, it.out, it.rows, it.rows, it.ldo});
                vo += (int64_t)it.rows * q;
                go += (int64_t)it.rows * it.rows;
            }
            gb_.run(s_);
            psd_chol_small(ch, stk_, s_);
        };

        // leaves: SVD of W_t = [P_lp[t] R(L, t, lp)^T]_lp through W_t^T (stacked R P^T blocks)
        const int nleaf = 1 << L;
        std::vector<int64_t> toff(nleaf + 1, 0);
        std::vector<int> trows(nleaf, 0);
        for (int t = 0; t < nleaf; ++t) {
            for (int lp = 0; lp <= L; ++lp) {
                auto it = rt.find(Key{L, t, lp});
                if (it != rt.end()) trows[t] += it->second.reff;
                if (gm.count(Key{L, t, lp})) trows[t] += bsize(L, t);
            }
            toff[t + 1] = toff[t] + (int64_t)trows[t] * bsize(L, t);
        }
        Tall.reserve((size_t)std::max<int64_t>(toff[nleaf], 1));
        int64_t ut = 0;
        for (int t = 0; t < nleaf; ++t) {
            utmp_off[t] = ut;
            ut += (int64_t)bsize(L, t) * bsize(L, t);
        }
        Utmp.reserve((size_t)ut);
        {
            std::vector<StackJob> jobs;
            std::vector<RowSeg> segs;
            std::vector<WideItem> witems;
            d_k.reserve(nleaf);
            for (int t = 0; t < nleaf; ++t) {
                int row = 0;
                for (int lp = 0; lp <= L; ++lp) {
                    auto it = rt.find(Key{L, t, lp});
                    if (it != rt.end() && it->second.reff) {
                        const int q = qw_[lp];
                        gb_.add(Rb.p + it->second.off, q, 0, Pp(L, t, lp), (int)N_, 1, Tall.p + toff[t] + row, trows[t],
                                it->second.reff, bsize(L, t), q, 1.0, 0.0);
                        row += it->second.reff;
                    }
                    auto wg = gm.find(Key{L, t, lp});
                    if (wg != gm.end()) {
                        witems.push_back(WideItem{Pp(L, t, lp), (int)N_, bsize(L, t), lp, Gw.p + wg->second,
                                                  Tall.p + toff[t] + row, trows[t]});
                        row += bsize(L, t);
                    }
                }
                jobs.push_back(StackJob{(int)segs.size(), (int)segs.size() + (trows[t] ? 1 : 0), bsize(L, t),
                                        Utmp.p + utmp_off[t], bsize(L, t), d_k.p + t, nullptr});
                if (trows[t]) segs.push_back(RowSeg{Tall.p + toff[t], trows[t], trows[t]});
            }
            gb_.run(s_);
            wide_blocks(witems);
            stacked_svd_trunc(jobs, segs, stk_, tau_basis_, o_.kmax, d_cap.p, s_);
            std::vector<int> kk = read_ints(d_k.p, nleaf);
            for (int t = 0; t < nleaf; ++t) K(L, t) = kk[t];
        }
        Tall.release();
        // projected pieces at the leaves: Pi_L(t) = U_t^T P[t]  (k_t x Q)
        auto level_rows = [&](int l) {
            rowoff[l].assign(1 << l, 0);
            int64_t r = 0;
            for (int b = 0; b < (1 << l); ++b) { rowoff[l][b] = r; r += K(l, b); }
            Krows[l] = std::max<int64_t>(r, 1);
            Pi[l].reserve((size_t)Krows[l] * Q);
        };
        level_rows(L);
        for (int t = 0; t < nleaf; ++t)
            gb_.add(Utmp.p + utmp_off[t], bsize(L, t), 1, Pall.p + bstart(L, t), (int)N_, 0, Pi[L].p + rowoff[L][t],
                    (int)Krows[L], K(L, t), (int)Q, bsize(L, t), 1.0, 0.0);
        gb_.run(s_);
        // upsweep: SVD of [U_c1^T W_p|c1; U_c2^T W_p|c2] = [Pi(c1); Pi(c2)] R(l, p, lp)^T, grouped by lp;
        // every box gets a (2 kmax)^2 slot for its stacked transfer matrices
        const int nmax = 2 * o_.kmax;
        Uhtmp.reserve((size_t)std::max<int64_t>((int64_t)h->koff[L] * nmax * nmax, 1));
        for (int64_t i = 0; i < h->koff[L]; ++i) uhtmp_off[i] = i * nmax * nmax;
        for (int l = L - 1; l >= 1; --l) {
            const int nb = 1 << l;
            const int64_t Kc = Krows[l + 1];
            std::vector<int64_t> to(nb + 1, 0);
            std::vector<int> nn(nb), tr(nb, 0);
            for (int p = 0; p < nb; ++p) {
                nn[p] = K(l + 1, 2 * p) + K(l + 1, 2 * p + 1);
                for (int lp = 0; lp <= l; ++lp) {
                    auto it = rt.find(Key{l, p, lp});
                    if (it != rt.end()) tr[p] += it->second.reff;
                    if (nn[p] && gm.count(Key{l, p, lp})) tr[p] += nn[p];
                }
                to[p + 1] = to[p] + (int64_t)tr[p] * nn[p];
            }
            DevBuf<double> Tb((size_t)std::max<int64_t>(to[nb], 1));
            std::vector<StackJob> jobs;
            std::vector<RowSeg> segs;
            std::vector<WideItem> witems;
            d_k.reserve(nb);
            for (int p = 0; p < nb; ++p) {
                const bool any = nn[p] && tr[p];
                if (any) {
                    const double* V = Pi[l + 1].p + rowoff[l + 1][2 * p];
                    int row = 0;
                    for (int lp = 0; lp <= l; ++lp) {
                        auto it = rt.find(Key{l, p, lp});
                        if (it != rt.end() && it->second.reff) {
                            const int q = qw_[lp];
                            gb_.add(Rb.p + it->second.off, q, 0, V + qoff[lp] * Kc, (int)Kc, 1, Tb.p + to[p] + row,
                                    tr[p], it->second.reff, nn[p], q, 1.0, 0.0);
                            row += it->second.reff;
                        }
                        auto wg = gm.find(Key{l, p, lp});
                        if (wg != gm.end()) {
                            witems.push_back(WideItem{V + qoff[lp] * Kc, (int)Kc, nn[p], lp, Gw.p + wg->second,
                                                      Tb.p + to[p] + row, tr[p]});
                            row += nn[p];
                        }
                    }
                }
                jobs.push_back(StackJob{(int)segs.size(), (int)segs.size() + (any ? 1 : 0), nn[p],
                                        Uhtmp.p + uhtmp_off[h->koff[l] + p], std::max(nn[p], 1), d_k.p + p, nullptr});
                if (any) segs.push_back(RowSeg{Tb.p + to[p], tr[p], tr[p]});
            }
            gb_.run(s_);
            wide_blocks(witems);
            stacked_svd_trunc(jobs, segs, stk_, tau_basis_, o_.kmax, d_cap.p, s_);
            std::vector<int> kk = read_ints(d_k.p, nb);
            for (int p = 0; p < nb; ++p) K(l, p) = kk[p];
            level_rows(l);
            for (int p = 0; p < nb; ++p) {
                if (!nn[p] || !K(l, p)) continue;
                const double* V = Pi[l + 1].p + rowoff[l + 1][2 * p];
                gb_.add(Uhtmp.p + uhtmp_off[h->koff[l] + p], nn[p], 1, V, (int)Kc, 0, Pi[l].p + rowoff[l][p],
                        (int)Krows[l], K(l, p), (int)Q, nn[p], 1.0, 0.0);
            }
            gb_.run(s_);
        }
    }
    // factor layout now that all ranks are known
    layout_factors(h);
    double* fac = h->fac64.p;
    if (L >= 1 && Q > 0) {
        std::vector<BlkDesc> d;
        for (int t = 0; t < (1 << L); ++t)
            if (K(L, t)) d.push_back(BlkDesc{utmp_off[t], h->u_off[t], bsize(L, t), K(L, t), bsize(L, t), bsize(L, t)});
        blocks(BLK_COPY, d, Utmp.p, fac);
        d.clear();
        for (int l = 1; l < L; ++l)
            for (int p = 0; p < (1 << l); ++p) {
                const int n = K(l + 1, 2 * p) + K(l + 1, 2 * p + 1), kp = K(l, p);
                if (n && kp) d.push_back(BlkDesc{uhtmp_off[h->koff[l] + p], h->uh_off[h->koff[l] + p], n, kp, n, n});
            }
        blocks(BLK_COPY, d, Uhtmp.p, fac);
        // couplings S_ts = Pi_lp(t) Pi_lp(s)^T (+ Pi_0(t) Pi_0(s)^T for the global piece, added in
        // a second batch: the problems of one batch must write disjoint blocks)
        for (const bool global : {false, true}) {
            if (global && !qw_[0]) break;
            for (int l = 1; l <= L; ++l)
                for (size_t i = 0; i < h->far_lower[l].size(); ++i) {
                    auto [t, sb] = h->far_lower[l][i];
                    const int lp = global ? 0 : pair_level(l, t, sb);
                    const int q = qw_[lp];
                    const int64_t Kl = Krows[l];
                    gb_.add(Pi[l].p + rowoff[l][t] + qoff[lp] * Kl, (int)Kl, 0, Pi[l].p + rowoff[l][sb] + qoff[lp] * Kl,
                            (int)Kl, 1, fac + h->s_off[l][i], std::max(K(l, t), 1), K(l, t), K(l, sb), q, 1.0,
                            global ? 1.0 : 0.0);
                }
            gb_.run(s_);
        }
        // off-diagonal near blocks D_ts = P_lp[t] P_lp[s]^T (+ B_t B_s^T)
        for (const bool global : {false, true}) {
            if (global && !qw_[0]) break;
            for (size_t i = 0; i < h->near_lower.size(); ++i) {
                auto [t, sb] = h->near_lower[i];
                if (t == sb) continue;
                const int lp = global ? 0 : pair_level(L, t, sb);
                gb_.add(Pall.p + bstart(L, t) + qoff[lp] * N_, (int)N_, 0, Pall.p + bstart(L, sb) + qoff[lp] * N_,
                        (int)N_, 1, fac + h->d_off[i], bsize(L, t), bsize(L, t), bsize(L, sb), qw_[lp], 1.0,
                        global ? 1.0 : 0.0);
            }
            gb_.run(s_);
        }
    }
    {
        std::vector<BlkDesc> d;
        for (size_t i = 0; i < h->near_lower.size(); ++i) {
            auto [t, sb] = h->near_lower[i];
            if (t != sb) continue;
            d.push_back(BlkDesc{ddiag_off_[t], h->d_off[i], bsize(L, t), bsize(L, t), bsize(L, t), bsize(L, t)});
        }
        blocks(BLK_COPY, d, Ddiag_.p, fac);
    }
    int cap = read_ints(d_cap.p, 1)[0];
    if (cap) cap_hit_ = true;
    H2_CUDA(cudaStreamSynchronize(s_));
}

void Builder::run(h2_handle_s* h) {
    const double t0 = now_s();
    const int nleaf = 1 << L_;
    if (T_.leaf_max > svd_max_order()) fail(H2_ERR_INVALID_ARG, "h2_build: leaf size above 96 is not supported");
    if (2 * o_.kmax > svd_max_order()) fail(H2_ERR_INVALID_ARG, "h2_build: kmax above 48 is not supported");
    {
        std::vector<int32_t> perm(N_), rl(N_);
        for (int64_t i = 0; i < N_; ++i) perm[i] = (int32_t)T_.perm[i];
        for (int t = 0; t < nleaf; ++t)
            for (int64_t i = 0; i < T_.size[L_][t]; ++i) rl[T_.start[L_][t] + i] = t;
        upload(d_perm_, perm, s_, stg_[0]);
        upload(d_row_leaf_, rl, s_, stg_[1]);
    }
    qcap_.assign(L_ + 1, 0);
    qw_.assign(L_ + 1, 0);
    pcol_.assign(L_ + 1, 0);
    kb_.assign(L_ + 1, {});
    range_probes_.assign(L_ + 1, 0);
    proj_probes_.assign(L_ + 1, 0);
    range_calls_.assign(L_ + 1, 0);
    range_need_.assign(L_ + 1, 0);
    range_passed_.assign(L_ + 1, 0);
    int64_t pc = 0;
    int qcmax = 1;
    cmax_ = std::max({o_.q0, o_.b_inc, o_.q_test, T_.leaf_max, 1});
    const bool hybrid = o_.global_rank > 0 && L_ >= 1;
    if (hybrid) {
        if (o_.global_rank >= N_) fail(H2_ERR_INVALID_ARG, "h2_build: global_rank must be below n");
        if (N_ > kGlobalMaxRows) fail(H2_ERR_INVALID_ARG, "h2_build: global_rank needs n <= 14,155,776");
        qcap_[0] = o_.global_rank;
        pc = o_.global_rank;
        cmax_ = std::max({cmax_, std::min(o_.q0, o_.global_rank) + o_.b_inc, o_.global_rank});
    }
    for (int l = 1; l <= L_; ++l) {
        int mb = 0;
        for (int i = 0; i < (1 << (l - 1)); ++i) mb = std::max(mb, bsize(l, 2 * i + 1));
        const int q1 = q_start(l);
        qcap_[l] = (q1 >= mb) ? mb : std::min(std::max(o_.q_max, q1), mb);
        // the first call draws the start block and the first test batch
        if (q1 < mb) cmax_ = std::max(cmax_, q1 + std::max(o_.q_test, o_.b_inc));
        pcol_[l] = pc;
        pc += qcap_[l];
        qcmax = std::max(qcmax, qcap_[l]);
        cmax_ = std::max(cmax_, qcap_[l]);
    }
    Om_.reserve((size_t)N_ * cmax_);
    Yo_.reserve((size_t)N_ * cmax_);
    Yt_.reserve((size_t)N_ * cmax_);
    Ot_.reserve((size_t)N_ * cmax_);
    Tw_.reserve((size_t)(N_ + nleaf) * cmax_);
    Cw_.reserve(std::max((size_t)std::max(1, nleaf / 2) * qcmax * PANEL,
                         hybrid ? (size_t)o_.global_rank * std::max(PANEL, o_.b_inc) : (size_t)0));
    Pcap_.reserve((size_t)std::max<int64_t>(N_ * pc, 1));
    fill_zero(Pcap_.p, (size_t)N_ * pc, s_);
    d_flag_.reserve(1);
    H2_CUDA(cudaMemsetAsync(d_flag_.p, 0, sizeof(int), s_));
    d_red_.reserve(std::max(nleaf, 4) + 4);

    const double tn = now_s();
    if (o_.norm_est > 0.0) norm_ = o_.norm_est;
    else norm_ = norm_estimate();
    const double tn1 = now_s();
    tau_test_ = tol_ * norm_ / (10.0 * std::sqrt(2.0 / M_PI));
    tau_basis_ = 2.0 * tol_ * norm_ / std::sqrt((double)nleaf);
    if (hybrid) global_pass();
    for (int l = 1; l <= L_; ++l) {
        if (covered_) {
            kb_[l].assign(1 << (l - 1), 0);
            range_passed_[l] = 2;   // not sampled: the global piece met the threshold
            continue;
        }
        peel_level(l);
    }
    leaf_pass();
    const double tp = now_s();
    assemble(h);
    const double ta = now_s();

    h2_stats& st = h->stats;
    std::memset(&st, 0, sizeof(st));
    st.n = N_;
    st.levels = L_;
    st.leaf_max = T_.leaf_max;
    st.samples = samples_;
    st.norm_products = norm_products_;
    st.op_calls = op_calls_;
    for (int l = 0; l <= L_ && l < H2_MAX_LEVELS; ++l) {
        st.range_probes[l] = range_probes_[l];
        st.proj_probes[l] = proj_probes_[l];
        st.range_calls[l] = range_calls_[l];
        st.range_need[l] = range_need_[l];
        st.range_passed[l] = range_passed_[l];
        int mx = 0;
        for (int b = 0; b < (1 << l); ++b) mx = std::max(mx, h->k[h->koff[l] + b]);
        st.max_rank[l] = mx;
    }
    st.norm_est = norm_;
    st.tau_basis = tau_basis_;
    st.tau_test = tau_test_;
    st.tol_met = cap_hit_ ? 0 : 1;
    st.t_total = ta - t0;
    st.t_norm = tn1 - tn;
    st.t_op = t_op_;
    st.t_peel = tp - tn1;
    st.t_assemble = ta - tp;
}

}  // namespace

int build_colored(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o, h2_handle_s* h);

int build_handle(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o,
                 h2_handle_s* h) {
    if (o.sampling == H2_SAMPLING_COLORED) return build_colored(op, ctx, tree, tol, o, h);
    h->tree = std::make_shared<h2_tree_s>(*tree);
    h->L = tree->L;
    h->N = tree->N;
    Builder b(*tree, op, ctx, tol, o);
    b.run(h);
    return h->stats.tol_met ? H2_OK : H2_WARN_TOL_NOT_MET;
}

}  // namespace h2
