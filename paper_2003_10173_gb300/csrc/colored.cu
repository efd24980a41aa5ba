// Construction by strong-structure coloured sampling (Section 3.3): the alternative to the weak
// sampling structure of build.cu, kept as a comparison mode for the trade between the number of
// probe blocks per level (C_l) and the rank of the sampled blocks (k).
//
// Level by level from coarse to fine, the far blocks of the destination partition are sampled
// themselves.  After the coarser levels' pieces are removed, the residual at level l has nonzero
// blocks only on the pairs that the partition visits at level l (V_l: far blocks and inadmissible
// pairs); a probe block may serve several column boxes at once when no row box sees two of them
// in V_l.  So:
//   range pass: the column boxes s of the lower far pairs (t > s) are coloured greedily (distance
//     2 in V_l, box order); colour c owns q Gaussian columns on its boxes; one product gives
//     H[t, s] Omega_s for every pair at once, and Q_ts is the signed Q factor of that block;
//   projection pass: the pairs get probe slots greedily (no two pairs of one slot share a row
//     box t, and no pair's row box reaches another's column box through V_l); slot j carries
//     Q_ts on the rows of t; one product gives Z_ts = H[s, t] Q_ts, and H[t, s] ~ Q_ts Z_ts^T;
//   leaf pass: the leaves are coloured over the near pairs; identity blocks per colour give
//     every near block after all pieces are removed.
// Assembly: every pair is one group of the recompression (QR-weighted block rows, Section 3.2):
// the far block row of box x collects Q_g[x] R(Z_g)^T for the pairs whose row box is x or an
// ancestor and Z_g[x] for the pairs whose column box is (R(Q_g) = I); leaf bases and transfer
// matrices come from truncated SVDs of these rows (leaves, then upsweep of the projected
// factors Pi_{x,g} = Ubar_x^T P_g[x]); couplings Pi_{t,g} Pi_{s,g}^T.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <set>
#include <string>

#include "handle.h"

namespace h2 {

namespace {

constexpr int STREAM_POWER = 2;
constexpr int STREAM_COLORED = 8;   // probes of the coloured range pass

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Sampling plan of one level.
struct ColorLevel {
    std::vector<std::pair<int, int>> pairs;   // lower far pairs (t > s), in (t, s) order
    std::vector<int32_t> color;                // per box: colour as a column box, -1 if none
    std::vector<int> slot;                     // per pair: probe slot of the projection pass
    std::vector<int> jq, jz;                   // per pair: index among the pairs of t (of s)
    std::vector<int> nq, nz;                   // per box: pairs with the box as t (as s)
    std::vector<std::vector<int>> by_t, by_s;  // per box: its pairs as t (as s), in order
    std::vector<int> zstart;                   // per box: pairs with a smaller column box
    int ncolors = 0, nslots = 0;
    int qcols = 0, zcols = 0;                  // columns of the Q and Z piece arrays
};

// V[l][t]: the boxes s with (t, s) visited at level l (far, or inadmissible and split further, or
// a near block), sorted.  Bottom-up: the inadmissible pairs of level l are the parents of the
// pairs visited at level l + 1; at the leaves they are the near blocks.
std::vector<std::vector<std::vector<int>>> visited(const h2_tree_s& T) {
    const int L = T.L;
    std::vector<std::set<std::pair<int, int>>> inadm(L + 1);
    for (auto [t, s] : T.near) inadm[L].insert({t, s});
    for (int l = L - 1; l >= 0; --l) {
        for (auto [t, s] : inadm[l + 1]) inadm[l].insert({t >> 1, s >> 1});
        for (auto [t, s] : T.far[l + 1]) inadm[l].insert({t >> 1, s >> 1});
    }
    std::vector<std::vector<std::vector<int>>> V(L + 1);
    for (int l = 0; l <= L; ++l) {
        V[l].assign(1 << l, {});
        for (auto [t, s] : inadm[l]) V[l][t].push_back(s);
        for (auto [t, s] : T.far[l]) V[l][t].push_back(s);
        for (auto& v : V[l]) {
            std::sort(v.begin(), v.end());
            v.erase(std::unique(v.begin(), v.end()), v.end());
        }
    }
    return V;
}

// Greedy distance-2 colouring of the boxes with active[b] (increasing order) over V.
std::vector<int32_t> color_boxes(const std::vector<std::vector<int>>& V, const std::vector<char>& active, int* ncolors) {
    const int nb = (int)V.size();
    std::vector<int32_t> color(nb, -1);
    std::vector<int> mark(nb + 1, -1);
    *ncolors = 0;
    for (int s = 0; s < nb; ++s) {
        if (!active[s]) continue;
        for (int t : V[s])
            for (int s2 : V[t])
                if (color[s2] >= 0) mark[color[s2]] = s;
        int c = 0;
        while (mark[c] == s) ++c;
        color[s] = c;
        *ncolors = std::max(*ncolors, c + 1);
    }
    return color;
}

std::vector<ColorLevel> color_plan(const h2_tree_s& T, const std::vector<std::vector<std::vector<int>>>& V, int q) {
    const int L = T.L;
    std::vector<ColorLevel> P(L + 1);
    for (int l = 1; l <= L; ++l) {
        ColorLevel& C = P[l];
        const int nb = 1 << l;
        for (auto [t, s] : T.far[l])
            if (t > s) C.pairs.push_back({t, s});
        std::sort(C.pairs.begin(), C.pairs.end());
        std::vector<char> active(nb, 0);
        for (auto [t, s] : C.pairs) {
            active[s] = 1;
            if (T.size[l][t] <= q) fail(H2_ERR_INVALID_ARG, "coloured sampling: q0 must be below every box size");
        }
        C.color = color_boxes(V[l], active, &C.ncolors);
        // probe slots of the projection pass
        std::vector<std::vector<char>> inT, inS;
        for (auto [t, s] : C.pairs) {
            int j = 0;
            for (; j < (int)inT.size(); ++j) {
                bool bad = inT[j][t] != 0;
                for (int x : V[l][s]) bad = bad || inT[j][x];
                for (int x : V[l][t]) bad = bad || inS[j][x];
                if (!bad) break;
            }
            if (j == (int)inT.size()) {
                inT.emplace_back(nb, 0);
                inS.emplace_back(nb, 0);
            }
            inT[j][t] = 1;
            inS[j][s] = 1;
            C.slot.push_back(j);
        }
        C.nslots = (int)inT.size();
        C.nq.assign(nb, 0);
        C.nz.assign(nb, 0);
        C.by_t.assign(nb, {});
        C.by_s.assign(nb, {});
        for (size_t p = 0; p < C.pairs.size(); ++p) {
            auto [t, s] = C.pairs[p];
            C.jq.push_back(C.nq[t]++);
            C.jz.push_back(C.nz[s]++);
            C.by_t[t].push_back((int)p);
            C.by_s[s].push_back((int)p);
        }
        C.zstart.assign(nb + 1, 0);
        for (int b = 0; b < nb; ++b) {
            C.qcols = std::max(C.qcols, C.nq[b] * q);
            C.zcols = std::max(C.zcols, C.nz[b] * q);
            C.zstart[b + 1] = C.zstart[b] + C.nz[b];
        }
    }
    return P;
}

class ColoredBuilder {
  public:
    ColoredBuilder(const h2_tree_s& T, h2_op_fn op, void* ctx, double tol, const h2_build_opts& o)
        : T_(T), op_(op), ctx_(ctx), tol_(tol), o_(o), s_((cudaStream_t)o.stream), N_(T.N), L_(T.L), q_(o.q0) {}
    void run(h2_handle_s* h);

  private:
    const h2_tree_s& T_;
    h2_op_fn op_;
    void* ctx_;
    double tol_;
    h2_build_opts o_;
    cudaStream_t s_;
    int64_t N_;
    int L_, q_;
    std::vector<std::vector<std::vector<int>>> V_;
    std::vector<ColorLevel> P_;
    std::vector<int32_t> leaf_color_;
    int nleafcol_ = 0;
    DevBuf<int32_t> d_perm_, d_row_leaf_, d_color_;
    DevBuf<double> Om_, Omt_, Yo_, Yt_, Sam_, Ysc_, T1_, T2_;
    std::vector<DevBuf<double>> Q_, Z_;   // per level: N x qcols (Q_ts of box t at column jq q) and
                                          // N x zcols (Z_ts of box s at column jz q), tree order
    DevBuf<double> Dn_;                   // near blocks (t >= s) in the order of the tree's near list
    std::vector<int64_t> dn_off_;
    GemmBatch gb_;
    TsqrWork tsqr_;
    StackWork stk_;
    Stager stg_[4];
    DevBuf<BlkDesc> d_blk_;
    DevBuf<SignItem> d_sign_;
    DevBuf<int> d_flag_;
    DevBuf<double> d_red_;
    Pinned pin_;
    int64_t samples_ = 0, norm_products_ = 0, op_calls_ = 0;
    double t_op_ = 0.0, norm_ = 0.0, tau_basis_ = 0.0;
    bool cap_hit_ = false;

    int64_t bstart(int l, int b) const { return T_.start[l][b]; }
    int bsize(int l, int b) const { return (int)T_.size[l][b]; }
    template <class T>
    T* dev_list(DevBuf<T>& buf, const std::vector<T>& v, int which) {
        upload(buf, v, s_, stg_[which & 3]);
        return buf.p;
    }
    void blocks(int kind, const std::vector<BlkDesc>& d, const double* src, double* dst) {
        if (d.empty()) return;
        const std::vector<BlkDesc> ds = kind == BLK_COPY ? split_copies(d) : d;
        block_op(kind, (int)ds.size(), dev_list(d_blk_, ds, 0), src, dst, s_);
    }
    const double* Qp(int l, int p) const {
        return Q_[l].p + bstart(l, P_[l].pairs[p].first) + (int64_t)P_[l].jq[p] * q_ * N_;
    }
    const double* Zp(int l, int p) const {
        return Z_[l].p + bstart(l, P_[l].pairs[p].second) + (int64_t)P_[l].jz[p] * q_ * N_;
    }
    void call_op(const double* X, double* Y, int ncols, bool count_sample);
    void check_flag(const char* where, int level);
    double norm_estimate();
    void subtract(const double* Xt, double* Yt, int c, int lmax);
    void sample_level(int l);
    void leaf_pass();
    void assemble(h2_handle_s* h);
};

void ColoredBuilder::call_op(const double* X, double* Y, int ncols, bool count_sample) {
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

void ColoredBuilder::check_flag(const char* where, int level) {
    int* f = pin_.get<int>(1);
    H2_CUDA(cudaMemcpyAsync(f, d_flag_.p, sizeof(int), cudaMemcpyDeviceToHost, s_));
    H2_CUDA(cudaStreamSynchronize(s_));
    if (*f)
        fail(H2_ERR_NAN, std::string("non-finite values in Hessian-vector products (") + where + ", level " +
                             std::to_string(level) + ")");
}

// ||H||_2 by power iteration from the construction's Gaussian start vector (Section 3.2).
double ColoredBuilder::norm_estimate() {
    DevBuf<double> V((size_t)2 * N_);
    double* v = V.p;
    double* w = V.p + N_;
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

// Y -= K X for the pieces of levels 1..lmax (tree order, N x c, ld N): for every pair,
// Y[t] -= Q_ts (Z_ts^T X[s]) and Y[s] -= Z_ts (Q_ts^T X[t]).  The small products of all pairs
// of a level go to T1 (stacked by row box) and T2 (stacked by column box), so that each box's
// update is one product with its contiguous piece columns; columns in chunks that bound T1, T2.
void ColoredBuilder::subtract(const double* Xt, double* Yt, int c, int lmax) {
    constexpr int64_t kChunkEntries = (int64_t)1 << 26;
    for (int l = 1; l <= lmax; ++l) {
        const ColorLevel& C = P_[l];
        const int np = (int)C.pairs.size();
        if (!np) continue;
        const int R = q_ * np;
        const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(c, kChunkEntries / R));
        for (int c0 = 0; c0 < c; c0 += chunk) {
            const int w = std::min(chunk, c - c0);
            T1_.reserve((size_t)R * w);
            T2_.reserve((size_t)R * w);
            const int64_t xo = (int64_t)c0 * N_;
            for (int p = 0; p < np; ++p) {
                auto [t, s] = C.pairs[p];
                gb_.add(Zp(l, p), (int)N_, 1, Xt + bstart(l, s) + xo, (int)N_, 0, T1_.p + (int64_t)p * q_, R, q_, w,
                        bsize(l, s), 1.0, 0.0);
                gb_.add(Qp(l, p), (int)N_, 1, Xt + bstart(l, t) + xo, (int)N_, 0,
                        T2_.p + (int64_t)(C.zstart[s] + C.jz[p]) * q_, R, q_, w, bsize(l, t), 1.0, 0.0);
            }
            gb_.run(s_);
            for (int t = 0; t < (1 << l); ++t)
                if (C.nq[t])
                    gb_.add(Q_[l].p + bstart(l, t), (int)N_, 0, T1_.p + (int64_t)C.by_t[t][0] * q_, R, 0,
                            Yt + bstart(l, t) + xo, (int)N_, bsize(l, t), w, C.nq[t] * q_, -1.0, 1.0);
            gb_.run(s_);
            for (int s = 0; s < (1 << l); ++s)
                if (C.nz[s])
                    gb_.add(Z_[l].p + bstart(l, s), (int)N_, 0, T2_.p + (int64_t)C.zstart[s] * q_, R, 0,
                            Yt + bstart(l, s) + xo, (int)N_, bsize(l, s), w, C.nz[s] * q_, -1.0, 1.0);
            gb_.run(s_);
        }
    }
}


// Range and projection passes of level l (see the file notes).
void ColoredBuilder::sample_level(int l) {
    const ColorLevel& C = P_[l];
    const int np = (int)C.pairs.size();
    const int q = q_;
    // range pass: colour c owns the probe columns [c q, (c + 1) q)
    const int cr = C.ncolors * q;
    upload(d_color_, C.color, s_, stg_[1]);
    probe_fill_colored(N_, q, C.ncolors, d_perm_.p, d_row_leaf_.p, L_ - l, d_color_.p, o_.seed, STREAM_COLORED, l, Om_.p,
                       Omt_.p, s_);
    call_op(Om_.p, Yo_.p, cr, true);
    gather_rows(N_, cr, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    check_flag("coloured range pass", l);
    subtract(Omt_.p, Yt_.p, cr, l - 1);
    // the sample block of every pair, Y[t, colour(s)], into its piece column; Q_ts = signed Q factor
    Q_[l].reserve((size_t)N_ * std::max(C.qcols, 1));
    Sam_.reserve((size_t)N_ * std::max(C.qcols, 1));
    Ysc_.reserve((size_t)N_ * std::max(C.qcols, 1));
    std::vector<BlkDesc> d;
    std::vector<int64_t> off;
    std::vector<int> m;
    std::vector<SignItem> signs;
    for (int p = 0; p < np; ++p) {
        auto [t, s] = C.pairs[p];
        const int64_t dst = bstart(l, t) + (int64_t)C.jq[p] * q * N_;
        d.push_back(BlkDesc{bstart(l, t) + (int64_t)C.color[s] * q * N_, dst, bsize(l, t), q, (int)N_, (int)N_});
        off.push_back(dst);
        m.push_back(bsize(l, t));
        for (int j = 0; j < q; ++j) signs.push_back(SignItem{dst + (int64_t)j * N_, dst + (int64_t)j * N_, bsize(l, t)});
    }
    blocks(BLK_COPY, d, Yt_.p, Sam_.p);
    blocks(BLK_COPY, d, Yt_.p, Ysc_.p);
    tsqr_panels(np, off.data(), off.data(), m.data(), q, Ysc_.p, (int)N_, Q_[l].p, (int)N_, tsqr_, s_);
    align_signs((int)signs.size(), dev_list(d_sign_, signs, 2), Q_[l].p, Sam_.p, s_);
    // projection pass: slot j carries Q_ts on the rows of t in the columns [j q, (j + 1) q)
    const int cp = C.nslots * q;
    fill_zero(Omt_.p, (size_t)N_ * cp, s_);
    d.clear();
    for (int p = 0; p < np; ++p) {
        auto [t, s] = C.pairs[p];
        d.push_back(BlkDesc{bstart(l, t) + (int64_t)C.jq[p] * q * N_, bstart(l, t) + (int64_t)C.slot[p] * q * N_,
                            bsize(l, t), q, (int)N_, (int)N_});
    }
    blocks(BLK_COPY, d, Q_[l].p, Omt_.p);
    scatter_rows(N_, cp, d_perm_.p, Omt_.p, N_, Om_.p, N_, s_);
    call_op(Om_.p, Yo_.p, cp, true);
    gather_rows(N_, cp, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    check_flag("coloured projection pass", l);
    subtract(Omt_.p, Yt_.p, cp, l - 1);
    Z_[l].reserve((size_t)N_ * std::max(C.zcols, 1));
    d.clear();
    for (int p = 0; p < np; ++p) {
        auto [t, s] = C.pairs[p];
        d.push_back(BlkDesc{bstart(l, s) + (int64_t)C.slot[p] * q * N_, bstart(l, s) + (int64_t)C.jz[p] * q * N_,
                            bsize(l, s), q, (int)N_, (int)N_});
    }
    blocks(BLK_COPY, d, Yt_.p, Z_[l].p);
    H2_CUDA(cudaStreamSynchronize(s_));
}

// Near blocks: identity probes on the leaves of each colour; after all pieces are removed, block
// (t, s) is read from the rows of t in the columns of colour(s) (diagonal blocks symmetrised).
void ColoredBuilder::leaf_pass() {
    const int L = L_, lm = T_.leaf_max, nleaf = 1 << L;
    const int c = nleafcol_ * lm;
    fill_zero(Omt_.p, (size_t)N_ * c, s_);
    std::vector<BlkDesc> d;
    for (int t = 0; t < nleaf; ++t)
        d.push_back(BlkDesc{0, bstart(L, t) + (int64_t)leaf_color_[t] * lm * N_, bsize(L, t), bsize(L, t), 0, (int)N_});
    blocks(BLK_IDENTITY, d, nullptr, Omt_.p);
    scatter_rows(N_, c, d_perm_.p, Omt_.p, N_, Om_.p, N_, s_);
    call_op(Om_.p, Yo_.p, c, true);
    gather_rows(N_, c, d_perm_.p, Yo_.p, N_, Yt_.p, N_, s_);
    check_flag("coloured leaf pass", L);
    subtract(Omt_.p, Yt_.p, c, L);
    dn_off_.clear();
    int64_t tot = 0;
    std::vector<BlkDesc> cp, sym;
    for (auto [t, s] : T_.near) {
        if (t < s) continue;
        dn_off_.push_back(tot);
        const BlkDesc b{bstart(L, t) + (int64_t)leaf_color_[s] * lm * N_, tot, bsize(L, t), bsize(L, s), (int)N_,
                        bsize(L, t)};
        (t == s ? sym : cp).push_back(b);
        tot += (int64_t)bsize(L, t) * bsize(L, s);
    }
    Dn_.reserve((size_t)std::max<int64_t>(tot, 1));
    blocks(BLK_COPY, cp, Yt_.p, Dn_.p);
    blocks(BLK_SYMMETRIZE, sym, Yt_.p, Dn_.p);
    H2_CUDA(cudaStreamSynchronize(s_));
}


// H^2 form of the sampled matrix: every pair is one group of the QR-weighted block rows.
void ColoredBuilder::assemble(h2_handle_s* h) {
    const int L = L_, q = q_, nleaf = 1 << L;
    h->koff.assign(L + 2, 0);
    for (int l = 0; l <= L + 1; ++l) h->koff[l] = (1LL << l) - 1;
    h->k.assign((size_t)h->koff[L + 1], 0);
    auto K = [&](int l, int b) -> int& { return h->k[h->koff[l] + b]; };
    // groups touching each box: its parent's, then the pairs of its own level with the box as t
    // (side 0: rows of Q_ts), then as s (side 1: rows of Z_ts)
    struct G { int l, p, side; };
    std::vector<std::vector<std::vector<G>>> own(L + 1);
    std::vector<std::vector<int>> ng(L + 1);
    ng[0].assign(1, 0);
    for (int l = 1; l <= L; ++l) {
        own[l].assign(1 << l, {});
        ng[l].assign(1 << l, 0);
        for (int b = 0; b < (1 << l); ++b) {
            if (!P_[l].pairs.empty()) {
                for (int p : P_[l].by_t[b]) own[l][b].push_back(G{l, p, 0});
                for (int p : P_[l].by_s[b]) own[l][b].push_back(G{l, p, 1});
            }
            ng[l][b] = ng[l - 1][b >> 1] + (int)own[l][b].size();
        }
    }
    auto group = [&](int l, int b, int i) -> G {   // the i-th group of box b at level l
        while (i < ng[l - 1][b >> 1]) {
            b >>= 1;
            --l;
        }
        return own[l][b][i - ng[l - 1][b >> 1]];
    };
    auto piece = [&](const G& g, int64_t row) -> const double* {   // rows of the group's factor
        const ColorLevel& C = P_[g.l];
        return g.side == 0 ? Q_[g.l].p + row + (int64_t)C.jq[g.p] * q * N_ : Z_[g.l].p + row + (int64_t)C.jz[g.p] * q * N_;
    };
    // weights: R of Z_ts for side 0, the identity for side 1 (Q_ts has orthonormal columns)
    std::vector<std::vector<int64_t>> rzoff(L + 1);
    int64_t rzt = 0;
    for (int l = 1; l <= L; ++l) {
        rzoff[l].assign(P_[l].pairs.size(), 0);
        for (size_t p = 0; p < P_[l].pairs.size(); ++p) { rzoff[l][p] = rzt; rzt += (int64_t)q * q; }
    }
    DevBuf<double> Rz((size_t)std::max<int64_t>(rzt, 1)), Iq((size_t)q * q);
    {
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int l = 1; l <= L; ++l)
            for (size_t p = 0; p < P_[l].pairs.size(); ++p) {
                jobs.push_back(StackJob{(int)segs.size(), (int)segs.size() + 1, q, Rz.p + rzoff[l][p], q, nullptr, nullptr});
                segs.push_back(RowSeg{Zp(l, (int)p), bsize(l, P_[l].pairs[p].second), (int)N_});
            }
        stacked_r(jobs, segs, stk_, s_);
        fill_zero(Iq.p, Iq.n, s_);
        blocks(BLK_IDENTITY, {BlkDesc{0, 0, q, q, 0, q}}, nullptr, Iq.p);
    }
    auto weight = [&](const G& g) -> const double* { return g.side == 0 ? Rz.p + rzoff[g.l][g.p] : Iq.p; };
    DevBuf<int> d_k((size_t)nleaf), d_cap(1);
    H2_CUDA(cudaMemsetAsync(d_cap.p, 0, sizeof(int), s_));
    auto read_ints = [&](const int* dsrc, int n) {
        std::vector<int> v(n);
        int* hp = pin_.get<int>(n);
        H2_CUDA(cudaMemcpyAsync(hp, dsrc, n * sizeof(int), cudaMemcpyDeviceToHost, s_));
        H2_CUDA(cudaStreamSynchronize(s_));
        std::memcpy(v.data(), hp, n * sizeof(int));
        return v;
    };
    // leaves
    std::vector<int64_t> uoff(nleaf + 1, 0), woff(nleaf + 1, 0);
    for (int x = 0; x < nleaf; ++x) {
        uoff[x + 1] = uoff[x] + (int64_t)bsize(L, x) * bsize(L, x);
        woff[x + 1] = woff[x] + (int64_t)q * ng[L][x] * bsize(L, x);
    }
    DevBuf<double> Utmp((size_t)std::max<int64_t>(uoff[nleaf], 1));
    std::vector<DevBuf<double>> Pi(L + 1);
    std::vector<std::vector<int64_t>> pioff(L + 1);
    {
        DevBuf<double> Wt((size_t)std::max<int64_t>(woff[nleaf], 1));
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int x = 0; x < nleaf; ++x) {
            const int rows = q * ng[L][x], m = bsize(L, x);
            for (int i = 0; i < ng[L][x]; ++i) {
                const G g = group(L, x, i);
                gb_.add(weight(g), q, 0, piece(g, bstart(L, x)), (int)N_, 1, Wt.p + woff[x] + (int64_t)i * q, rows, q, m, q,
                        1.0, 0.0);
            }
            if (rows) segs.push_back(RowSeg{Wt.p + woff[x], rows, rows});
            jobs.push_back(StackJob{(int)segs.size() - (rows ? 1 : 0), (int)segs.size(), m, Utmp.p + uoff[x], m, d_k.p + x,
                                    nullptr});
        }
        gb_.run(s_);
        stacked_svd_trunc(jobs, segs, stk_, tau_basis_, o_.kmax, d_cap.p, s_);
        std::vector<int> kk = read_ints(d_k.p, nleaf);
        for (int x = 0; x < nleaf; ++x) K(L, x) = kk[x];
        pioff[L].assign(nleaf + 1, 0);
        for (int x = 0; x < nleaf; ++x) pioff[L][x + 1] = pioff[L][x] + (int64_t)K(L, x) * q * ng[L][x];
        Pi[L].reserve((size_t)std::max<int64_t>(pioff[L][nleaf], 1));
        for (int x = 0; x < nleaf; ++x) {
            const int k = K(L, x);
            if (!k) continue;
            for (int i = 0; i < ng[L][x]; ++i)
                gb_.add(Utmp.p + uoff[x], bsize(L, x), 1, piece(group(L, x, i), bstart(L, x)), (int)N_, 0,
                        Pi[L].p + pioff[L][x] + (int64_t)i * k * q, k, k, q, bsize(L, x), 1.0, 0.0);
        }
        gb_.run(s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    }
    // upsweep: V_{y,i} = [Pi_{c1,i}; Pi_{c2,i}], SVD of the stacked R_i V_{y,i}^T, Pi_{y,i} = Ebar^T V_{y,i}
    const int nmax = 2 * o_.kmax;
    std::vector<int64_t> uhoff(h->koff[std::max(L, 1)], 0);
    for (size_t i = 0; i < uhoff.size(); ++i) uhoff[i] = (int64_t)i * nmax * nmax;
    DevBuf<double> Uh((size_t)std::max<int64_t>((int64_t)uhoff.size() * nmax * nmax, 1));
    for (int l = L - 1; l >= 1; --l) {
        const int nb = 1 << l;
        std::vector<int> nn(nb);
        std::vector<int64_t> voff(nb + 1, 0), wo(nb + 1, 0);
        for (int y = 0; y < nb; ++y) {
            nn[y] = K(l + 1, 2 * y) + K(l + 1, 2 * y + 1);
            voff[y + 1] = voff[y] + (int64_t)nn[y] * q * ng[l][y];
            wo[y + 1] = wo[y] + (int64_t)q * ng[l][y] * nn[y];
        }
        DevBuf<double> V((size_t)std::max<int64_t>(voff[nb], 1)), W((size_t)std::max<int64_t>(wo[nb], 1));
        std::vector<BlkDesc> d;
        for (int y = 0; y < nb; ++y) {
            if (!nn[y]) continue;
            for (int i = 0; i < ng[l][y]; ++i) {
                int row = 0;
                for (const int c : {2 * y, 2 * y + 1}) {
                    const int kc = K(l + 1, c);
                    if (kc)
                        d.push_back(BlkDesc{pioff[l + 1][c] + (int64_t)i * kc * q, voff[y] + (int64_t)i * nn[y] * q + row, kc, q,
                                            kc, nn[y]});
                    row += kc;
                }
            }
        }
        blocks(BLK_COPY, d, Pi[l + 1].p, V.p);
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        d_k.reserve(nb);
        for (int y = 0; y < nb; ++y) {
            const int rows = q * ng[l][y];
            const bool any = rows && nn[y];
            if (any) {
                for (int i = 0; i < ng[l][y]; ++i)
                    gb_.add(weight(group(l, y, i)), q, 0, V.p + voff[y] + (int64_t)i * nn[y] * q, nn[y], 1,
                            W.p + wo[y] + (int64_t)i * q, rows, q, nn[y], q, 1.0, 0.0);
                segs.push_back(RowSeg{W.p + wo[y], rows, rows});
            }
            jobs.push_back(StackJob{(int)segs.size() - (any ? 1 : 0), (int)segs.size(), nn[y], Uh.p + uhoff[h->koff[l] + y],
                                    std::max(nn[y], 1), d_k.p + y, nullptr});
        }
        gb_.run(s_);
        stacked_svd_trunc(jobs, segs, stk_, tau_basis_, o_.kmax, d_cap.p, s_);
        std::vector<int> kk = read_ints(d_k.p, nb);
        for (int y = 0; y < nb; ++y) K(l, y) = nn[y] ? kk[y] : 0;
        pioff[l].assign(nb + 1, 0);
        for (int y = 0; y < nb; ++y) pioff[l][y + 1] = pioff[l][y] + (int64_t)K(l, y) * q * ng[l][y];
        Pi[l].reserve((size_t)std::max<int64_t>(pioff[l][nb], 1));
        for (int y = 0; y < nb; ++y) {
            const int k = K(l, y);
            if (!k) continue;
            for (int i = 0; i < ng[l][y]; ++i)
                gb_.add(Uh.p + uhoff[h->koff[l] + y], nn[y], 1, V.p + voff[y] + (int64_t)i * nn[y] * q, nn[y], 0,
                        Pi[l].p + pioff[l][y] + (int64_t)i * k * q, k, k, q, nn[y], 1.0, 0.0);
        }
        gb_.run(s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    }
    // factors
    layout_factors(h);
    double* fac = h->fac64.p;
    std::vector<BlkDesc> d;
    for (int x = 0; x < nleaf; ++x)
        if (K(L, x)) d.push_back(BlkDesc{uoff[x], h->u_off[x], bsize(L, x), K(L, x), bsize(L, x), bsize(L, x)});
    blocks(BLK_COPY, d, Utmp.p, fac);
    d.clear();
    for (int l = 1; l < L; ++l)
        for (int y = 0; y < (1 << l); ++y) {
            const int n = K(l + 1, 2 * y) + K(l + 1, 2 * y + 1), k = K(l, y);
            if (n && k) d.push_back(BlkDesc{uhoff[h->koff[l] + y], h->uh_off[h->koff[l] + y], n, k, n, n});
        }
    blocks(BLK_COPY, d, Uh.p, fac);
    // couplings S_ts = Pi_{t,g} Pi_{s,g}^T of the pair g = (t, s)
    for (int l = 1; l <= L; ++l) {
        const ColorLevel& C = P_[l];
        for (size_t i = 0; i < h->far_lower[l].size(); ++i) {
            auto [t, s] = h->far_lower[l][i];
            const int kt = K(l, t), ks = K(l, s);
            if (!kt || !ks) continue;
            int p = -1;
            for (int x : C.by_t[t])
                if (C.pairs[x].second == s) p = x;
            if (p < 0) fail(H2_ERR_INVALID_ARG, "coloured assembly: far block without a sampled pair");
            const int it = ng[l - 1][t >> 1] + C.jq[p];
            const int is = ng[l - 1][s >> 1] + C.nq[s] + C.jz[p];
            gb_.add(Pi[l].p + pioff[l][t] + (int64_t)it * kt * q, kt, 0, Pi[l].p + pioff[l][s] + (int64_t)is * ks * q, ks, 1,
                    fac + h->s_off[l][i], kt, kt, ks, q, 1.0, 0.0);
        }
        gb_.run(s_);
    }
    d.clear();
    for (size_t i = 0; i < h->near_lower.size(); ++i) {
        auto [t, s] = h->near_lower[i];
        d.push_back(BlkDesc{dn_off_[i], h->d_off[i], bsize(L, t), bsize(L, s), bsize(L, t), bsize(L, t)});
    }
    blocks(BLK_COPY, d, Dn_.p, fac);
    int cap = 0;
    H2_CUDA(cudaMemcpyAsync(&cap, d_cap.p, sizeof(int), cudaMemcpyDeviceToHost, s_));
    H2_CUDA(cudaStreamSynchronize(s_));
    cap_hit_ = cap != 0;
}


void ColoredBuilder::run(h2_handle_s* h) {
    const double t0 = now_s();
    const int L = L_, nleaf = 1 << L;
    if (q_ < 1 || q_ > 16) fail(H2_ERR_INVALID_ARG, "coloured sampling: q0 must be in 1..16");
    if (2 * o_.kmax > svd_max_order()) fail(H2_ERR_INVALID_ARG, "coloured sampling: kmax above 48");
    if (T_.leaf_max > svd_max_order()) fail(H2_ERR_INVALID_ARG, "coloured sampling: leaf size above 96");
    {
        std::vector<int32_t> perm(N_), rl(N_);
        for (int64_t i = 0; i < N_; ++i) perm[i] = (int32_t)T_.perm[i];
        for (int t = 0; t < nleaf; ++t)
            for (int64_t i = 0; i < T_.size[L][t]; ++i) rl[T_.start[L][t] + i] = t;
        upload(d_perm_, perm, s_, stg_[0]);
        upload(d_row_leaf_, rl, s_, stg_[1]);
    }
    V_ = visited(T_);
    P_ = color_plan(T_, V_, q_);
    leaf_color_ = color_boxes(V_[L], std::vector<char>(nleaf, 1), &nleafcol_);
    int cmax = nleafcol_ * T_.leaf_max;
    for (int l = 1; l <= L; ++l) cmax = std::max({cmax, P_[l].ncolors * q_, P_[l].nslots * q_});
    Om_.reserve((size_t)N_ * cmax);
    Omt_.reserve((size_t)N_ * cmax);
    Yo_.reserve((size_t)N_ * cmax);
    Yt_.reserve((size_t)N_ * cmax);
    Q_.resize(L + 1);
    Z_.resize(L + 1);
    d_flag_.reserve(1);
    H2_CUDA(cudaMemsetAsync(d_flag_.p, 0, sizeof(int), s_));
    d_red_.reserve(4);
    const double tn = now_s();
    norm_ = o_.norm_est > 0.0 ? o_.norm_est : norm_estimate();
    const double tn1 = now_s();
    tau_basis_ = 2.0 * tol_ * norm_ / std::sqrt((double)nleaf);
    for (int l = 1; l <= L; ++l)
        if (!P_[l].pairs.empty()) sample_level(l);
    leaf_pass();
    Om_.release(); Omt_.release(); Yo_.release(); Yt_.release(); Sam_.release(); Ysc_.release();
    T1_.release(); T2_.release();
    const double tp = now_s();
    assemble(h);
    const double ta = now_s();
    h2_stats& st = h->stats;
    std::memset(&st, 0, sizeof(st));
    st.n = N_;
    st.levels = L;
    st.leaf_max = T_.leaf_max;
    st.samples = samples_;
    st.norm_products = norm_products_;
    st.op_calls = op_calls_;
    for (int l = 0; l <= L && l < H2_MAX_LEVELS; ++l) {
        st.range_probes[l] = P_[l].ncolors * q_;
        st.proj_probes[l] = P_[l].nslots * q_;
        st.range_calls[l] = P_[l].pairs.empty() ? 0 : 1;
        int mx = 0;
        for (int b = 0; b < (1 << l); ++b) mx = std::max(mx, h->k[h->koff[l] + b]);
        st.max_rank[l] = mx;
    }
    st.norm_est = norm_;
    st.tau_basis = tau_basis_;
    st.tol_met = cap_hit_ ? 0 : 1;
    st.t_total = ta - t0;
    st.t_norm = tn1 - tn;
    st.t_op = t_op_;
    st.t_peel = tp - tn1;
    st.t_assemble = ta - tp;
}

}  // namespace

int build_colored(h2_op_fn op, void* ctx, const h2_tree_s* tree, double tol, const h2_build_opts& o, h2_handle_s* h) {
    h->tree = std::make_shared<h2_tree_s>(*tree);
    h->L = tree->L;
    h->N = tree->N;
    ColoredBuilder b(*tree, op, ctx, tol, o);
    b.run(h);
    return h->stats.tol_met ? H2_OK : H2_WARN_TOL_NOT_MET;
}

// Colours and probe slots per level (the sampling plan alone, without products): for every level
// l, out[3 l] = colours of the range pass, out[3 l + 1] = slots of the projection pass, out[3 l + 2]
// = lower far pairs; out[3 (L + 1)] = leaf colours.
void colored_plan_counts(const h2_tree_s* tree, int q, int* out) {
    const auto V = visited(*tree);
    const auto P = color_plan(*tree, V, q);
    for (int l = 0; l <= tree->L; ++l) {
        out[3 * l] = P[l].ncolors;
        out[3 * l + 1] = P[l].nslots;
        out[3 * l + 2] = (int)P[l].pairs.size();
    }
    int nlc = 0;
    color_boxes(V[tree->L], std::vector<char>((size_t)1 << tree->L, 1), &nlc);
    out[3 * (tree->L + 1)] = nlc;
}

}  // namespace h2
