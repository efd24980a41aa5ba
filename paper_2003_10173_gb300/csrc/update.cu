// Low-rank update of a built H^2 matrix followed by recompression (Section 3.2, Eqs. 3.3-3.4).
//
// The updated matrix is A~ = A + B M B^T (B: n x r, M: r x r symmetric; M = I gives the paper's
// X Y^T with X = Y = B, M = -I a downdate).  In the extended bases X_t = [U_t  B_t] every far block
// is X_t blkdiag(S_ts, M) X_s^T and every dense block D_ts + B_t M B_s^T, so the ranks grow by r;
// the extended bases stay nested: X_p restricted to its child c is X_c Phi_c, Phi_c =
// blkdiag(E_c, I_r).  Recompression finds new nested orthonormal bases from the far block rows of
// A~ and projects the couplings on them:
//   R_t  R factor of X_t: one QR per leaf, then an upsweep of QRs of [R_c1 Phi_c1; R_c2 Phi_c2];
//   T_t  R factor of G_t, the coefficients of the far block row of t in X_t (F_t = X_t G_t^T):
//        a downsweep of QRs of [T_p Phi_t^T; R_s blkdiag(S_ts, M)^T for every far block (t, s)];
//   leaves: the left singular vectors of X_t T_t^T above the basis threshold (F_t F_t^T =
//        X_t T_t^T T_t X_t^T), Pi_t = Ubar_t^T X_t;
//   upsweep: the left singular vectors of V_p T_p^T, V_p = [Pi_c1 Phi_c1; Pi_c2 Phi_c2], give the
//        transfer matrices, Pi_p = Ebar_p^T V_p;
//   couplings Pi_t blkdiag(S_ts, M) Pi_s^T; dense blocks D_ts + B_t M B_s^T.
// Only small dense blocks are factorised (the stacked QR and the Jacobi SVD kernels), level by
// level; the threshold is the construction's, 2 tol ||A~||_2 / sqrt(#leaves), with ||A~||_2 given
// or estimated by power iteration on products with A~.
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>

#include "handle.h"

namespace h2 {

void finish_handle(h2_handle_s* h, const h2_build_opts& o, cudaStream_t s);

namespace {

constexpr int STREAM_POWER = 2;   // start vector of the norm estimate (the construction's stream)

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

class Updater {
  public:
    Updater(h2_handle_s* A, const double* B, int64_t ldb, int r, const double* M, double tol, const h2_build_opts& o)
        : A_(A), T_(*A->tree), B_(B), ldb_(ldb), r_(r), tol_(tol), o_(o), s_((cudaStream_t)o.stream) {
        M_.assign((size_t)r * r, 0.0);
        // the symmetric part of M (the update of a symmetric matrix)
        for (int j = 0; j < r; ++j)
            for (int i = 0; i < r; ++i)
                M_[i + (size_t)j * r] = M ? 0.5 * (M[i + (size_t)j * r] + M[j + (size_t)i * r]) : (i == j ? 1.0 : 0.0);
    }
    void run(h2_handle_s* h);

  private:
    h2_handle_s* A_;
    const h2_tree_s& T_;
    const double* B_;
    int64_t ldb_;
    int r_;
    double tol_;
    h2_build_opts o_;
    cudaStream_t s_;
    std::vector<double> M_;
    GemmBatch gb_;
    StackWork stk_;
    Stager stg_[2];
    DevBuf<BlkDesc> d_blk_;
    DevBuf<double> Md_, BMo_, d_red_;
    Pinned pin_;
    double norm_ = 0.0;

    int K(int l, int b) const { return A_->k[A_->koff[l] + b]; }
    int C(int l, int b) const { return K(l, b) + r_; }
    int n(int l, int b) const { return (int)T_.size[l][b]; }
    int64_t start(int l, int b) const { return T_.start[l][b]; }
    const double* fac() const { return A_->fac64.p; }
    // transfer matrix E_c (k_c x k_parent) of box c at level l and its leading dimension
    const double* E(int l, int c, int* ld) const {
        const int p = c >> 1;
        *ld = K(l, 2 * p) + K(l, 2 * p + 1);
        return fac() + A_->uh_off[A_->koff[l - 1] + p] + ((c & 1) ? K(l, c - 1) : 0);
    }
    void blocks(int kind, const std::vector<BlkDesc>& d, const double* src, double* dst) {
        if (d.empty()) return;
        const std::vector<BlkDesc> ds = kind == BLK_COPY ? split_copies(d) : d;
        upload(d_blk_, ds, s_, stg_[0]);
        block_op(kind, (int)ds.size(), d_blk_.p, src, dst, s_);
    }
    std::vector<int> read_ints(const int* d, int count) {
        std::vector<int> v(count);
        if (!count) return v;
        int* hp = pin_.get<int>(count);
        H2_CUDA(cudaMemcpyAsync(hp, d, count * sizeof(int), cudaMemcpyDeviceToHost, s_));
        H2_CUDA(cudaStreamSynchronize(s_));
        std::memcpy(v.data(), hp, count * sizeof(int));
        return v;
    }
    double norm_estimate();
};

// ||A~||_2 by power iteration with the construction's start vector and stopping rule; one
// product is an H^2 matvec of A plus (B M) (B^T v).
double Updater::norm_estimate() {
    const int64_t N = T_.N;
    DevBuf<double> V((size_t)2 * N), u((size_t)std::max(r_, 1));
    double* v = V.p;
    double* w = V.p + N;
    d_red_.reserve(4);
    gaussian_vector(N, A_->d_perm.p, o_.seed, STREAM_POWER, v, s_);
    auto sqnorm = [&](const double* x) {
        col_sqnorms(N, 1, x, N, d_red_.p, s_);
        double* hp = pin_.get<double>(1);
        H2_CUDA(cudaMemcpyAsync(hp, d_red_.p, sizeof(double), cudaMemcpyDeviceToHost, s_));
        H2_CUDA(cudaStreamSynchronize(s_));
        return *hp;
    };
    auto scale = [&](double* x, double f) {
        double* hp = pin_.get<double>(1);
        *hp = f;
        H2_CUDA(cudaMemcpyAsync(d_red_.p + 1, hp, sizeof(double), cudaMemcpyHostToDevice, s_));
        scale_cols(N, 1, x, N, d_red_.p + 1, s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    };
    auto apply = [&](const double* x, double* y) {
        run_matvec(A_, x, N, y, N, 1, H2_FP64, s_);
        if (!r_) return;
        gb_.add(B_, (int)ldb_, 1, x, (int)N, 0, u.p, r_, r_, 1, (int)N, 1.0, 0.0);
        gb_.run(s_);
        gb_.add(BMo_.p, (int)N, 0, u.p, r_, 0, y, (int)N, (int)N, 1, r_, 1.0, 1.0);
        gb_.run(s_);
    };
    const double g = std::sqrt(sqnorm(v));
    if (!(g > 0.0)) fail(H2_ERR_CUDA, "power iteration: zero start vector");
    scale(v, 1.0 / g);
    double lam = 0.0, prev = 0.0;
    for (int it = 1; it <= o_.norm_maxit; ++it) {
        apply(v, w);
        lam = std::sqrt(sqnorm(w));
        if (!std::isfinite(lam)) fail(H2_ERR_NAN, "h2_lowrank_update: non-finite product");
        if (lam == 0.0) break;
        scale(w, 1.0 / lam);
        std::swap(v, w);
        if (it > 1 && std::fabs(lam - prev) <= o_.norm_rtol * lam) break;
        prev = lam;
    }
    return lam;
}

void Updater::run(h2_handle_s* h) {
    const double t0 = now_s();
    const int L = T_.L;
    const int64_t N = T_.N;
    const int nleaf = 1 << L;
    const int r = r_;
    int kold = 0;
    for (int k : A_->k) kold = std::max(kold, k);
    if (kold + r > stacked_r_max_columns())
        fail(H2_ERR_INVALID_ARG, "h2_lowrank_update: largest rank plus update rank above 144");
    if (2 * o_.kmax > svd_max_order()) fail(H2_ERR_INVALID_ARG, "h2_lowrank_update: kmax above 48");
    if (T_.leaf_max > svd_max_order()) fail(H2_ERR_INVALID_ARG, "h2_lowrank_update: leaf size above 96");

    // B in tree order, M on the device, B M in both orders
    DevBuf<double> Bt((size_t)std::max<int64_t>(N * r, 1)), BM((size_t)std::max<int64_t>(N * r, 1));
    Md_.reserve((size_t)std::max(r * r, 1));
    if (r) {
        H2_CUDA(cudaMemcpyAsync(Md_.p, M_.data(), M_.size() * sizeof(double), cudaMemcpyHostToDevice, s_));
        gather_rows(N, r, A_->d_perm.p, B_, ldb_, Bt.p, N, s_);
        gb_.add(Bt.p, (int)N, 0, Md_.p, r, 0, BM.p, (int)N, (int)N, r, r, 1.0, 0.0);
        BMo_.reserve((size_t)N * r);
        gb_.add(B_, (int)ldb_, 0, Md_.p, r, 0, BMo_.p, (int)N, (int)N, r, r, 1.0, 0.0);
        gb_.run(s_);
    }
    const double tn = now_s();
    norm_ = o_.norm_est > 0.0 ? o_.norm_est : norm_estimate();
    const double tn1 = now_s();
    const double tau = 2.0 * tol_ * norm_ / std::sqrt((double)nleaf);
    const int64_t nbox = A_->koff[L + 1];
    auto id = [&](int l, int b) { return A_->koff[l] + b; };

    // far blocks of every box (row box t -> column boxes s) and the stored coupling of each
    std::vector<std::vector<std::vector<int>>> own(L + 1);
    std::map<std::tuple<int, int, int>, int64_t> soff;   // (l, t, s), t > s -> offset of S_ts
    for (int l = 1; l <= L; ++l) {
        own[l].assign(1 << l, {});
        for (auto [t, s] : T_.far[l]) own[l][t].push_back(s);
        for (size_t i = 0; i < A_->far_lower[l].size(); ++i) {
            auto [t, s] = A_->far_lower[l][i];
            soff[{l, t, s}] = A_->s_off[l][i];
        }
    }
    // S_ts^T (k_s x k_t) as a GEMM operand: pointer, leading dimension, transpose flag
    auto st_op = [&](int l, int t, int s, int* ld, int* tr) -> const double* {
        if (t > s) {
            *ld = std::max(K(l, t), 1);
            *tr = 1;
            return fac() + soff.at({l, t, s});
        }
        *ld = std::max(K(l, s), 1);
        *tr = 0;
        return fac() + soff.at({l, s, t});
    };

    // ---- extended leaf bases X_t = [U_t B_t] and the R factors of all X_t (upsweep) ----
    std::vector<int64_t> xoff(nleaf + 1, 0);
    for (int t = 0; t < nleaf; ++t) xoff[t + 1] = xoff[t] + (int64_t)n(L, t) * C(L, t);
    DevBuf<double> Xw((size_t)std::max<int64_t>(xoff[nleaf], 1));
    {
        std::vector<BlkDesc> du, db;
        for (int t = 0; t < nleaf; ++t) {
            if (K(L, t)) du.push_back(BlkDesc{A_->u_off[t], xoff[t], n(L, t), K(L, t), n(L, t), n(L, t)});
            if (r) db.push_back(BlkDesc{start(L, t), xoff[t] + (int64_t)K(L, t) * n(L, t), n(L, t), r, (int)N, n(L, t)});
        }
        blocks(BLK_COPY, du, fac(), Xw.p);
        blocks(BLK_COPY, db, Bt.p, Xw.p);
    }
    std::vector<int64_t> ruoff(nbox, 0), toff(nbox, 0);
    std::vector<int> rrows(nbox, 0), trows(nbox, 0);
    int64_t rtot = 0;
    for (int l = 1; l <= L; ++l)
        for (int b = 0; b < (1 << l); ++b) {
            ruoff[id(l, b)] = rtot;
            toff[id(l, b)] = rtot;
            rtot += (int64_t)C(l, b) * C(l, b);
        }
    DevBuf<double> Ru((size_t)std::max<int64_t>(rtot, 1)), Tb((size_t)std::max<int64_t>(rtot, 1));
    fill_zero(Ru.p, Ru.n, s_);
    fill_zero(Tb.p, Tb.n, s_);
    if (L >= 1) {
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int t = 0; t < nleaf; ++t) {
            jobs.push_back(StackJob{(int)segs.size(), (int)segs.size() + 1, C(L, t), Ru.p + ruoff[id(L, t)], C(L, t),
                                    nullptr, nullptr});
            segs.push_back(RowSeg{Xw.p + xoff[t], n(L, t), n(L, t)});
            rrows[id(L, t)] = std::min(n(L, t), C(L, t));
        }
        stacked_r(jobs, segs, stk_, s_);
    }
    for (int l = L - 1; l >= 1; --l) {
        // [R_c1 Phi_c1; R_c2 Phi_c2] for every box p of level l
        std::vector<int64_t> zoff(1 << (l + 1), 0);
        int64_t zt = 0;
        for (int c = 0; c < (1 << (l + 1)); ++c) {
            zoff[c] = zt;
            zt += (int64_t)rrows[id(l + 1, c)] * C(l, c >> 1);
        }
        DevBuf<double> Zb((size_t)std::max<int64_t>(zt, 1));
        std::vector<BlkDesc> d;
        for (int c = 0; c < (1 << (l + 1)); ++c) {
            const int rr = rrows[id(l + 1, c)], p = c >> 1;
            if (!rr) continue;
            int lde;
            const double* Ec = E(l + 1, c, &lde);
            const double* Rc = Ru.p + ruoff[id(l + 1, c)];
            const int cc = C(l + 1, c);
            gb_.add(Rc, cc, 0, Ec, std::max(lde, 1), 0, Zb.p + zoff[c], rr, rr, K(l, p), K(l + 1, c), 1.0, 0.0);
            if (r) d.push_back(BlkDesc{ruoff[id(l + 1, c)] + (int64_t)K(l + 1, c) * cc, zoff[c] + (int64_t)K(l, p) * rr,
                                       rr, r, cc, rr});
        }
        gb_.run(s_);
        blocks(BLK_COPY, d, Ru.p, Zb.p);
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int p = 0; p < (1 << l); ++p) {
            StackJob jb{(int)segs.size(), 0, C(l, p), Ru.p + ruoff[id(l, p)], C(l, p), nullptr, nullptr};
            int rows = 0;
            for (const int c : {2 * p, 2 * p + 1}) {
                const int rr = rrows[id(l + 1, c)];
                if (!rr) continue;
                segs.push_back(RowSeg{Zb.p + zoff[c], rr, rr});
                rows += rr;
            }
            jb.seg_end = (int)segs.size();
            jobs.push_back(jb);
            rrows[id(l, p)] = std::min(C(l, p), rows);
        }
        stacked_r(jobs, segs, stk_, s_);
        H2_CUDA(cudaStreamSynchronize(s_));   // Zb is released at the end of the scope
    }

    // ---- far-row factors T_t (downsweep) ----
    for (int l = 1; l <= L; ++l) {
        std::vector<int64_t> yoff;
        std::vector<int> yrows;
        struct Src { int kind, t, s; };   // kind 0: from the parent, 1: own far block (t, s)
        std::vector<Src> src;
        std::vector<int> first(1 << l, 0);
        int64_t yt = 0;
        for (int t = 0; t < (1 << l); ++t) {
            first[t] = (int)src.size();
            const int ct = C(l, t);
            if (l >= 2 && trows[id(l - 1, t >> 1)]) {
                src.push_back(Src{0, t, -1});
                yoff.push_back(yt);
                yrows.push_back(trows[id(l - 1, t >> 1)]);
                yt += (int64_t)yrows.back() * ct;
            }
            for (int s : own[l][t]) {
                if (!rrows[id(l, s)]) continue;
                src.push_back(Src{1, t, s});
                yoff.push_back(yt);
                yrows.push_back(rrows[id(l, s)]);
                yt += (int64_t)yrows.back() * ct;
            }
        }
        first.push_back((int)src.size());
        DevBuf<double> Yb((size_t)std::max<int64_t>(yt, 1));
        std::vector<BlkDesc> dT;
        for (size_t i = 0; i < src.size(); ++i) {
            const Src& q = src[i];
            const int t = q.t, kt = K(l, t), rr = yrows[i];
            double* Y = Yb.p + yoff[i];
            if (q.kind == 0) {   // T_p Phi_t^T = [T_p[:, :k_p] E_t^T, T_p[:, k_p:]]
                const int p = t >> 1, cp = C(l - 1, p), kp = K(l - 1, p);
                int lde;
                const double* Et = E(l, t, &lde);
                const double* Tp = Tb.p + toff[id(l - 1, p)];
                gb_.add(Tp, cp, 0, Et, std::max(lde, 1), 1, Y, rr, rr, kt, kp, 1.0, 0.0);
                if (r) dT.push_back(BlkDesc{toff[id(l - 1, p)] + (int64_t)kp * cp, yoff[i] + (int64_t)kt * rr, rr, r, cp, rr});
            } else {             // R_s blkdiag(S_ts, M)^T = [R_s[:, :k_s] S_ts^T, R_s[:, k_s:] M]
                const int s = q.s, cs = C(l, s), ks = K(l, s);
                const double* Rs = Ru.p + ruoff[id(l, s)];
                int lds, trs;
                const double* St = st_op(l, t, s, &lds, &trs);
                gb_.add(Rs, cs, 0, St, lds, trs, Y, rr, rr, kt, ks, 1.0, 0.0);
                if (r) gb_.add(Rs + (int64_t)ks * cs, cs, 0, Md_.p, r, 0, Y + (int64_t)kt * rr, rr, rr, r, r, 1.0, 0.0);
            }
        }
        gb_.run(s_);
        blocks(BLK_COPY, dT, Tb.p, Yb.p);
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int t = 0; t < (1 << l); ++t) {
            if (first[t] == first[t + 1]) continue;
            StackJob jb{(int)segs.size(), 0, C(l, t), Tb.p + toff[id(l, t)], C(l, t), nullptr, nullptr};
            int rows = 0;
            for (int i = first[t]; i < first[t + 1]; ++i) {
                segs.push_back(RowSeg{Yb.p + yoff[i], yrows[i], yrows[i]});
                rows += yrows[i];
            }
            jb.seg_end = (int)segs.size();
            jobs.push_back(jb);
            trows[id(l, t)] = std::min(C(l, t), rows);
        }
        stacked_r(jobs, segs, stk_, s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    }

    // ---- new leaf bases: SVD of X_t T_t^T through its transpose T_t X_t^T ----
    h->tree = A_->tree;
    h->L = L;
    h->N = N;
    h->koff = A_->koff;
    h->k.assign((size_t)nbox, 0);
    auto Kn = [&](int l, int b) -> int& { return h->k[id(l, b)]; };
    DevBuf<int> d_k((size_t)nleaf), d_cap(1);
    H2_CUDA(cudaMemsetAsync(d_cap.p, 0, sizeof(int), s_));
    std::vector<int64_t> uoff(nleaf + 1, 0);
    for (int t = 0; t < nleaf; ++t) uoff[t + 1] = uoff[t] + (int64_t)n(L, t) * n(L, t);
    DevBuf<double> Utmp((size_t)std::max<int64_t>(uoff[nleaf], 1));
    std::vector<std::vector<int64_t>> pioff(L + 1);
    std::vector<DevBuf<double>> Pi(L + 1);
    if (L >= 1) {
        std::vector<int64_t> woff(nleaf + 1, 0);
        for (int t = 0; t < nleaf; ++t) woff[t + 1] = woff[t] + (int64_t)trows[id(L, t)] * n(L, t);
        DevBuf<double> Wt((size_t)std::max<int64_t>(woff[nleaf], 1));
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        for (int t = 0; t < nleaf; ++t) {
            const int rT = trows[id(L, t)];
            if (rT) {
                gb_.add(Tb.p + toff[id(L, t)], C(L, t), 0, Xw.p + xoff[t], n(L, t), 1, Wt.p + woff[t], rT, rT, n(L, t),
                        C(L, t), 1.0, 0.0);
                segs.push_back(RowSeg{Wt.p + woff[t], rT, rT});
            }
            jobs.push_back(StackJob{(int)segs.size() - (rT ? 1 : 0), (int)segs.size(), n(L, t), Utmp.p + uoff[t],
                                    n(L, t), d_k.p + t, nullptr});
        }
        gb_.run(s_);
        stacked_svd_trunc(jobs, segs, stk_, tau, o_.kmax, d_cap.p, s_);
        std::vector<int> kk = read_ints(d_k.p, nleaf);
        for (int t = 0; t < nleaf; ++t) Kn(L, t) = kk[t];
        // Pi_t = Ubar_t^T X_t (kbar_t x c_t)
        pioff[L].assign(nleaf + 1, 0);
        for (int t = 0; t < nleaf; ++t) pioff[L][t + 1] = pioff[L][t] + (int64_t)Kn(L, t) * C(L, t);
        Pi[L].reserve((size_t)std::max<int64_t>(pioff[L][nleaf], 1));
        for (int t = 0; t < nleaf; ++t)
            if (Kn(L, t))
                gb_.add(Utmp.p + uoff[t], n(L, t), 1, Xw.p + xoff[t], n(L, t), 0, Pi[L].p + pioff[L][t], Kn(L, t),
                        Kn(L, t), C(L, t), n(L, t), 1.0, 0.0);
        gb_.run(s_);
    }

    // ---- upsweep: transfer matrices from the SVD of V_p T_p^T ----
    const int nmax = 2 * o_.kmax;
    std::vector<int64_t> uhoff(nbox, 0);
    for (int64_t i = 0; i < nbox; ++i) uhoff[i] = i * (int64_t)nmax * nmax;
    DevBuf<double> Uh((size_t)std::max<int64_t>(A_->koff[std::max(L, 0)] * (int64_t)nmax * nmax, 1));
    for (int l = L - 1; l >= 1; --l) {
        const int nb = 1 << l;
        std::vector<int> nn(nb);
        std::vector<int64_t> voff(nb + 1, 0), woff(nb + 1, 0);
        for (int p = 0; p < nb; ++p) {
            nn[p] = Kn(l + 1, 2 * p) + Kn(l + 1, 2 * p + 1);
            voff[p + 1] = voff[p] + (int64_t)nn[p] * C(l, p);
            woff[p + 1] = woff[p] + (int64_t)trows[id(l, p)] * nn[p];
        }
        DevBuf<double> V((size_t)std::max<int64_t>(voff[nb], 1)), W((size_t)std::max<int64_t>(woff[nb], 1));
        std::vector<BlkDesc> d;
        for (int p = 0; p < nb; ++p) {
            int row = 0;
            for (const int c : {2 * p, 2 * p + 1}) {
                const int kb = Kn(l + 1, c), kc = K(l + 1, c), cc = C(l + 1, c);
                if (!kb) continue;
                int lde;
                const double* Ec = E(l + 1, c, &lde);
                const double* Pc = Pi[l + 1].p + pioff[l + 1][c];
                gb_.add(Pc, kb, 0, Ec, std::max(lde, 1), 0, V.p + voff[p] + row, nn[p], kb, K(l, p), kc, 1.0, 0.0);
                if (r) d.push_back(BlkDesc{pioff[l + 1][c] + (int64_t)kc * kb, voff[p] + row + (int64_t)K(l, p) * nn[p],
                                           kb, r, kb, nn[p]});
                (void)cc;
                row += kb;
            }
        }
        gb_.run(s_);
        blocks(BLK_COPY, d, Pi[l + 1].p, V.p);
        std::vector<StackJob> jobs;
        std::vector<RowSeg> segs;
        d_k.reserve(nb);
        for (int p = 0; p < nb; ++p) {
            const int rT = trows[id(l, p)];
            const bool any = rT && nn[p];
            if (any) {
                gb_.add(Tb.p + toff[id(l, p)], C(l, p), 0, V.p + voff[p], nn[p], 1, W.p + woff[p], rT, rT, nn[p],
                        C(l, p), 1.0, 0.0);
                segs.push_back(RowSeg{W.p + woff[p], rT, rT});
            }
            jobs.push_back(StackJob{(int)segs.size() - (any ? 1 : 0), (int)segs.size(), nn[p],
                                    Uh.p + uhoff[id(l, p)], std::max(nn[p], 1), d_k.p + p, nullptr});
        }
        gb_.run(s_);
        stacked_svd_trunc(jobs, segs, stk_, tau, o_.kmax, d_cap.p, s_);
        std::vector<int> kk = read_ints(d_k.p, nb);
        for (int p = 0; p < nb; ++p) Kn(l, p) = nn[p] ? kk[p] : 0;
        pioff[l].assign(nb + 1, 0);
        for (int p = 0; p < nb; ++p) pioff[l][p + 1] = pioff[l][p] + (int64_t)Kn(l, p) * C(l, p);
        Pi[l].reserve((size_t)std::max<int64_t>(pioff[l][nb], 1));
        for (int p = 0; p < nb; ++p)
            if (Kn(l, p))
                gb_.add(Uh.p + uhoff[id(l, p)], nn[p], 1, V.p + voff[p], nn[p], 0, Pi[l].p + pioff[l][p], Kn(l, p),
                        Kn(l, p), C(l, p), nn[p], 1.0, 0.0);
        gb_.run(s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    }

    // ---- the new factors ----
    layout_factors(h);
    double* nf = h->fac64.p;
    {
        std::vector<BlkDesc> d;
        for (int t = 0; t < nleaf; ++t)
            if (Kn(L, t)) d.push_back(BlkDesc{uoff[t], h->u_off[t], n(L, t), Kn(L, t), n(L, t), n(L, t)});
        blocks(BLK_COPY, d, Utmp.p, nf);
        d.clear();
        for (int l = 1; l < L; ++l)
            for (int p = 0; p < (1 << l); ++p) {
                const int nnp = Kn(l + 1, 2 * p) + Kn(l + 1, 2 * p + 1);
                if (nnp && Kn(l, p)) d.push_back(BlkDesc{uhoff[id(l, p)], h->uh_off[id(l, p)], nnp, Kn(l, p), nnp, nnp});
            }
        blocks(BLK_COPY, d, Uh.p, nf);
    }
    // couplings: Sbar_ts = [Pi_t[:, :k_t] S_ts, Pi_t[:, k_t:] M] Pi_s^T
    for (int l = 1; l <= L; ++l) {
        const auto& fl = h->far_lower[l];
        std::vector<int64_t> qoff(fl.size() + 1, 0);
        for (size_t i = 0; i < fl.size(); ++i)
            qoff[i + 1] = qoff[i] + (int64_t)Kn(l, fl[i].first) * C(l, fl[i].second);
        DevBuf<double> Q1((size_t)std::max<int64_t>(qoff[fl.size()], 1));
        for (size_t i = 0; i < fl.size(); ++i) {
            auto [t, s] = fl[i];
            const int kb = Kn(l, t);
            if (!kb || !Kn(l, s)) continue;
            const double* Pt = Pi[l].p + pioff[l][t];
            gb_.add(Pt, kb, 0, fac() + A_->s_off[l][i], std::max(K(l, t), 1), 0, Q1.p + qoff[i], kb, kb, K(l, s), K(l, t),
                    1.0, 0.0);
            if (r) gb_.add(Pt + (int64_t)K(l, t) * kb, kb, 0, Md_.p, r, 0, Q1.p + qoff[i] + (int64_t)K(l, s) * kb, kb, kb,
                           r, r, 1.0, 0.0);
        }
        gb_.run(s_);
        for (size_t i = 0; i < fl.size(); ++i) {
            auto [t, s] = fl[i];
            const int kb = Kn(l, t), ks = Kn(l, s);
            if (!kb || !ks) continue;
            gb_.add(Q1.p + qoff[i], kb, 0, Pi[l].p + pioff[l][s], ks, 1, nf + h->s_off[l][i], kb, kb, ks, C(l, s), 1.0,
                    0.0);
        }
        gb_.run(s_);
        H2_CUDA(cudaStreamSynchronize(s_));
    }
    // dense blocks: D_ts + (B M)_t B_s^T
    {
        std::vector<BlkDesc> d;
        for (size_t i = 0; i < h->near_lower.size(); ++i) {
            auto [t, s] = h->near_lower[i];
            d.push_back(BlkDesc{A_->d_off[i], h->d_off[i], n(L, t), n(L, s), n(L, t), n(L, t)});
        }
        blocks(BLK_COPY, d, fac(), nf);
        if (r) {
            for (size_t i = 0; i < h->near_lower.size(); ++i) {
                auto [t, s] = h->near_lower[i];
                gb_.add(BM.p + start(L, t), (int)N, 0, Bt.p + start(L, s), (int)N, 1, nf + h->d_off[i], n(L, t), n(L, t),
                        n(L, s), r, 1.0, 1.0);
            }
            gb_.run(s_);
        }
    }
    int cap = 0;
    H2_CUDA(cudaMemcpyAsync(&cap, d_cap.p, sizeof(int), cudaMemcpyDeviceToHost, s_));
    H2_CUDA(cudaStreamSynchronize(s_));
    const double t1 = now_s();

    h2_stats& st = h->stats;
    std::memset(&st, 0, sizeof(st));
    st.n = N;
    st.levels = L;
    st.leaf_max = T_.leaf_max;
    for (int l = 0; l <= L && l < H2_MAX_LEVELS; ++l) {
        int mx = 0;
        for (int b = 0; b < (1 << l); ++b) mx = std::max(mx, Kn(l, b));
        st.max_rank[l] = mx;
    }
    st.norm_est = norm_;
    st.tau_basis = tau;
    st.tol_met = cap ? 0 : 1;
    st.t_total = t1 - t0;
    st.t_norm = tn1 - tn;
    st.t_assemble = t1 - tn1;
}

}  // namespace

int update_handle(h2_handle_s* A, const double* B, int64_t ldb, int r, const double* M, double tol,
                  const h2_build_opts& o, h2_handle_s* h) {
    Updater u(A, B, ldb, r, M, tol, o);
    u.run(h);
    finish_handle(h, o, (cudaStream_t)o.stream);
    return h->stats.tol_met ? H2_OK : H2_WARN_TOL_NOT_MET;
}

}  // namespace h2
