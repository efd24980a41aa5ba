"""H^2 destination assembly, nested bases, couplings, matvec and norms (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Representation (Section 3.1, Figure 1, Eq. (3.1)): A = D + U S U^T for a
symmetric matrix (the row basis tree equals the column basis tree).  Leaf
boxes hold explicit orthonormal bases U_t; every other box t with children
c1, c2 holds transfer matrices E_c1, E_c2 so that U_t = [U_c1 E_c1; U_c2 E_c2].
Every far (admissible) block (t, s) has a coupling S_ts (A_ts = U_t S_ts U_s^T)
and every near block a dense leaf block D_ts.  Only the lower triangle
(box index t > s within a level) and the diagonal are stored; the upper
blocks are their transposes.

Construction from the sampled pieces (Section 3.2, recompression):
* every destination block (t, s), t != s, lies inside exactly one sampled
  sibling block, the one of the level below the lowest common ancestor, so
  A_ts = P_lp[t] P_lp[s]^T for that pair level lp;
* the basis of box t must span the far block row of t and of all its
  ancestors restricted to t's rows.  Grouping the far blocks by pair level,
  the block row is  sum_lp P_lp[t] C_lp^T  with C_lp the stacked P_lp[s] of
  its columns; with C_lp = Q R_lp the block row has the same left singular
  vectors and values as the compact matrix [P_lp[t] R_lp^T]_lp (the
  "U_t R_t from a QR of the block row" of Section 3.2);
* leaves: U_t = leading left singular vectors with singular value > tau,
  at most kmax;  upper levels (upsweep): the same truncated SVD applied to
  [U_c1^T W|c1 ; U_c2^T W|c2] gives [E_c1; E_c2];
* couplings S_ts = (U_t^T P_lp[t]) (U_s^T P_lp[s])^T, near blocks
  D_ts = P_lp[t] P_lp[s]^T, diagonal leaf blocks from the leaf pass.
"""
from __future__ import annotations

import numpy as np

from .tree import ClusterTree, Partition


class H2Matrix:
    def __init__(self, tree: ClusterTree, part: Partition):
        self.tree, self.part = tree, part
        L = tree.L
        self.U = {}                 # leaf box -> explicit basis (|t| x k_t)
        self.E = {}                 # (level, box) -> transfer matrix (k_child x k_parent)
        self.k = [np.zeros(1 << l, dtype=np.int64) for l in range(L + 1)]
        self.Uexp = [dict() for _ in range(L + 1)]   # explicit bases for every box
        self.S = {}                 # (level, t, s) lower far blocks -> coupling
        self.D = {}                 # (t, s) lower near blocks and diagonal -> dense block
        self.sv = {}                # (level, box) -> singular values of the weighted block row
        self.cap_hit = False

    # ------------------------------------------------------------------
    def far_lower(self, level):
        f = self.part.far[level]
        return [(int(t), int(s)) for t, s in f if t > s]

    def near_lower(self):
        return [(int(t), int(s)) for t, s in self.part.near if t >= s]


def basis_threshold(tol: float, norm_est: float, n_leaves: int) -> float:
    """Absolute truncation threshold of the nested bases.

    Reading (the paper fixes only the overall target): the leaf block rows partition
    the rows, so independent per-row truncation errors add in quadrature in the
    2-norm; the bases are truncated at 2 tol ||H|| / sqrt(#leaves), which keeps the
    measured relative 2-norm error near 0.4 tol on the heat Hessians (n = 32..256)."""
    return 2.0 * tol * norm_est / (n_leaves ** 0.5)


def _truncate(W: np.ndarray, tau: float, kmax: int, k_given=None):
    """Leading left singular vectors of W with singular value > tau (at most kmax).  With
    k_given (rank replay) exactly that many are kept, whatever the threshold says."""
    if W.size == 0 or W.shape[1] == 0:
        if k_given:
            raise ValueError("rank replay asks for vectors of an empty block row")
        return np.zeros((W.shape[0], 0)), np.zeros(0), False
    U, s, _ = np.linalg.svd(W, full_matrices=False)
    if k_given is not None:
        if k_given > U.shape[1]:
            raise ValueError("rank replay asks for more vectors than the block row has")
        return U[:, :k_given], s, False
    k = int(np.sum(s > tau))
    cap = k > kmax
    k = min(k, kmax)
    return U[:, :k], s, cap


def block_row_weights(tree: ClusterTree, part: Partition, pieces):
    """R_lp factors of every box's far block row (QR downsweep of Section 3.2).

    The far block row of box t (far blocks of t and of all its ancestors, restricted
    to the rows of t) is, grouped by pair level lp, sum_lp P_lp[t] C_lp(t)^T with
    C_lp(t) the stacked P_lp[s] of its column boxes.  R_lp(t) is the R factor of a QR
    of C_lp(t); it follows from the parent's by one QR of
    [R_lp(parent); P_lp[s] for the far blocks (t, s) of t itself with pair level lp]."""
    L = tree.L
    R = [dict() for _ in range(L + 1)]
    R[0][0] = {}                      # the root has no far blocks
    for l in range(1, L + 1):
        for t in range(1 << l):
            groups = {lp: [Rp] for lp, Rp in R[l - 1].get(t >> 1, {}).items()}
            for s in part.far_of[l].get(t, ()):
                lp = Partition.pair_level(l, t, s)
                for g in (lp, 0) if 0 in pieces else (lp,):   # the global piece covers every block
                    if pieces[g].shape[1]:
                        groups.setdefault(g, []).append(pieces[g][tree.rows(l, s)])
            R[l][t] = {lp: np.linalg.qr(np.vstack(b), mode="r") for lp, b in sorted(groups.items())}
    return R


def assemble(tree: ClusterTree, part: Partition, peel_res, tau: float, kmax: int, ranks=None) -> H2Matrix:
    """Destination assembly, nested bases, couplings and dense blocks from the pieces.

    ranks (rank replay, optional): per level l a sequence of the basis rank of every box of
    that level; the truncations keep exactly these ranks instead of deciding by tau.  The
    ranks of another implementation can be replayed this way, so that two constructions
    that agree on every rank decision can be compared to rounding error."""
    L = tree.L
    P = peel_res.pieces
    h = H2Matrix(tree, part)
    # weights of every box's far block row
    R = block_row_weights(tree, part, P)
    # leaves
    for t in range(1 << L):
        rows = tree.rows(L, t)
        cols = [P[lp][rows] @ Rl.T for lp, Rl in R[L][t].items()]
        W = np.hstack(cols) if cols else np.zeros((rows.stop - rows.start, 0))
        U, s, cap = _truncate(W, tau, kmax, None if ranks is None else int(ranks[L][t]))
        h.cap_hit |= cap
        h.sv[(L, t)] = s
        h.U[t] = U
        h.Uexp[L][t] = U
        h.k[L][t] = U.shape[1]
    # upsweep
    for l in range(L - 1, 0, -1):
        for t in range(1 << l):
            c1, c2 = 2 * t, 2 * t + 1
            U1, U2 = h.Uexp[l + 1][c1], h.Uexp[l + 1][c2]
            r1, r2 = tree.rows(l + 1, c1), tree.rows(l + 1, c2)
            top, bot = [], []
            for lp, Rl in R[l][t].items():
                top.append(U1.T @ P[lp][r1] @ Rl.T)
                bot.append(U2.T @ P[lp][r2] @ Rl.T)
            k1, k2 = U1.shape[1], U2.shape[1]
            if top:
                W = np.vstack([np.hstack(top), np.hstack(bot)])
            else:
                W = np.zeros((k1 + k2, 0))
            Uh, s, cap = _truncate(W, tau, kmax, None if ranks is None else int(ranks[l][t]))
            h.cap_hit |= cap
            h.sv[(l, t)] = s
            h.E[(l + 1, c1)] = Uh[:k1]
            h.E[(l + 1, c2)] = Uh[k1:]
            Ue = np.zeros((r1.stop - r1.start + r2.stop - r2.start, Uh.shape[1]))
            Ue[: r1.stop - r1.start] = U1 @ Uh[:k1]
            Ue[r1.stop - r1.start:] = U2 @ Uh[k1:]
            h.Uexp[l][t] = Ue
            h.k[l][t] = Uh.shape[1]
    h.Uexp[0][0] = np.zeros((tree.N, 0))
    # couplings of the lower far blocks
    for l in range(1, L + 1):
        for t, s in h.far_lower(l):
            lps = [Partition.pair_level(l, t, s)] + ([0] if 0 in P else [])
            S = np.zeros((int(h.k[l][t]), int(h.k[l][s])))
            for lp in lps:
                Pt = P[lp][tree.rows(l, t)]
                Ps = P[lp][tree.rows(l, s)]
                S += (h.Uexp[l][t].T @ Pt) @ (h.Uexp[l][s].T @ Ps).T
            h.S[(l, t, s)] = S
    # dense near blocks
    for t, s in h.near_lower():
        if t == s:
            h.D[(t, s)] = peel_res.D_diag[t].copy()
        else:
            lp = Partition.pair_level(L, t, s)
            D = P[lp][tree.rows(L, t)] @ P[lp][tree.rows(L, s)].T
            if 0 in P:
                D = D + P[0][tree.rows(L, t)] @ P[0][tree.rows(L, s)].T
            h.D[(t, s)] = D
    return h


# ----------------------------------------------------------------------
# Operations on the H^2 matrix
# ----------------------------------------------------------------------

def matvec(h: H2Matrix, X: np.ndarray) -> np.ndarray:
    """Y = A X in original node order by the four stages of Section 3.2, Eq. (3.2):
    dense blocks D X, upsweep of the basis tree (leaf bases then transfer matrices),
    couplings per level, downsweep (transfer matrices then leaf bases)."""
    tree = h.tree
    L = tree.L
    vec = X.ndim == 1
    if vec:
        X = X[:, None]
    Xt = np.asarray(X, dtype=np.float64)[tree.perm]
    Yt = np.zeros_like(Xt)
    # near field
    for (t, s), D in h.D.items():
        rt, rs = tree.rows(L, t), tree.rows(L, s)
        Yt[rt] += D @ Xt[rs]
        if t != s:
            Yt[rs] += D.T @ Xt[rt]
    if L >= 1:
        # upsweep
        xh = [dict() for _ in range(L + 1)]
        for t in range(1 << L):
            xh[L][t] = h.U[t].T @ Xt[tree.rows(L, t)]
        for l in range(L - 1, 0, -1):
            for t in range(1 << l):
                c1, c2 = 2 * t, 2 * t + 1
                xh[l][t] = h.E[(l + 1, c1)].T @ xh[l + 1][c1] + h.E[(l + 1, c2)].T @ xh[l + 1][c2]
        # couplings
        yh = [{t: np.zeros((int(h.k[l][t]), Xt.shape[1])) for t in range(1 << l)} for l in range(L + 1)]
        for (l, t, s), S in h.S.items():
            yh[l][t] += S @ xh[l][s]
            yh[l][s] += S.T @ xh[l][t]
        # downsweep
        for l in range(1, L):
            for t in range(1 << l):
                c1, c2 = 2 * t, 2 * t + 1
                yh[l + 1][c1] += h.E[(l + 1, c1)] @ yh[l][t]
                yh[l + 1][c2] += h.E[(l + 1, c2)] @ yh[l][t]
        for t in range(1 << L):
            Yt[tree.rows(L, t)] += h.U[t] @ yh[L][t]
    Y = np.empty_like(Yt)
    Y[tree.perm] = Yt
    return Y[:, 0] if vec else Y


def expand_dense(h: H2Matrix) -> np.ndarray:
    """Explicit N x N matrix (original order) from explicit bases (small N only)."""
    tree = h.tree
    L = tree.L
    A = np.zeros((tree.N, tree.N))
    for (t, s), D in h.D.items():
        rt, rs = tree.rows(L, t), tree.rows(L, s)
        A[rt, rs] = D
        if t != s:
            A[rs, rt] = D.T
    for (l, t, s), S in h.S.items():
        rt, rs = tree.rows(l, t), tree.rows(l, s)
        B = h.Uexp[l][t] @ S @ h.Uexp[l][s].T
        A[rt, rs] = B
        A[rs, rt] = B.T
    out = np.empty_like(A)
    out[np.ix_(tree.perm, tree.perm)] = A
    return out


def frobenius_norm(h: H2Matrix) -> float:
    """||A||_F from the stored data (Section 3.2): with orthonormal bases
    ||U_t S U_s^T||_F = ||S||_F, so ||A||_F^2 = sum over both triangles of ||S||_F^2 + ||D||_F^2."""
    tot = 0.0
    for (_, t, s), S in h.S.items():
        tot += 2.0 * float(np.sum(S * S))
    for (t, s), D in h.D.items():
        tot += (1.0 if t == s else 2.0) * float(np.sum(D * D))
    return float(np.sqrt(tot))


def storage_entries(h: H2Matrix) -> dict:
    """Stored floating-point entries per component (lower-triangle storage)."""
    L = h.tree.L
    return {
        "D": int(sum(D.size for D in h.D.values())),
        "S": int(sum(S.size for S in h.S.values())),
        "U": int(sum(U.size for U in h.U.values())),
        "E": int(sum(E.size for E in h.E.values())),
    }


def factor_arrays(h: H2Matrix):
    """The factors in the flat layout of the library's import/export calls: ranks of every box
    (levels 0..L, 2^l boxes each); leaf bases |t| x k_t; transfer matrices k_c x k_parent of
    every box c of levels 2..L (level-1 boxes have none: the root's rank is 0); couplings of
    the lower far blocks per level in partition order; near blocks with t >= s in partition
    order; all column-major FP64."""
    tree, part = h.tree, h.part
    L = tree.L
    ranks = np.concatenate([np.asarray(h.k[l], dtype=np.int32) for l in range(L + 1)])
    U = [h.U[t].flatten(order="F") for t in range(1 << L)]
    E = [h.E[(l, c)].flatten(order="F") for l in range(2, L + 1) for c in range(1 << l)]
    S = [h.S[(l, int(t), int(s))].flatten(order="F") for l in range(1, L + 1) for t, s in part.far[l] if t > s]
    D = [h.D[(int(t), int(s))].flatten(order="F") for t, s in part.near if t >= s]
    cat = lambda xs: np.concatenate(xs) if xs else np.zeros(0)
    return ranks, cat(U), cat(E), cat(S), cat(D)


def from_factor_arrays(tree: ClusterTree, part: Partition, ranks, U, E, S, D) -> H2Matrix:
    """An H2Matrix holding given factors in the layout of factor_arrays."""
    L = tree.L
    h = H2Matrix(tree, part)
    o = 0
    for l in range(L + 1):
        h.k[l] = np.asarray(ranks[o:o + (1 << l)], dtype=np.int64)
        o += 1 << l
    o = 0
    for t in range(1 << L):
        r = tree.rows(L, t)
        m, k = r.stop - r.start, int(h.k[L][t])
        h.U[t] = np.asarray(U[o:o + m * k]).reshape((m, k), order="F")
        h.Uexp[L][t] = h.U[t]
        o += m * k
    o = 0
    for l in range(2, L + 1):
        for c in range(1 << l):
            kc, kp = int(h.k[l][c]), int(h.k[l - 1][c >> 1])
            h.E[(l, c)] = np.asarray(E[o:o + kc * kp]).reshape((kc, kp), order="F")
            o += kc * kp
    for l in range(1, L + 1):
        for c in range(1 << l):
            if (l, c) not in h.E:
                h.E[(l, c)] = np.zeros((int(h.k[l][c]), int(h.k[l - 1][c >> 1])))
    for l in range(L - 1, 0, -1):
        for t in range(1 << l):
            h.Uexp[l][t] = np.vstack([h.Uexp[l + 1][2 * t] @ h.E[(l + 1, 2 * t)],
                                      h.Uexp[l + 1][2 * t + 1] @ h.E[(l + 1, 2 * t + 1)]])
    h.Uexp[0][0] = np.zeros((tree.N, 0))
    o = 0
    for l in range(1, L + 1):
        for t, s in part.far[l]:
            if t > s:
                kt, ks = int(h.k[l][t]), int(h.k[l][s])
                h.S[(l, int(t), int(s))] = np.asarray(S[o:o + kt * ks]).reshape((kt, ks), order="F")
                o += kt * ks
    o = 0
    for t, s in part.near:
        if t >= s:
            rt, rs = tree.rows(L, t), tree.rows(L, s)
            mt, ms = rt.stop - rt.start, rs.stop - rs.start
            h.D[(int(t), int(s))] = np.asarray(D[o:o + mt * ms]).reshape((mt, ms), order="F")
            o += mt * ms
    return h


def power_norm(apply, N: int, v0: np.ndarray, maxit: int = 200, rtol: float = 1e-2):
    """2-norm of a symmetric operator by power iteration, stopping once two significant
    digits are stable (Section 3.2)."""
    v = v0 / np.linalg.norm(v0)
    lam_prev = 0.0
    lam = 0.0
    for it in range(1, maxit + 1):
        w = apply(v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            return 0.0
        v = w / lam
        if it > 1 and abs(lam - lam_prev) <= rtol * lam:
            break
        lam_prev = lam
    return lam
