"""Low-rank update of an H^2 matrix with recompression (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Section 3.2 (Eqs. 3.3-3.4): adding a global low-rank term to an H^2 matrix
raises the rank of every block (the block (t, s) becomes a triple product in
the bases [U_t X_t] and [V_s Y_s]), and recompression finds new nested bases
of lower rank for the sum and projects it on them, so that the result stays
within the threshold to which the matrix itself is represented.  The paper
computes the new bases from R factors of the block rows (a QR downsweep) and
truncated SVDs (an upsweep); those R factors only compress the block rows,
whose left singular vectors and values they leave unchanged.  The oracle
therefore writes the result out by its definition, on the explicit updated
matrix A~ = A + B M B^T (symmetric; M = I is X Y^T with X = Y = B):

* the far block row of box t is A~ restricted to the rows of t and to the
  columns of every far block (t', s) of t and of its ancestors t';
* leaves: the new basis is the leading left singular vectors of the far block
  row with singular value > tau (at most kmax);
* upper levels: the same truncation of [U_c1^T F_p|c1 ; U_c2^T F_p|c2] (F_p the
  far block row of the parent, U_c the children's new explicit bases) gives the
  transfer matrices [E_c1; E_c2];
* couplings S_ts = U_t^T A~_ts U_s, dense blocks D_ts = A~_ts.

tau is the construction's basis threshold 2 tol ||A~||_2 / sqrt(#leaves), with
||A~||_2 given or estimated by the construction's power iteration on products
with A~.  Dense: for the small sizes of the tests only.
"""
from __future__ import annotations

import numpy as np

from .h2 import H2Matrix, _truncate, basis_threshold, expand_dense
from .peel import TreeOperator, norm2_estimate
from .tree import ClusterTree, Partition


def far_columns(tree: ClusterTree, part: Partition, l: int, t: int) -> np.ndarray:
    """Tree-order column indices of the far blocks of box t (level l) and of its ancestors."""
    cols = []
    for lv in range(l, 0, -1):
        tb = t >> (l - lv)
        for s in part.far_of[lv].get(tb, ()):
            r = tree.rows(lv, s)
            cols.append(np.arange(r.start, r.stop))
    return np.concatenate(cols) if cols else np.zeros(0, dtype=np.int64)


def compress_dense(tree: ClusterTree, part: Partition, At: np.ndarray, tau: float, kmax: int,
                   ranks=None) -> H2Matrix:
    """Nested-basis H^2 form of the symmetric dense matrix At (tree order) by truncated SVDs of the
    far block rows (leaves, then upsweep) and projection.  ranks (optional, per level a sequence of
    the rank of every box): keep exactly these ranks (replay of another implementation's rank
    decisions)."""
    L = tree.L
    h = H2Matrix(tree, part)
    for t in range(1 << L):
        rows = tree.rows(L, t)
        W = At[rows][:, far_columns(tree, part, L, t)]
        U, s, cap = _truncate(W, tau, kmax, None if ranks is None else int(ranks[L][t]))
        h.cap_hit |= cap
        h.sv[(L, t)] = s
        h.U[t] = U
        h.Uexp[L][t] = U
        h.k[L][t] = U.shape[1]
    for l in range(L - 1, 0, -1):
        for p in range(1 << l):
            c1, c2 = 2 * p, 2 * p + 1
            U1, U2 = h.Uexp[l + 1][c1], h.Uexp[l + 1][c2]
            r1, r2 = tree.rows(l + 1, c1), tree.rows(l + 1, c2)
            cols = far_columns(tree, part, l, p)
            W = np.vstack([U1.T @ At[r1][:, cols], U2.T @ At[r2][:, cols]])
            k1 = U1.shape[1]
            Uh, s, cap = _truncate(W, tau, kmax, None if ranks is None else int(ranks[l][p]))
            h.cap_hit |= cap
            h.sv[(l, p)] = s
            h.E[(l + 1, c1)] = Uh[:k1]
            h.E[(l + 1, c2)] = Uh[k1:]
            Ue = np.zeros((r1.stop - r1.start + r2.stop - r2.start, Uh.shape[1]))
            Ue[: r1.stop - r1.start] = U1 @ Uh[:k1]
            Ue[r1.stop - r1.start:] = U2 @ Uh[k1:]
            h.Uexp[l][p] = Ue
            h.k[l][p] = Uh.shape[1]
    h.Uexp[0][0] = np.zeros((tree.N, 0))
    for l in range(1, L + 1):
        for t, s in h.far_lower(l):
            rt, rs = tree.rows(l, t), tree.rows(l, s)
            h.S[(l, t, s)] = h.Uexp[l][t].T @ At[rt, rs] @ h.Uexp[l][s]
    for t, s in h.near_lower():
        h.D[(t, s)] = At[tree.rows(L, t), tree.rows(L, s)].copy()
    return h


def lowrank_update(h: H2Matrix, B: np.ndarray, tol: float, kmax: int, M=None, norm_est=None, seed: int = 7,
                   norm_maxit: int = 50, norm_rtol: float = 1e-3, ranks=None):
    """A~ = A + B M B^T (B: N x r in original order; M: r x r, its symmetric part is used, None:
    identity) recompressed to tol.  Returns (H2Matrix, norm estimate, tau)."""
    tree = h.tree
    B = np.asarray(B, dtype=np.float64).reshape(tree.N, -1)
    r = B.shape[1]
    M = np.eye(r) if M is None else 0.5 * (np.asarray(M, dtype=np.float64) + np.asarray(M, dtype=np.float64).T)
    A = expand_dense(h) + B @ M @ B.T
    if norm_est is None:
        norm_est, _ = norm2_estimate(TreeOperator(lambda X: A @ X, tree), tree.N, seed, norm_maxit, norm_rtol)
    tau = basis_threshold(tol, norm_est, 1 << tree.L)
    At = A[np.ix_(tree.perm, tree.perm)]
    return compress_dense(tree, h.part, At, tau, kmax, ranks=ranks), float(norm_est), tau
