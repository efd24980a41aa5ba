"""Planted test matrices with an exactly known hierarchical structure.

Each generator returns a dense symmetric matrix (original node order) whose
sampled sibling blocks and far block rows have exactly known, small ranks, so
that a correct construction must recover it to rounding error.  The
structures are assembled directly from random factors placed on the cluster
tree; they use only the tree and partition (pinned on their own) and no
construction code.
"""
import numpy as np

from oracle.tree import ClusterTree, Partition


def _orth(rng, m, k):
    q, _ = np.linalg.qr(rng.standard_normal((m, k)))
    return q[:, :k]


def to_original(tree: ClusterTree, A_tree: np.ndarray) -> np.ndarray:
    out = np.empty_like(A_tree)
    out[np.ix_(tree.perm, tree.perm)] = A_tree
    return out


def global_low_rank(N: int, r: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((N, r)) / np.sqrt(N)
    return B @ B.T


def block_diagonal(tree: ClusterTree, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    A = np.zeros((tree.N, tree.N))
    for t in range(1 << tree.L):
        r = tree.rows(tree.L, t)
        m = r.stop - r.start
        M = rng.standard_normal((m, m))
        A[r, r] = M + M.T
    return to_original(tree, A)


def nested_bases(tree: ClusterTree, k: int, seed: int):
    """Random orthonormal nested bases of rank k (rank min(k, |t|) at small boxes)."""
    rng = np.random.default_rng(seed)
    L = tree.L
    U = [dict() for _ in range(L + 1)]
    for t in range(1 << L):
        r = tree.rows(L, t)
        m = r.stop - r.start
        U[L][t] = _orth(rng, m, min(k, m))
    for l in range(L - 1, -1, -1):
        for t in range(1 << l):
            U1, U2 = U[l + 1][2 * t], U[l + 1][2 * t + 1]
            kk = min(k, U1.shape[1] + U2.shape[1])
            Eh = _orth(rng, U1.shape[1] + U2.shape[1], kk)
            top = U1 @ Eh[:U1.shape[1]]
            bot = U2 @ Eh[U1.shape[1]:]
            U[l][t] = np.vstack([top, bot])
    return U


def planted_h2(tree: ClusterTree, part: Partition, k: int, near_rank: int, seed: int, grade: float = 1.0) -> np.ndarray:
    """Symmetric H^2 matrix on the given partition: far blocks U_t S U_s^T with nested
    orthonormal bases of rank k; off-diagonal near blocks of rank near_rank; dense
    symmetric diagonal leaf blocks.  With grade < 1 the couplings are S = G_t M G_s with
    G = diag(grade^i): basis direction i of every box carries weight grade^i, so the far
    block rows have geometrically graded singular values."""
    rng = np.random.default_rng(seed + 1)
    U = nested_bases(tree, k, seed)
    L = tree.L
    A = np.zeros((tree.N, tree.N))
    for l, far in enumerate(part.far):
        for t, s in far:
            if t < s:
                continue
            S = rng.standard_normal((U[l][t].shape[1], U[l][s].shape[1]))
            S = (grade ** np.arange(S.shape[0]))[:, None] * S * (grade ** np.arange(S.shape[1]))[None, :]
            B = U[l][t] @ S @ U[l][s].T
            A[tree.rows(l, t), tree.rows(l, s)] = B
            A[tree.rows(l, s), tree.rows(l, t)] = B.T
    for t, s in part.near:
        if t < s:
            continue
        rt, rs = tree.rows(L, t), tree.rows(L, s)
        if t == s:
            M = rng.standard_normal((rt.stop - rt.start,) * 2)
            A[rt, rt] = M + M.T
        else:
            B = rng.standard_normal((rt.stop - rt.start, near_rank)) @ \
                rng.standard_normal((near_rank, rs.stop - rs.start)) / 4.0
            A[rt, rs] = B
            A[rs, rt] = B.T
    return to_original(tree, A)
