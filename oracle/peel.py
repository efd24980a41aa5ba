"""Randomized peeling construction from Hessian-vector products (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

Follows Section 3.3 (Figure 2) with the weak-admissibility sampling structure
the paper's implementation uses:

* Levels are processed coarse to fine.  At level l the sampled blocks are the
  off-diagonal sibling blocks H[b, a] of every pair (a, b) = (child 0,
  child 1) of a level-(l-1) box.  One probe block serves all pairs of a level
  at once: Gaussian on the rows of every child-0 box, zero elsewhere.
* The blocks of coarser levels already sampled are removed from the samples
  (Y = H Omega - K Omega, K = sum of the coarser pieces), so that
  Y[b] = H[b, a] Omega[a].
* A QR factorisation of Y[b] gives the column basis Q_b; the product of the
  matrix with [0; Q_b] (the projection pass, Psi) gives the row factor
  Z[a] = H[a, b] Q_b, and the piece H[b, a] ~ Q_b Z[a]^T is stored as a local
  low-rank update.  Sampling is repeated until the approximation of every
  sampled block meets the threshold: adaptive probes, grown by b_inc columns
  until the new columns' residuals (I - Q Q^T) y are all below
  tau / (10 sqrt(2/pi)) (the a-posteriori range test of the randomized
  range finder, halko11, cited in Section 3.3).
* Certified basis (option `certified`): the test columns of the test that passes
  are not added to Q_b.  The passing test certifies the basis it was run against
  (the adaptive range finder in its textbook form, halko11 Algorithm 4.2: test
  vectors join the basis only while the test fails), so the projection pass and
  every later step use that basis; with certified=False (the default) Q_b spans
  every range probe drawn, the passing test columns included.
* If a level's boxes are no larger than the probe count, the range of H[b, a]
  is the whole of R^|b| and Q_b = I (no range pass is spent).
* Finally identity probes on every leaf give the dense diagonal leaf blocks,
  after removing all sampled pieces; they are symmetrised.
* Predicted start counts (the learned-rank path): with q_level[l] given, level l
  starts from q_level[l] probes instead of q0 (identity when q_level[l] >= the
  largest child-1 box) and the first a-posteriori test uses q_test columns;
  when that test fails, growth by b_inc resumes as above, so the prediction
  only changes where the adaptive finder starts (Section 3.3: the per-level
  sample count C_l k is the quantity being tuned).
* The first test batch is drawn in the same operator call as the start block
  (the probes are indexed by column, so this changes the number of calls, not
  the arithmetic).

Pieces of level l are stored in one N x q_l array P_l (tree order): rows of
child-1 boxes hold Q_b, rows of child-0 boxes hold Z[a], so that for every
pair H[b, a] ~ P_l[b] P_l[a]^T and H[a, b] ~ P_l[a] P_l[b]^T.

Global low rank first (Section 3.3, end; the hybrid construction): with a
global rank budget r_max > 0, a randomized range finder on the whole matrix
(probes Gaussian on every row, from the `global` stream; start q0, growth b_inc
up to r_max, the same a-posteriori test and fused first test batch as the
levels) gives an orthonormal Q; one more product gives M = Q^T H Q
(symmetrised), and its semidefinite Cholesky factor C (C C^T = M) gives
B = Q C, so that B B^T = Q Q^T H Q Q^T.  B is stored as the level-0 piece
P_0: every block of B B^T is P_0[t] P_0[s]^T, including the diagonal blocks,
so it is removed from every later sample together with the level pieces
(the levels then sample the residual H - B B^T) and added back in the
assembly, where it joins the block rows of every box as one more group
(the low-rank update followed by recompression of Section 3.2).  When the
global range test passes within the budget, the global approximation already
meets the target and the residual is not sampled at all: every level piece is
empty (passed = 2) and the diagonal leaf blocks are those of B B^T.
"""
from __future__ import annotations

import math

import numpy as np

from . import rng
from .tree import ClusterTree


class TreeOperator:
    """Wraps an operator acting in original node order so that it acts in tree order."""

    def __init__(self, op, tree: ClusterTree):
        self.op, self.tree = op, tree
        self.samples = 0

    def __call__(self, Om_tree: np.ndarray) -> np.ndarray:
        perm = self.tree.perm
        X = np.zeros_like(Om_tree)
        X[perm] = Om_tree
        self.samples += Om_tree.shape[1]
        return np.asarray(self.op(X))[perm]


def norm2_estimate(opt: TreeOperator, N: int, seed: int, maxit: int = 50, rtol: float = 1e-3):
    """2-norm of the symmetric PSD operator by power iteration (Section 3.2: p-norms by
    matrix-vector products).  Start vector: Gaussian from the `power` stream.  Stops when
    the estimate changes by at most rtol relative, or after maxit products."""
    v = rng.gaussian_block(seed, rng.STREAM_POWER, 0, N, 0, 1)
    v /= np.linalg.norm(v)
    lam_prev = 0.0
    lam = 0.0
    it = 0
    for it in range(1, maxit + 1):
        w = opt(v)
        lam = float(np.linalg.norm(w))
        if lam == 0.0:
            break
        v = w / lam
        if it > 1 and abs(lam - lam_prev) <= rtol * lam:
            break
        lam_prev = lam
    return lam, it


def apply_pieces(pieces, levels, tree: ClusterTree, Om: np.ndarray) -> np.ndarray:
    """K Om for K = sum over the given levels of the sampled sibling pieces (flat low rank);
    level 0 is the global piece B, whose block pattern is the whole matrix: K += B B^T."""
    out = np.zeros_like(Om)
    for l in levels:
        if l not in pieces:
            continue
        P = pieces[l]
        if l == 0:
            out += P @ (P.T @ Om)
            continue
        for i in range(1 << (l - 1)):
            a, b = tree.rows(l, 2 * i), tree.rows(l, 2 * i + 1)
            out[b] += P[b] @ (P[a].T @ Om[a])
            out[a] += P[a] @ (P[b].T @ Om[b])
    return out


def range_basis(Y: np.ndarray) -> np.ndarray:
    """Orthonormal column basis of a sample block (Section 3.3: "a QR factorization of
    (A Omega)_1 gives the orthogonal columns basis U").  Reading: the basis is the Q factor of
    the thin QR with a non-negative diagonal of R, the unique one when Y has full column rank,
    so that the basis -- not only its span -- is fixed by the samples (the projection pass
    applies all blocks' bases at once, and the coarse levels' residual couples them); once
    the samples have at least as many columns as rows, the range is all of R^m and U = I."""
    m, q = Y.shape
    if q >= m:
        return np.eye(m)
    Q, R = np.linalg.qr(Y)
    sgn = np.where(np.diag(R) < 0.0, -1.0, 1.0)
    return Q * sgn


def psd_cholesky(M: np.ndarray) -> np.ndarray:
    """Lower-triangular C with C C^T = M for a symmetric positive semidefinite M (right-looking
    Cholesky).  A pivot at or below n * 2^-52 * max(diag M) is rounding noise of a zero
    eigenvalue: its column of C is left zero and the elimination continues."""
    n = M.shape[0]
    A = np.array(M, dtype=np.float64)
    C = np.zeros_like(A)
    if n == 0:
        return C
    drop = n * 2.0 ** -52 * max(float(np.max(np.diag(A))), 0.0)
    for j in range(n):
        d = A[j, j]
        if d <= drop:
            continue
        C[j, j] = math.sqrt(d)
        C[j + 1:, j] = A[j + 1:, j] / C[j, j]
        A[j + 1:, j + 1:] -= np.outer(C[j + 1:, j], C[j + 1:, j])
    return C


def global_lowrank(opt, N: int, thr: float, q0: int, b_inc: int, r_max: int, adaptive: bool, seed: int, res):
    """The global piece B (N x r, tree order), B B^T = Q Q^T H Q Q^T (Section 3.3, end)."""
    def probe(col0, ncols):
        return opt(rng.gaussian_block(seed, rng.STREAM_GLOBAL, 0, N, col0, ncols))

    q = min(q0, r_max, N)
    c1 = min(b_inc, r_max - q) if (adaptive and q < r_max and q < N) else 0
    Y = probe(0, q + c1)
    calls = 1
    pending = Y[:, q:] if c1 else None
    Ys = Y[:, :q]
    Q = np.linalg.qr(Ys)[0]
    passed = 0
    errs = []
    while adaptive and q < r_max and q < N:
        c = min(b_inc, r_max - q)
        if pending is not None:
            Yn, pending = pending, None
        else:
            Yn = probe(q, c)
            calls += 1
        r = Yn - Q @ (Q.T @ Yn)
        err = float(np.linalg.norm(r, axis=0).max())
        errs.append(err)
        Ys = np.hstack([Ys, Yn])
        Q = np.linalg.qr(Ys)[0]
        q += c
        if err <= thr:
            passed = 1
            break
    Z = opt(Q)
    M = Q.T @ Z
    M = 0.5 * (M + M.T)
    B = Q @ psd_cholesky(M)
    res.global_rank = q
    res.global_calls = calls
    res.global_passed = passed
    res.global_test_err = errs
    return B


class PeelResult:
    def __init__(self):
        self.pieces = {}          # level -> N x q_l array (tree order)
        self.rank = {}            # level -> per-pair number of columns of Q_b
        self.range_probes = {}    # level -> range-pass probes spent
        self.proj_probes = {}     # level -> projection-pass probes spent
        self.test_err = {}        # level -> list of max residual per pair of each adaptive test
        self.range_calls = {}     # level -> operator calls of the range pass
        self.passed = {}          # level -> 1 test passed, 0 no test passed, -1 identity range
        self.need = {}            # level -> probes of the range basis that passed the test
        self.D_diag = []          # dense leaf diagonal blocks, per leaf
        self.samples = 0
        self.norm_est = 0.0
        self.norm_its = 0
        self.tau = 0.0
        self.global_rank = 0      # columns of the global range basis (0: no global piece)
        self.global_calls = 0     # operator calls of its range finder
        self.global_passed = 0    # 1: its a-posteriori test passed within the budget
        self.global_test_err = []


def peel(op, tree: ClusterTree, tol: float, q0: int, b_inc: int, q_max: int, adaptive: bool,
         seed: int, norm_est: float | None = None, q_level=None, q_test: int = 8,
         global_rank: int = 0, q_exact=None, certified: bool = False) -> PeelResult:
    """Construct the sibling pieces and the leaf diagonal blocks from products with op.

    q_level: optional sequence indexed by level (entries <= 0 mean q0) of start counts.
    global_rank: budget of the global low-rank piece (0: none).
    q_exact (replay of another run's decisions): sequence indexed by level; level l draws
    exactly q_exact[l] range probes without any test, and takes the identity range when
    q_exact[l] == 0.  Overrides q0, q_level and adaptive.
    certified: the passing test's columns stay out of the basis (see the module notes)."""
    N = tree.N
    opt = TreeOperator(op, tree)
    res = PeelResult()
    if norm_est is None:
        res.norm_est, res.norm_its = norm2_estimate(opt, N, seed)
    else:
        res.norm_est, res.norm_its = float(norm_est), 0
    tau = tol * res.norm_est
    res.tau = tau
    thr = tau / (10.0 * math.sqrt(2.0 / math.pi))
    if global_rank > 0 and tree.L >= 1:   # a single leaf is one dense block: nothing to split off
        res.pieces[0] = global_lowrank(opt, N, thr, q0, b_inc, global_rank, adaptive, seed, res)

    covered = global_rank > 0 and res.global_passed == 1
    for l in range(1, tree.L + 1):
        npairs = 1 << (l - 1)
        if covered:
            res.pieces[l] = np.zeros((N, 0))
            res.rank[l] = [0] * npairs
            res.range_probes[l] = res.proj_probes[l] = res.range_calls[l] = res.need[l] = 0
            res.passed[l] = 2
            res.test_err[l] = []
            continue
        A = [tree.rows(l, 2 * i) for i in range(npairs)]
        B = [tree.rows(l, 2 * i + 1) for i in range(npairs)]
        mb = max(b.stop - b.start for b in B)
        below = range(0, l)
        Qs = []
        res.test_err[l] = []
        ql = q0
        predicted = q_level is not None and l < len(q_level) and q_level[l] > 0
        if predicted:
            ql = int(q_level[l])
        if q_exact is not None:
            ql = int(q_exact[l])
            adaptive = False
        res.range_calls[l] = 0
        res.passed[l] = 0
        if (ql >= mb and q_exact is None) or (q_exact is not None and ql == 0):
            # the range of H[b, a] is all of R^|b|
            for b in B:
                Qs.append(np.eye(b.stop - b.start))
            res.range_probes[l] = 0
            res.passed[l] = -1
            res.need[l] = mb
        else:
            def probe(col0, ncols):
                Om = np.zeros((N, ncols))
                for a in A:
                    r = np.arange(a.start, a.stop, dtype=np.uint64)[:, None]
                    c = np.arange(col0, col0 + ncols, dtype=np.uint64)[None, :]
                    Om[a] = rng.gaussian(seed, rng.STREAM_PROBE, l, r, c)
                return opt(Om) - apply_pieces(res.pieces, below, tree, Om)

            q = ql
            inc = q_test if predicted else b_inc
            # the first test batch is drawn together with the start block (one operator call)
            c1 = min(inc, q_max - q) if (adaptive and q < q_max and q < mb) else 0
            Y = probe(0, q + c1)
            res.range_calls[l] += 1
            pending = Y[:, q:] if c1 else None
            Y = Y[:, :q]
            Ys = [Y[b] for b in B]
            Qs = [range_basis(y) for y in Ys]
            res.need[l] = q
            while adaptive and q < q_max and q < mb:
                c = min(inc, q_max - q)
                inc = b_inc
                if pending is not None:
                    Yn, pending = pending, None
                else:
                    Yn = probe(q, c)
                    res.range_calls[l] += 1
                errs = []
                for i, b in enumerate(B):
                    yb = Yn[b]
                    if Qs[i].shape[1] >= yb.shape[0]:
                        errs.append(0.0)
                    else:
                        r = yb - Qs[i] @ (Qs[i].T @ yb)
                        errs.append(float(np.linalg.norm(r, axis=0).max()))
                res.test_err[l].append(errs)
                res.need[l] = q
                q += c
                ok = max(errs) <= thr
                if not (ok and certified):
                    for i, b in enumerate(B):
                        Ys[i] = np.hstack([Ys[i], Yn[b]])
                        Qs[i] = range_basis(Ys[i])
                if ok:
                    res.passed[l] = 1
                    break
            if res.passed[l] != 1:
                res.need[l] = q
            res.range_probes[l] = q
        ranks = [Q.shape[1] for Q in Qs]
        qp = max(ranks)
        Psi = np.zeros((N, qp))
        for b, Q in zip(B, Qs):
            Psi[b, :Q.shape[1]] = Q
        Z = opt(Psi) - apply_pieces(res.pieces, below, tree, Psi)
        P = np.zeros((N, qp))
        for a, b, Q in zip(A, B, Qs):
            k = Q.shape[1]
            P[b, :k] = Q
            P[a, :k] = Z[a, :k]
        res.pieces[l] = P
        res.rank[l] = ranks
        res.proj_probes[l] = qp

    # leaf diagonal blocks from identity probes
    L = tree.L
    lm = tree.leaf_max
    if covered:
        for t in range(1 << L):
            B = res.pieces[0][tree.rows(L, t)]
            res.D_diag.append(B @ B.T)
        res.samples = opt.samples
        return res
    Om = np.zeros((N, lm))
    nleaf = 1 << L
    for t in range(nleaf):
        r = tree.rows(L, t)
        m = r.stop - r.start
        Om[r.start + np.arange(m), np.arange(m)] = 1.0
    Y = opt(Om) - apply_pieces(res.pieces, range(0, L + 1), tree, Om)
    for t in range(nleaf):
        r = tree.rows(L, t)
        m = r.stop - r.start
        D = Y[r, :m]
        D = 0.5 * (D + D.T)
        if 0 in res.pieces:
            B = res.pieces[0][r]
            D = D + B @ B.T
        res.D_diag.append(D)
    res.samples = opt.samples
    return res
