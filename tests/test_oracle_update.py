"""Pins of the oracle's low-rank update with recompression (Section 3.2, Eqs. 3.3-3.4).

Planted H^2 matrices have exactly known ranks: every box whose far block row (its own far
blocks and its ancestors') is non-empty has rank k, the others rank 0.  Adding B M B^T with a
generic B of rank r makes every such far block row of rank k + r exactly (leaves and far
column sets are wide enough here), and the recompressed matrix must equal A + B M B^T to
rounding.  Removing the same term again (M = -I) must give back rank k and A.  At a loose
tolerance the result must stay within the target in the 2-norm.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

import planted


def _setup(adm, k=4, n=16, leaf=16, seed=3, grade=1.0):
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, adm, 0.7)
    A = planted.planted_h2(tree, part, k, 2, seed, grade=grade)
    return tree, part, A


def _has_far_row(tree, part, l, t):
    return O.far_columns(tree, part, l, t).size > 0


def _expected_ranks(tree, part, k):
    return [[k if _has_far_row(tree, part, l, t) else 0 for t in range(1 << l)] for l in range(tree.L + 1)]


def _compress(tree, part, A, tol=1e-13, kmax=48):
    At = A[np.ix_(tree.perm, tree.perm)]
    nrm = np.linalg.norm(A, 2)
    return O.compress_dense(tree, part, At, O.basis_threshold(tol, nrm, 1 << tree.L), kmax)


@pytest.mark.parametrize("adm", [ADM_STRONG, ADM_WEAK])
def test_far_columns_cover_every_far_block(adm):
    # the far block rows partition every row's off-near columns: for each leaf, the far columns
    # of the leaf and of its ancestors together with its near blocks' columns are all N columns,
    # each exactly once
    tree = ClusterTree(W.grid_coords(16), 16)
    part = Partition(tree, adm, 0.7)
    L = tree.L
    near_of = {}
    for t, s in part.near:
        near_of.setdefault(int(t), []).append(int(s))
    for t in range(1 << L):
        cols = list(O.far_columns(tree, part, L, t))
        for s in near_of.get(t, []):
            r = tree.rows(L, s)
            cols += list(range(r.start, r.stop))
        assert sorted(cols) == list(range(tree.N))


@pytest.mark.parametrize("adm", [ADM_STRONG, ADM_WEAK])
def test_compress_planted_recovers_ranks(adm):
    tree, part, A = _setup(adm)
    h = _compress(tree, part, A)
    want = _expected_ranks(tree, part, 4)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(h.k[l], want[l])
    assert np.linalg.norm(O.expand_dense(h) - A, 2) <= 1e-12 * np.linalg.norm(A, 2)


@pytest.mark.parametrize("adm,r", [(ADM_STRONG, 3), (ADM_WEAK, 3), (ADM_STRONG, 5)])
def test_update_rank_k_plus_r(adm, r):
    tree, part, A = _setup(adm)
    h = _compress(tree, part, A)
    rng = np.random.default_rng(11)
    B = rng.standard_normal((tree.N, r)) / np.sqrt(tree.N)
    hu, nrm, tau = O.lowrank_update(h, B, 1e-13, 48)
    want = _expected_ranks(tree, part, 4 + r)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(hu.k[l], want[l])
    At = A + B @ B.T
    assert np.linalg.norm(O.expand_dense(hu) - At, 2) <= 1e-12 * np.linalg.norm(At, 2)
    # the power iteration's estimate ||A~ v|| (||v|| = 1) is a lower bound of ||A~||_2; this
    # planted matrix is indefinite, so it converges slowly but must come close
    assert 0.9 * np.linalg.norm(At, 2) <= nrm <= (1 + 1e-12) * np.linalg.norm(At, 2)


def test_update_with_general_symmetric_m():
    tree, part, A = _setup(ADM_STRONG)
    h = _compress(tree, part, A)
    rng = np.random.default_rng(5)
    r = 3
    B = rng.standard_normal((tree.N, r)) / np.sqrt(tree.N)
    M = rng.standard_normal((r, r))
    hu, _, _ = O.lowrank_update(h, B, 1e-13, 48, M=M)
    At = A + B @ (0.5 * (M + M.T)) @ B.T
    assert np.linalg.norm(O.expand_dense(hu) - At, 2) <= 1e-12 * np.linalg.norm(At, 2)


def test_downdate_recovers_planted():
    tree, part, A = _setup(ADM_STRONG)
    h = _compress(tree, part, A)
    rng = np.random.default_rng(12)
    B = rng.standard_normal((tree.N, 4)) / np.sqrt(tree.N)
    hu, _, _ = O.lowrank_update(h, B, 1e-13, 48)
    hd, _, _ = O.lowrank_update(hu, B, 1e-13, 48, M=-np.eye(4))
    want = _expected_ranks(tree, part, 4)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(hd.k[l], want[l])
    assert np.linalg.norm(O.expand_dense(hd) - A, 2) <= 1e-12 * np.linalg.norm(A, 2)


def test_update_inside_the_bases_keeps_ranks():
    # B supported on the rows of one box b (the coarsest box 0 with a far row) with columns in
    # the span of b's basis: for a box t inside b, B_t lies in span(U_t) (the bases are nested);
    # for a box outside b, B_t = 0.  No far block row gains a direction, so every rank stays k.
    tree, part, A = _setup(ADM_STRONG)
    h = _compress(tree, part, A)
    rng = np.random.default_rng(2)
    B = np.zeros((tree.N, 2))
    lb = min(l for l in range(1, tree.L + 1) if _has_far_row(tree, part, l, 0))
    r = tree.rows(lb, 0)
    Ue = h.Uexp[lb][0]
    assert Ue.shape[1] == 4
    B[tree.perm[r.start:r.stop]] = Ue @ rng.standard_normal((4, 2))
    hu, _, _ = O.lowrank_update(h, B, 1e-13, 48)
    want = _expected_ranks(tree, part, 4)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(hu.k[l], want[l])
    At = A + B @ B.T
    assert np.linalg.norm(O.expand_dense(hu) - At, 2) <= 1e-12 * np.linalg.norm(At, 2)


def test_update_loose_tolerance_within_target():
    tree, part, A = _setup(ADM_STRONG, k=8, grade=0.35)
    h = _compress(tree, part, A)
    rng = np.random.default_rng(13)
    B = rng.standard_normal((tree.N, 6)) * (0.5 ** np.arange(6))[None, :] / np.sqrt(tree.N)
    tol = 1e-3
    hu, _, _ = O.lowrank_update(h, B, tol, 48)
    At = A + B @ B.T
    err = np.linalg.norm(O.expand_dense(hu) - At, 2) / np.linalg.norm(At, 2)
    assert err <= tol
    # the truncation is active: some box keeps fewer than k + r vectors
    assert max(int(x) for l in range(tree.L + 1) for x in hu.k[l]) < 8 + 6


def test_update_rank_replay_is_exact_when_ranks_agree():
    # replaying the ranks the update chose must give the same matrix (the replay path the GPU
    # parity tests use)
    tree, part, A = _setup(ADM_STRONG, k=6, grade=0.5)
    h = _compress(tree, part, A, tol=1e-6)
    rng = np.random.default_rng(14)
    B = rng.standard_normal((tree.N, 3)) / np.sqrt(tree.N)
    hu, nrm, _ = O.lowrank_update(h, B, 1e-6, 48)
    hr, _, _ = O.lowrank_update(h, B, 1e-6, 48, norm_est=nrm, ranks=hu.k)
    assert np.array_equal(np.concatenate(hu.k), np.concatenate(hr.k))
    assert np.abs(O.expand_dense(hu) - O.expand_dense(hr)).max() == 0.0
