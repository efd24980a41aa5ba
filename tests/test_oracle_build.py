"""Pins of the oracle's peeling construction, assembly and matvec.

Exact recovery of planted structures (global low rank, block diagonal, HSS on
the weak partition, H^2 on the strong partition), matvec against the dense
expansion, symmetry, the Frobenius identity, the power-iteration norm against
a dense SVD, and the approximation quality on the small heat Hessian.  Two
mutation tests plant a mistake in the oracle and check that the pins catch it.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
import importlib
peel_mod = importlib.import_module("oracle.peel")
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

import planted


def _build(A, n, leaf, adm, q0=32, q_max=256, adaptive=True, kmax=64, tol=1e-6):
    op = O.DenseOperator(A)
    h, res = O.build(op, W.grid_coords(n), leaf, adm, 0.7, tol, kmax, q0, 16, q_max, adaptive, 5)
    return h, res


def _rel(A, B):
    return np.linalg.norm(A - B, 2) / np.linalg.norm(A, 2)


@pytest.mark.parametrize("adm", [ADM_WEAK, ADM_STRONG])
def test_exact_recovery_global_low_rank(adm):
    A = planted.global_low_rank(24 * 24, 9, 1)
    h, res = _build(A, 24, 16, adm)
    assert _rel(A, O.expand_dense(h)) < 1e-12
    assert max(int(k.max()) for k in h.k) <= 9


@pytest.mark.parametrize("adm", [ADM_WEAK, ADM_STRONG])
def test_exact_recovery_block_diagonal(adm):
    tree = ClusterTree(W.grid_coords(16), 8)
    A = planted.block_diagonal(tree, 2)
    h, res = _build(A, 16, 8, adm)
    np.testing.assert_array_equal(O.expand_dense(h), A)
    assert all(int(k.max()) == 0 for k in h.k)
    for P in res.pieces.values():
        assert np.abs(P).max() <= 1.0 + 1e-12     # only Q columns, Z rows are exactly zero


def test_exact_recovery_planted_hss():
    n, leaf, k = 16, 8, 4
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_WEAK, 0.7)
    A = planted.planted_h2(tree, part, k, 0, 3)
    h, res = _build(A, n, leaf, ADM_WEAK, q0=8, kmax=16)
    assert _rel(A, O.expand_dense(h)) < 1e-12
    for l in range(1, tree.L + 1):
        assert int(h.k[l].max()) == k


def test_exact_recovery_planted_strong_h2():
    n, leaf, k = 16, 8, 3
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_STRONG, 0.7)
    A = planted.planted_h2(tree, part, k, 2, 4)
    h, res = _build(A, n, leaf, ADM_STRONG, q0=16, kmax=16)
    assert _rel(A, O.expand_dense(h)) < 1e-12
    for l in range(1, tree.L + 1):
        assert int(h.k[l].max()) <= k
    assert int(h.k[tree.L].max()) == k


def test_matvec_equals_dense_expansion_and_symmetry():
    n = 32
    p = W.SMALL_N32["problem"]
    op = O.HeatHessian(n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    h, res = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 16, 64, 16, 64, False, 7)
    Ad = O.expand_dense(h)
    np.testing.assert_array_equal(Ad, Ad.T)
    X = W.rhs(p.N, 7, 3)
    Y = O.matvec(h, X)
    assert np.linalg.norm(Y - Ad @ X) <= 1e-13 * np.linalg.norm(Ad @ X)
    # Frobenius identity with orthonormal bases (Section 3.2)
    assert abs(O.frobenius_norm(h) - np.linalg.norm(Ad)) <= 1e-12 * np.linalg.norm(Ad)
    for U in h.U.values():
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)


def test_single_leaf_is_one_dense_block():
    """N <= leaf: no levels, the approximation is the dense matrix from identity probes."""
    op = O.HeatHessian(4, 0.01, 0.5, 0.01, W.sensor_mask(16, 5, 5))
    h, res = O.build(op, W.grid_coords(4), 16, ADM_STRONG, 0.7, 1e-6, 8, 8, 8, 8, False, 3)
    assert h.tree.L == 0 and res.samples - res.norm_its == 16
    H = op.dense()
    np.testing.assert_allclose(O.expand_dense(h), 0.5 * (H + H.T), rtol=0, atol=1e-12 * np.abs(H).max())
    X = W.rhs(16, 3, 1)
    np.testing.assert_allclose(O.matvec(h, X), O.expand_dense(h) @ X, rtol=1e-13, atol=1e-13)


def test_norm_estimates_against_dense_svd():
    n = 20
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, W.sensor_mask(n * n, 60, 9))
    H = op.dense()
    true = np.linalg.norm(H, 2)
    tree = ClusterTree(W.grid_coords(n), 16)
    est, its = O.norm2_estimate(O.TreeOperator(op, tree), n * n, 7)
    assert abs(est - true) <= 1e-2 * true and its <= 50
    v0 = np.random.default_rng(1).standard_normal(n * n)
    assert abs(O.power_norm(lambda v: H @ v, n * n, v0) - true) <= 2e-2 * true


@pytest.mark.parametrize("adm,expect_ok", [(ADM_STRONG, True), (ADM_WEAK, False)])
def test_small_heat_hessian_quality(adm, expect_ok):
    """Heat Hessian at 32 x 32, leaf 32, 64 fixed probes per level, rank cap 16.
    Strong admissibility meets the tolerance; the weak (HSS) partition needs ranks
    above the cap of 16 and reports it."""
    c = W.SMALL_N32
    p, b = c["problem"], c["build"]
    op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    H = op.dense()
    h, res = O.build(op, W.grid_coords(p.n), b.leaf, adm, b.eta, b.tol, b.kmax, b.q0, b.b_inc,
                     b.q_max, b.adaptive, b.seed)
    err = _rel(H, O.expand_dense(h))
    if expect_ok:
        assert err <= b.tol and not h.cap_hit
    else:
        assert h.cap_hit and err > b.tol
    # deterministic sample count: 3 range passes of 64, projections 64,64,64,64,32, leaf pass 32
    assert res.samples - res.norm_its == 3 * 64 + 4 * 64 + 32 + 32


# ---------------------------------------------------------------- planted mistakes

def test_mutation_dropping_coarse_subtraction_is_caught(monkeypatch):
    """Without removing the coarser pieces from the samples, exact recovery fails."""
    n, leaf, k = 16, 8, 3
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_STRONG, 0.7)
    A = planted.planted_h2(tree, part, k, 2, 4)
    real = peel_mod.apply_pieces
    monkeypatch.setattr(peel_mod, "apply_pieces", lambda P, lv, t, Om: 0.0 * real(P, lv, t, Om))
    h, res = _build(A, n, leaf, ADM_STRONG, q0=16, kmax=16)
    assert _rel(A, O.expand_dense(h)) > 1e-3


def test_mutation_transposed_piece_is_caught(monkeypatch):
    """Storing the sibling piece with swapped factors breaks the exact-recovery pin."""
    n, leaf, k = 16, 8, 4
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_WEAK, 0.7)
    A = planted.planted_h2(tree, part, k, 0, 3)
    real_peel = peel_mod.peel

    def bad_peel(*args, **kw):
        res = real_peel(*args, **kw)
        t = args[1]
        for l, P in res.pieces.items():
            for i in range(1 << (l - 1)):
                a, b = t.rows(l, 2 * i), t.rows(l, 2 * i + 1)
                Pa, Pb = P[a].copy(), P[b].copy()
                P[a], P[b] = Pb, Pa
        return res

    monkeypatch.setattr(O, "peel", bad_peel)
    h, res = _build(A, n, leaf, ADM_WEAK, q0=8, kmax=16)
    assert _rel(A, O.expand_dense(h)) > 1e-3


@pytest.mark.parametrize("adm", [ADM_STRONG, ADM_WEAK])
def test_rank_replay_reproduces_adaptive_build(adm):
    """Rank replay (the probe counts, norm estimate and basis ranks of a finished construction
    given as data) reproduces that construction: same samples and ranks, same matrix to
    rounding.  This is the oracle mode that consumes another implementation's decisions."""
    n, m = 24, 120
    mask = W.sensor_mask(n * n, m, 41)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    h, res = O.build(op, W.grid_coords(n), 32, adm, 0.7, 1e-6, 24, 16, 16, 256, True, 3)
    probes = [res.range_probes.get(l, 0) for l in range(h.tree.L + 1)]
    assert any(res.passed[l] == -1 for l in range(1, h.tree.L + 1)) or min(probes[1:]) > 0
    hr, rr = O.replay_build(op, W.grid_coords(n), 32, adm, 0.7, 1e-6, 24, 3, res.norm_est, probes,
                            [np.asarray(k) for k in h.k])
    assert rr.samples == res.samples - res.norm_its
    for l in range(h.tree.L + 1):
        np.testing.assert_array_equal(hr.k[l], h.k[l])
    A, B = O.expand_dense(h), O.expand_dense(hr)
    assert np.linalg.norm(A - B, 2) <= 1e-13 * res.norm_est


def test_rank_replay_keeps_given_ranks_below_threshold():
    """Replayed ranks override the threshold: one rank fewer at every leaf changes the result
    by about the dropped singular value (a planted mistake that the 1e-12 comparison sees)."""
    n, m = 24, 120
    mask = W.sensor_mask(n * n, m, 41)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    h, res = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 24, 16, 16, 256, True, 3)
    L = h.tree.L
    probes = [res.range_probes.get(l, 0) for l in range(L + 1)]
    ranks = [np.asarray(k).copy() for k in h.k]
    ranks[L] = np.maximum(ranks[L] - 1, 0)
    for l in range(1, L):   # parents cannot keep more than their children offer
        ranks[l] = np.minimum(ranks[l], ranks[l + 1][0::2] + ranks[l + 1][1::2])
    hr, _ = O.replay_build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 24, 3, res.norm_est, probes, ranks)
    np.testing.assert_array_equal(hr.k[L], ranks[L])
    d = np.linalg.norm(O.expand_dense(h) - O.expand_dense(hr), 2) / res.norm_est
    assert d > 1e-9


def test_tight_tolerance_graded_planted():
    """A planted H^2 matrix whose far block rows have geometrically graded singular values
    (grade 0.2 per basis direction): at tol 1e-9 dozens of kept singular values lie between
    tau_basis and 1e-7 ||A||, below the square root of the rounding unit times the largest
    one, and the construction still meets the tolerance against the dense matrix."""
    n, leaf = 16, 16
    tree = ClusterTree(W.grid_coords(n), leaf)
    A = planted.planted_h2(tree, Partition(tree, ADM_STRONG, 0.7), 14, 2, 4, grade=0.2)
    nrm = np.linalg.norm(A, 2)
    h, res = O.build(O.DenseOperator(A), W.grid_coords(n), leaf, ADM_STRONG, 0.7, 1e-9, 32, 16, 16, 256, True, 5,
                     norm_est=nrm)
    svs = np.concatenate(list(h.sv.values()))
    assert np.sum((svs > res.tau_basis) & (svs < 1e-7 * nrm)) >= 20
    assert np.linalg.norm(O.expand_dense(h) - A, 2) <= 1e-9 * nrm


def test_replay_sensitivity_adaptive_64():
    """How closely two correct implementations can agree at the 64^2 adaptive configuration
    (leaf 64, strong 0.7, tol 1e-6): the oracle's own rank-replay construction moves by more
    than 1e-12 relative when the operator's products are perturbed at the level of one
    rounding (1e-16 relative).  The range bases of the finest levels have more probes than
    the sampled blocks' numerical rank, and the projection pass applies all sibling blocks'
    bases at once, so the coarse levels' residual couples every basis vector (weak ones
    included) into the pieces.  The GPU parity bound for this configuration, 2e-11, is a
    small multiple of this measured sensitivity; at 32^2 the same comparison is 1e-12."""
    n, m = 64, 256
    mask = W.sensor_mask(n * n, m, 1002)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    h, res = O.build(op, W.grid_coords(n), 64, ADM_STRONG, 0.7, 1e-6, 32, 32, 16, 256, True, 7)
    L = h.tree.L
    probes = [res.range_probes.get(l, 0) for l in range(L + 1)]
    rng = np.random.default_rng(5)

    def perturbed(X):
        Y = op(X)
        return Y * (1.0 + 1e-16 * rng.standard_normal(Y.shape))

    hp, _ = O.replay_build(perturbed, W.grid_coords(n), 64, ADM_STRONG, 0.7, 1e-6, 32, 7, res.norm_est, probes,
                           [np.asarray(k) for k in h.k])
    d = np.linalg.norm(O.expand_dense(hp) - O.expand_dense(h), 2) / res.norm_est
    assert 1e-12 < d < 1e-11
