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
