"""Pins of the oracle's hybrid construction: a global low-rank piece B B^T first, then H^2 on
the residual H - B B^T, with B B^T added back in the recompression (Section 3.3, end), and of
the semidefinite Cholesky factor that gives B.

Independent of the oracle's own code: the factor against numpy's Cholesky and an exactly
singular integer example; level 0 of the piece product against B B^T written out; exact
recovery of a globally low-rank matrix by the global piece alone (no level sampled) and of a
planted H^2 plus a global low-rank term through the residual route; on the small heat Hessian
the hybrid meets the tolerance with the same ranks and fewer products.  A planted mistake (the
transposed Cholesky factor) must fail the recovery pin.
"""
import importlib

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ClusterTree, Partition

import planted

peel_mod = importlib.import_module("oracle.peel")


def _rel(A, B):
    return np.linalg.norm(A - B, 2) / np.linalg.norm(A, 2)


def test_psd_cholesky_positive_definite_equals_library():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20, 20))
    M = A @ A.T + np.eye(20)
    C = O.psd_cholesky(M)
    np.testing.assert_allclose(C, np.linalg.cholesky(M), rtol=0, atol=1e-12 * np.abs(M).max())


def test_psd_cholesky_zero_pivot_is_dropped():
    # second pivot is exactly 1 - 2*2/4 = 0: its column stays zero, the third continues
    M = np.array([[4.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 9.0]])
    C = O.psd_cholesky(M)
    np.testing.assert_array_equal(C, np.array([[2.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 3.0]]))


def test_psd_cholesky_semidefinite_reproduces_matrix():
    rng = np.random.default_rng(6)
    V, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    lam = np.array([9.0, 4.0, 2.0, 1.0, 0.5] + [0.0] * 7)
    M = (V * lam) @ V.T
    M = 0.5 * (M + M.T)
    C = O.psd_cholesky(M)
    assert np.allclose(C, np.tril(C))
    assert np.linalg.norm(C @ C.T - M) <= 1e-12 * np.linalg.norm(M)


def test_level_zero_piece_product_is_b_bt():
    tree = ClusterTree(W.grid_coords(12), 16)
    rng = np.random.default_rng(2)
    B = rng.standard_normal((tree.N, 5))
    Om = rng.standard_normal((tree.N, 3))
    got = O.apply_pieces({0: B}, [0], tree, Om)
    np.testing.assert_allclose(got, B @ (B.T @ Om), rtol=1e-13, atol=1e-13)


def _build(A, n, leaf, global_rank, q0=32, q_max=256, tol=1e-6):
    return O.build(O.DenseOperator(A), W.grid_coords(n), leaf, ADM_STRONG, 0.7, tol, 64, q0, 16, q_max, True, 5,
                   global_rank=global_rank)


def test_global_low_rank_is_recovered_by_the_global_piece_alone():
    A = planted.global_low_rank(24 * 24, 9, 1)
    h, res = _build(A, 24, 16, 64)
    assert res.global_passed == 1 and res.global_rank == 48
    assert all(v == 2 for v in res.passed.values())
    # range finder 32 + first test batch 16 in one call, projection 48; no level and no leaf pass
    assert res.samples - res.norm_its == 48 + 48
    assert _rel(A, O.expand_dense(h)) < 1e-12
    assert max(int(k.max()) for k in h.k) <= 9


def test_residual_route_recovers_planted_h2_plus_global_low_rank():
    n, leaf = 16, 8
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_STRONG, 0.7)
    A = planted.planted_h2(tree, part, 3, 2, 4) + planted.global_low_rank(n * n, 5, 8)
    h, res = _build(A, n, leaf, 32)
    assert res.global_passed == 0 and res.global_rank == 32
    assert all(v != 2 for v in res.passed.values())
    assert _rel(A, O.expand_dense(h)) < 1e-12


def test_hybrid_heat_hessian_same_ranks_fewer_products():
    c = W.SMALL_N32
    p, b = c["problem"], c["build"]
    op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    H = op.dense()
    # rank cap 32: a partial global piece raises the level ranks above the 32 x 32 default cap of 16
    args = (op, W.grid_coords(p.n), b.leaf, ADM_STRONG, b.eta, b.tol, 32, 32, 16, 256, True, b.seed)
    h0, r0 = O.build(*args)
    h1, r1 = O.build(*args, global_rank=256)
    assert r1.global_passed == 1
    assert r1.samples < r0.samples
    assert _rel(H, O.expand_dense(h1)) <= b.tol
    for k0, k1 in zip(h0.k, h1.k):
        np.testing.assert_array_equal(k0, k1)
    # a budget below the global rank takes the residual route and still meets the tolerance
    h2m, r2 = O.build(*args, global_rank=64)
    assert r2.global_passed == 0 and not h2m.cap_hit
    assert _rel(H, O.expand_dense(h2m)) <= b.tol


def test_mutation_transposed_factor_is_caught(monkeypatch):
    """B = Q C^T instead of Q C (the factor's transpose) breaks exact recovery."""
    A = planted.global_low_rank(24 * 24, 9, 1)
    real = peel_mod.psd_cholesky
    monkeypatch.setattr(peel_mod, "psd_cholesky", lambda M: real(M).T)
    h, res = _build(A, 24, 16, 64)
    assert _rel(A, O.expand_dense(h)) > 1e-3
