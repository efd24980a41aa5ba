"""Pins of the certified range basis (the adaptive range finder in its textbook form, halko11
Algorithm 4.2, cited in Section 3.3): the columns of the test that passes are not added to the
basis, so the projection pass applies only the basis the test certified.

* Exact recovery of a planted H^2 matrix whose far blocks have rank <= k.
* At level 1 (nothing coarser is removed) the certified basis of every sibling block spans
  the leading columns of the basis that the default construction (passing test columns
  included) builds from the same probes.  Its trailing columns sit at the test threshold and
  move with rounding by about eps / (threshold / ||H||), so the two are compared through the
  sampled block itself: the projections Q Q^T H[b, a] agree to rounding.
* On heat Hessians (32^2, 48^2, strong partition, tol 1e-6) the construction meets the
  tolerance against the dense Hessian with fewer products than the default.
* Rank replay with the certified basis sizes as the probe counts reproduces the construction.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ClusterTree, Partition

import planted


def _heat(n, m, seed):
    return O.HeatHessian(n, 0.01, 0.5, 0.01, W.sensor_mask(n * n, m, seed))


def test_certified_planted_exact():
    n, leaf, k = 16, 8, 3
    tree = ClusterTree(W.grid_coords(n), leaf)
    A = planted.planted_h2(tree, Partition(tree, ADM_STRONG, 0.7), k, 2, 4)
    nrm = np.linalg.norm(A, 2)
    h, res = O.build(O.DenseOperator(A), W.grid_coords(n), leaf, ADM_STRONG, 0.7, 1e-6, 16, 8, 8, 256, True, 5,
                     norm_est=nrm, certified=True)
    assert np.linalg.norm(O.expand_dense(h) - A, 2) <= 1e-12 * nrm
    for l in range(1, tree.L + 1):
        if res.passed[l] == 1:
            assert res.proj_probes[l] == res.need[l] < res.range_probes[l]
    assert int(h.k[tree.L].max()) == k


@pytest.mark.parametrize("n,m", [(32, 200), (48, 300)])
def test_certified_basis_is_the_tested_prefix(n, m):
    op = _heat(n, m, 17)
    h0, r0 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 16, 256, True, 3)
    h1, r1 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 16, 256, True, 3,
                     norm_est=r0.norm_est, certified=True)
    tree = h0.tree
    for l in range(1, tree.L + 1):   # the same probes and tests at every level
        assert r1.range_probes[l] == r0.range_probes[l] and r1.need[l] == r0.need[l]
    assert r1.passed[1] == 1
    Ht = op.dense()[np.ix_(tree.perm, tree.perm)]
    a, b = tree.rows(1, 0), tree.rows(1, 1)
    kc = r1.rank[1][0]
    assert kc == r1.need[1] < r0.rank[1][0]
    Qc, Q0 = r1.pieces[1][b, :kc], r0.pieces[1][b, :kc]
    Hba = Ht[b, a]
    d = np.linalg.norm(Qc @ (Qc.T @ Hba) - Q0 @ (Q0.T @ Hba), 2) / r0.norm_est
    assert d <= 1e-13
    # and the certified basis alone meets the level's threshold on the sampled block
    res = np.linalg.norm(Hba - Qc @ (Qc.T @ Hba), 2)
    assert res <= 1e-6 * r0.norm_est


@pytest.mark.parametrize("n,m", [(32, 200), (48, 300)])
def test_certified_heat_meets_tolerance_with_fewer_products(n, m):
    op = _heat(n, m, 23)
    H = op.dense()
    nh = np.linalg.norm(H, 2)
    tol = 1e-6
    h0, r0 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, tol, 32, 16, 16, 256, True, 3)
    h1, r1 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, tol, 32, 16, 16, 256, True, 3,
                     norm_est=r0.norm_est, certified=True)
    e0 = np.linalg.norm(O.expand_dense(h0) - H, 2) / nh
    e1 = np.linalg.norm(O.expand_dense(h1) - H, 2) / nh
    print(f"heat {n}^2: default {r0.samples - r0.norm_its} products, error {e0:.1e}; "
          f"certified {r1.samples - r1.norm_its}, error {e1:.1e}")
    assert e1 <= tol
    assert r1.samples < r0.samples


def test_certified_replay_reproduces():
    n, m = 32, 200
    op = _heat(n, m, 29)
    h, res = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 16, 256, True, 3, certified=True)
    L = h.tree.L
    probes = [0 if res.range_probes.get(l, 0) == 0 else res.proj_probes[l] for l in range(L + 1)]
    hr, rr = O.replay_build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 3, res.norm_est, probes,
                            [np.asarray(k) for k in h.k])
    for l in range(L + 1):
        np.testing.assert_array_equal(hr.k[l], h.k[l])
    d = np.linalg.norm(O.expand_dense(h) - O.expand_dense(hr), 2) / res.norm_est
    assert d <= 1e-13


def test_certified_after_predicted_starts():
    """With predicted start counts (the learned-rank path: start q_level[l], first test of q_test
    columns) the certified basis keeps the start block when that first test passes, so the
    projection pass uses exactly the predicted count; the construction meets the tolerance."""
    n, m = 32, 200
    op = _heat(n, m, 31)
    H = op.dense()
    h0, r0 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 16, 256, True, 3)
    L = h0.tree.L
    # start each level from what the adaptive finder needed (a perfect prediction)
    q_level = [0] + [int(r0.need[l]) if r0.passed[l] == 1 else 0 for l in range(1, L + 1)]
    h1, r1 = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 16, 256, True, 3,
                     norm_est=r0.norm_est, q_level=q_level, q_test=8, certified=True)
    checked = 0
    for l in range(1, L + 1):
        if q_level[l] and r1.passed[l] == 1 and r1.range_calls[l] == 1:   # the first test passed
            assert r1.proj_probes[l] == q_level[l] == r1.need[l]
            assert r1.range_probes[l] == q_level[l] + 8
            checked += 1
    assert checked > 0
    e = np.linalg.norm(O.expand_dense(h1) - H, 2) / np.linalg.norm(H, 2)
    assert e <= 1e-6
    assert r1.samples < r0.samples
