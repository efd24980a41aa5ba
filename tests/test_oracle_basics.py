"""Pins of the oracle's building blocks against facts fixed outside the oracle.

Generator: published SplitMix64 outputs and Gaussian statistics.
Operator: closed-form eigenpairs, a library matrix exponential, symmetry,
positive semi-definiteness and the rank bound of the sensor mask.
Tree / partition: a hand-worked KD tree, the depths the paper states,
brute-force cover and admissibility checks.
"""
import math
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.stats

import workloads as W
from oracle import heat, rng
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- generator

def test_splitmix64_reference_outputs():
    want = [int(x, 16) for x in _golden_lines("splitmix64.txt")]
    got = [int(rng.splitmix_at(np.uint64(0), i)) for i in range(len(want))]
    assert got == want


def test_gaussian_probe_statistics():
    g = rng.gaussian_block(123, rng.STREAM_PROBE, 3, 4096, 0, 64).ravel()
    assert abs(g.mean()) < 0.01
    assert abs(g.var() - 1.0) < 0.01
    assert scipy.stats.kstest(g, "norm").pvalue > 1e-3
    # counter-based: a sub-block equals the same entries of a larger block
    big = rng.gaussian_block(123, rng.STREAM_PROBE, 3, 100, 5, 7)
    one = rng.gaussian(123, rng.STREAM_PROBE, 3, np.uint64(42), np.uint64(9))
    assert big[42, 4] == one
    # streams and levels decorrelate
    other = rng.gaussian_block(123, rng.STREAM_PROBE, 4, 4096, 0, 64).ravel()
    assert abs(np.corrcoef(g, other)[0, 1]) < 0.01


# ---------------------------------------------------------------- operator

def test_dst_orthonormal_symmetric():
    for n in (1, 5, 32):
        S = heat.dst_matrix(n)
        np.testing.assert_allclose(S, S.T, atol=1e-15)
        np.testing.assert_allclose(S @ S, np.eye(n), atol=1e-13)


def test_sine_modes_are_eigenvectors_of_F():
    n, kappa, T = 12, 0.02, 0.5
    op = heat.HeatHessian(n, kappa, T, 1.0, np.ones(n * n))
    h = 1.0 / (n + 1)
    for (a, b) in [(1, 1), (2, 7), (12, 3)]:
        i = np.arange(1, n + 1)
        mode = np.outer(np.sin(np.pi * a * i * h), np.sin(np.pi * b * i * h)).ravel()
        mu = lambda k: 4.0 / h ** 2 * math.sin(k * math.pi * h / 2) ** 2
        lam = math.exp(-T * kappa * (mu(a) + mu(b)))
        np.testing.assert_allclose(op.apply_F(mode[:, None])[:, 0], lam * mode, rtol=1e-12, atol=1e-14)


def test_F_equals_library_expm_of_5pt_laplacian():
    for n in (4, 9, 13):
        kappa, T = 0.01, 0.5
        op = heat.HeatHessian(n, kappa, T, 1.0, np.ones(n * n))
        F_lib = scipy.linalg.expm(T * kappa * heat.laplacian_5pt(n))
        np.testing.assert_allclose(op.dense_F(), F_lib, rtol=0, atol=1e-12)


def test_hessian_structure():
    n, m = 10, 17
    mask = W.sensor_mask(n * n, m, 3)
    op = heat.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    H = op.dense()
    F = scipy.linalg.expm(0.5 * 0.01 * heat.laplacian_5pt(n))
    np.testing.assert_allclose(H, F @ np.diag(mask) @ F / 0.01 ** 2, rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-10 * np.abs(H).max())
    ev = np.linalg.eigvalsh(H)
    assert ev.min() > -1e-10 * ev.max()
    assert int(np.sum(ev > 1e-10 * ev.max())) == m


# ---------------------------------------------------------------- tree

def test_tree_hand_worked_4x4():
    lines = _golden_lines("tree_4x4.txt")
    t = ClusterTree(W.grid_coords(4), 4)
    assert t.L == int(lines[0])
    assert t.perm.tolist() == [int(x) for x in lines[1].split()]


def test_tree_depths_stated_in_paper():
    for line in _golden_lines("paper_levels.txt"):
        n, dim, leaf, levels = (int(x) for x in line.split())
        if dim == 1:
            coords = (np.arange(n, dtype=np.float64)[:, None] + 1) / (n + 1)
        else:
            coords = W.grid_coords(n)
        assert ClusterTree(coords, leaf).L == levels


@pytest.mark.parametrize("n,leaf", [(16, 8), (23, 16), (32, 32), (37, 64)])
def test_tree_invariants(n, leaf):
    coords = W.grid_coords(n)
    t = ClusterTree(coords, leaf)
    N = n * n
    assert sorted(t.perm.tolist()) == list(range(N))
    assert t.sizes[t.L].max() <= leaf
    if t.L > 0:
        assert -(-N // (1 << (t.L - 1))) > leaf
    for l in range(t.L + 1):
        sz = t.sizes[l]
        assert sz.sum() == N and sz.max() - sz.min() <= 1
        assert (t.starts[l] == np.concatenate([[0], np.cumsum(sz)[:-1]])).all()
    for l in range(t.L):
        for i in range(1 << l):
            r0, r1 = t.rows(l + 1, 2 * i), t.rows(l + 1, 2 * i + 1)
            p0, p1 = coords[t.perm[r0]], coords[t.perm[r1]]
            ext = t.hi[l][i] - t.lo[l][i]
            d = int(np.argmax(ext))
            # median split: child 0 never lies beyond child 1 along the split coordinate
            assert p0[:, d].max() <= p1[:, d].min()
            assert r0.stop - r0.start == (r0.stop - r0.start + r1.stop - r1.start) // 2


@pytest.mark.parametrize("adm", [ADM_WEAK, ADM_STRONG])
@pytest.mark.parametrize("n,leaf", [(16, 8), (21, 16)])
def test_partition_exact_cover_symmetric_admissible(adm, n, leaf):
    t = ClusterTree(W.grid_coords(n), leaf)
    p = Partition(t, adm, 0.7)
    N = n * n
    cover = np.zeros((N, N), dtype=np.int32)
    for l, far in enumerate(p.far):
        for a, b in far:
            cover[t.rows(l, a), t.rows(l, b)] += 1
            # admissibility checked by brute force over the points of both boxes
            assert a != b
            if adm == ADM_STRONG:
                pa, pb = W.grid_coords(n)[t.perm[t.rows(l, a)]], W.grid_coords(n)[t.perm[t.rows(l, b)]]
                da = np.linalg.norm(pa.max(0) - pa.min(0))
                db = np.linalg.norm(pb.max(0) - pb.min(0))
                gap = np.maximum(0, np.maximum(pb.min(0) - pa.max(0), pa.min(0) - pb.max(0)))
                assert max(da, db) <= 0.7 * np.linalg.norm(gap)
                # maximality: the parent pair was not admissible
                if l > 1:
                    assert not p.admissible(l - 1, a // 2, b // 2)
    for a, b in p.near:
        cover[t.rows(t.L, a), t.rows(t.L, b)] += 1
        assert not p.admissible(t.L, a, b)
    assert (cover == 1).all()
    farset = {(l, int(a), int(b)) for l, f in enumerate(p.far) for a, b in f}
    assert all((l, b, a) in farset for (l, a, b) in farset)
    nearset = {(int(a), int(b)) for a, b in p.near}
    assert all((b, a) in nearset for (a, b) in nearset)
    if adm == ADM_WEAK:
        assert farset == {(l, 2 * i + c, 2 * i + 1 - c) for l in range(1, t.L + 1)
                          for i in range(1 << (l - 1)) for c in (0, 1)}
        assert nearset == {(i, i) for i in range(1 << t.L)}


def test_pair_level():
    assert Partition.pair_level(2, 2, 3) == 2
    assert Partition.pair_level(3, 0, 7) == 1
    assert Partition.pair_level(3, 4, 6) == 2


def test_factor_layout_round_trip():
    """tests/factors.py: oracle factors -> h2_import layout -> oracle H2Matrix gives the same
    matrix (the test helper that reads exported GPU factors into the oracle)."""
    import factors
    import oracle as O

    n = 24
    mask = W.sensor_mask(n * n, 100, 7)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    h = O.build(op, W.grid_coords(n), 32, ADM_STRONG, 0.7, 1e-6, 24, 16, 16, 128, True, 3)[0]
    g = factors.import_to_oracle(h.tree, h.part, *factors.oracle_to_import(h))
    A = O.expand_dense(h)
    assert np.abs(O.expand_dense(g) - A).max() <= 1e-14 * np.abs(A).max()   # BLAS layouts differ: rounding only
    X = W.rhs(n * n, 3, 1)
    Y = O.matvec(h, X)
    assert np.abs(O.matvec(g, X) - Y).max() <= 1e-14 * np.abs(Y).max()
