"""Pins of the oracle's strong-structure coloured sampling (Section 3.3), and integer parity of the
library's sampling plan (colours, probe slots, leaf colours) with the oracle's.

* The colourings are valid by their definition: no row box sees two column boxes of one colour
  among its visited pairs; no slot holds two pairs that share a row box or whose row box reaches the
  other pair's column box.
* Sampling is exact on a planted H^2 matrix whose far blocks have rank <= q: the sampled
  approximation K equals the matrix to rounding, and the H^2 form recovers its ranks.
* On the 32^2 heat Hessian the coloured construction meets the tolerance.
* The library's plan (host code, no GPU) has the same counts as the oracle's at 32^2 .. 256².
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import colored as C
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

import planted


def _tree(n, leaf, adm=ADM_STRONG):
    tree = ClusterTree(W.grid_coords(n), leaf)
    return tree, Partition(tree, adm, 0.7)


@pytest.mark.parametrize("adm", [ADM_STRONG, ADM_WEAK])
def test_visited_pairs_are_the_partition(adm):
    tree, part = _tree(32, 32, adm)
    V = C.visited_pairs(tree, part)
    L = tree.L
    for l in range(L + 1):
        for t, ss in V[l].items():
            for s in ss:
                assert t in V[l][s]          # symmetric
        far = {(int(t), int(s)) for t, s in part.far[l]}
        got = {(t, s) for t, ss in V[l].items() for s in ss}
        assert far <= got
        if l == L:
            assert got == far | {(int(t), int(s)) for t, s in part.near}
        else:   # every other visited pair is split: its four children are visited
            for t, s in got - far:
                for ct in (2 * t, 2 * t + 1):
                    for cs in (2 * s, 2 * s + 1):
                        assert cs in V[l + 1].get(ct, [])


@pytest.mark.parametrize("n,leaf,adm", [(32, 32, ADM_STRONG), (64, 64, ADM_STRONG), (32, 32, ADM_WEAK)])
def test_colourings_are_interference_free(n, leaf, adm):
    tree, part = _tree(n, leaf, adm)
    plan = C.ColoredPlan(tree, part, 8)
    for l in range(tree.L + 1):
        V = plan.V[l]
        col = plan.color[l]
        for t, ss in V.items():
            seen = [col[s] for s in ss if s in col]
            assert len(seen) == len(set(seen)), (l, t)
        slots = {}
        for (t, s), j in zip(plan.pairs[l], plan.slot[l]):
            slots.setdefault(j, []).append((t, s))
        for j, ps in slots.items():
            rows = [t for t, _ in ps]
            assert len(rows) == len(set(rows))
            for t, s in ps:
                for t2, s2 in ps:
                    if (t, s) != (t2, s2):
                        assert s not in V.get(t2, []) and s2 not in V.get(t, [])
    for t, ss in plan.V[tree.L].items():
        cs = [plan.leaf_color[s] for s in ss]
        assert len(cs) == len(set(cs))


def test_colored_sampling_exact_on_planted():
    tree, part = _tree(16, 16)
    A = planted.planted_h2(tree, part, 4, 2, 3)
    op = O.DenseOperator(A)
    res = C.peel_colored(op, tree, part, 1e-10, 8, 5, norm_est=float(np.linalg.norm(A, 2)))
    K = C.dense_from_colored(tree, part, res)
    At = A[np.ix_(tree.perm, tree.perm)]
    assert np.linalg.norm(K - At, 2) <= 1e-12 * np.linalg.norm(A, 2)
    plan = C.ColoredPlan(tree, part, 8)
    assert res.samples == plan.samples()


def test_colored_build_recovers_planted_ranks():
    tree, part = _tree(16, 16)
    A = planted.planted_h2(tree, part, 4, 2, 3)
    h, res, plan = C.build_colored(O.DenseOperator(A), W.grid_coords(16), 16, ADM_STRONG, 0.7, 1e-13, 48, 8, 5,
                                   norm_est=float(np.linalg.norm(A, 2)))
    for l in range(tree.L + 1):
        want = [4 if O.far_columns(tree, part, l, t).size else 0 for t in range(1 << l)]
        np.testing.assert_array_equal(h.k[l], want)
    assert np.linalg.norm(O.expand_dense(h) - A, 2) <= 1e-12 * np.linalg.norm(A, 2)


def test_colored_heat32_meets_tolerance():
    p = W.SMALL_N32["problem"]
    op = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, W.sensor_mask(p.N, p.m, p.sensor_seed))
    h, res, plan = C.build_colored(op, W.grid_coords(p.n), 32, ADM_STRONG, 0.7, 1e-6, 32, 16, 7)
    H = op(np.eye(p.N))
    err = np.linalg.norm(O.expand_dense(h) - H, 2) / np.linalg.norm(H, 2)
    assert err <= 1e-6
    assert res.samples == plan.samples()


@pytest.mark.parametrize("n,leaf,adm,q", [(32, 32, ADM_STRONG, 16), (64, 64, ADM_STRONG, 16), (128, 64, ADM_STRONG, 16),
                                          (256, 64, ADM_STRONG, 16), (64, 32, ADM_WEAK, 8)])
def test_library_plan_matches_oracle(n, leaf, adm, q):
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    gt = m.Tree(W.grid_coords(n), leaf, adm, 0.7)
    got = gt.colored_plan(q)
    tree, part = _tree(n, leaf, adm)
    plan = C.ColoredPlan(tree, part, q)
    assert got["colors"] == plan.ncolors
    assert got["slots"] == plan.nslots
    assert got["pairs"] == [len(p) for p in plan.pairs]
    assert got["leaf_colors"] == plan.nleafcolors
