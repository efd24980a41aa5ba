"""Element-wise comparison of a computed matvec result with a reference.

Two measures, both required to be within the test's bound:
* per column: ||got_j - want_j||_2 / ||want_j||_2 for every right-hand side j, so that
  one wrong right-hand-side tile cannot hide behind the others;
* per leaf block: max |got - want| / max |want| over the rows of every leaf box (all
  columns), so that one wrong leaf block cannot hide behind the rest of the vector.
Arrays are N x nrhs in original node order; leaves are the original indices of every
leaf box (from the oracle's cluster tree).
"""
import numpy as np


def leaf_index_sets(tree):
    L = tree.L
    return [tree.perm[tree.rows(L, t)] for t in range(1 << L)]


def column_rel(got, want):
    got = np.asarray(got, dtype=np.float64).reshape(want.shape[0], -1)
    want = np.asarray(want, dtype=np.float64).reshape(want.shape[0], -1)
    num = np.linalg.norm(got - want, axis=0)
    den = np.linalg.norm(want, axis=0)
    return float(np.max(num / np.where(den > 0, den, 1.0)))


def leaf_block_rel(got, want, leaves):
    got = np.asarray(got, dtype=np.float64).reshape(want.shape[0], -1)
    want = np.asarray(want, dtype=np.float64).reshape(want.shape[0], -1)
    worst = 0.0
    for idx in leaves:
        d = float(np.abs(got[idx] - want[idx]).max())
        r = float(np.abs(want[idx]).max())
        worst = max(worst, d / r if r > 0 else (0.0 if d == 0 else np.inf))
    return worst


def assert_elementwise(got, want, leaves, tol, what=""):
    c = column_rel(got, want)
    b = leaf_block_rel(got, want, leaves)
    assert np.all(np.isfinite(got)), f"{what}: non-finite entries"
    assert c <= tol, f"{what}: worst column error {c:.2e} > {tol:.0e}"
    assert b <= tol, f"{what}: worst leaf-block error {b:.2e} > {tol:.0e}"
    return c, b
