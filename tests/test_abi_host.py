"""Host-side checks of the C-ABI library (no GPU needed).

* The shared library builds, loads and exports every function include/h2.h declares.
* The cluster tree and the block partition computed by the library's host code
  equal the oracle's exactly (permutation, box ranges, far and near lists).
* Argument validation returns the documented status codes.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def h2():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    m.lib()
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "h2.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(h2_[a-z0-9_]+)\s*\(", src))
    return sorted(n for n in names if n != "h2_op_fn")


def test_every_declared_function_is_exported(h2):
    names = _declared()
    assert len(names) >= 25
    so = ctypes.CDLL(h2.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    # and the binding covers them all
    assert set(names) <= set(h2.exported_symbols())


@pytest.mark.parametrize("adm", [ADM_WEAK, ADM_STRONG])
@pytest.mark.parametrize("n,leaf", [(4, 4), (16, 8), (23, 16), (32, 32), (64, 64), (97, 64)])
def test_tree_and_partition_match_oracle(h2, adm, n, leaf):
    coords = W.grid_coords(n)
    ot = ClusterTree(coords, leaf)
    op = Partition(ot, adm, 0.7)
    t = h2.Tree(coords, leaf, adm, 0.7)
    assert t.L == ot.L and t.N == ot.N
    np.testing.assert_array_equal(t.perm(), ot.perm)
    for l in range(t.L + 1):
        st, sz = t.boxes(l)
        np.testing.assert_array_equal(st, ot.starts[l])
        np.testing.assert_array_equal(sz, ot.sizes[l])
        np.testing.assert_array_equal(t.far(l), op.far[l])
    np.testing.assert_array_equal(t.near(), op.near)


def test_tree_of_scattered_points_matches_oracle(h2):
    rng = np.random.default_rng(4)
    coords = rng.random((3000, 2))
    coords[::7] = np.round(coords[::7], 1)      # many ties in both coordinates
    ot = ClusterTree(coords, 40)
    op = Partition(ot, ADM_STRONG, 1.1)
    t = h2.Tree(coords, 40, ADM_STRONG, 1.1)
    np.testing.assert_array_equal(t.perm(), ot.perm)
    for l in range(t.L + 1):
        np.testing.assert_array_equal(t.far(l), op.far[l])
    np.testing.assert_array_equal(t.near(), op.near)


def test_argument_validation(h2):
    L = h2.lib()
    h = ctypes.c_void_p()
    c = np.zeros((4, 2))
    assert L.h2_tree_create(c.ctypes.data, 4, 2, 1, 0, 0.7, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    assert L.h2_tree_create(c.ctypes.data, 0, 2, 4, 0, 0.7, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    assert L.h2_tree_create(c.ctypes.data, 4, 2, 4, 7, 0.7, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    assert L.h2_tree_create(c.ctypes.data, 4, 2, 4, 1, -1.0, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    c[1, 0] = np.nan
    assert L.h2_tree_create(c.ctypes.data, 4, 2, 4, 0, 0.7, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    assert b"non-finite" in L.h2_last_error()
    assert L.h2_build(None, None, None, 1e-6, None, ctypes.byref(h)) == h2.H2_ERR_INVALID_ARG
    assert L.h2_matvec(None, None, 1, None, 1, 1, 0, None) == h2.H2_ERR_INVALID_ARG
    assert L.h2_error_string(h2.H2_ERR_OOM) == b"H2_ERR_OOM"
    L.h2_free(None)
    L.h2_tree_free(None)
    o = h2.default_opts()
    assert (o.kmax, o.q0, o.b_inc, o.q_max, o.adaptive) == (32, 32, 16, 256, 1)
    assert (o.q_level, o.q_level_stride, o.q_test, o.global_rank) == (None, 0, 8, 0)
    assert (o.sampling, o.batch_workers, o.certified) == (0, 0, 0)


def test_build_option_validation(h2):
    """Build options are checked before any device work: every bad value is rejected with
    H2_ERR_INVALID_ARG and a message naming it (no GPU needed)."""
    L = h2.lib()
    coords = W.grid_coords(8)
    tree = ctypes.c_void_p()
    assert L.h2_tree_create(coords.ctypes.data, 64, 2, 16, 1, 0.7, ctypes.byref(tree)) == 0
    never = h2.OP_FN(lambda *a: 1)   # not called: validation fails first
    cases = [(dict(certified=2), b"certified"), (dict(sampling=5), b"sampling"),
             (dict(batch_workers=-1), b"batch_workers"), (dict(b_inc=17), b"b_inc"),
             (dict(q_test=0), b"q_test"), (dict(kmax=0), b"kmax"),
             (dict(sampling=h2.H2_SAMPLING_COLORED, q0=32), b"coloured")]
    try:
        for kw, word in cases:
            o = h2.default_opts(**kw)
            out = ctypes.c_void_p()
            st = L.h2_build(never, None, tree, 1e-6, ctypes.byref(o), ctypes.byref(out))
            assert st == h2.H2_ERR_INVALID_ARG, kw
            assert word in L.h2_last_error(), (kw, L.h2_last_error())
            assert not out.value
        out = ctypes.c_void_p()
        assert L.h2_build(never, None, tree, -1.0, None, ctypes.byref(out)) == h2.H2_ERR_INVALID_ARG
    finally:
        L.h2_tree_free(tree)


@pytest.mark.parametrize("n,leaf,adm", [(4, 4, ADM_WEAK), (37, 16, ADM_STRONG), (64, 64, ADM_STRONG)])
def test_rank_features_match_oracle(h2, n, leaf, adm):
    """The library's per-level rank-model features equal the oracle's (host code, no GPU)."""
    from oracle import mlp
    coords = W.grid_coords(n)
    t = h2.Tree(coords, leaf, adm, 0.7)
    got = h2.rank_features(t, 0.005, 0.125, 1e-6)
    want = mlp.level_features(ClusterTree(coords, leaf), 0.005, 0.125, 1e-6)
    assert got.shape == want.shape
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-15)


def test_rank_model_argument_validation(h2):
    L = h2.lib()
    t = h2.Tree(W.grid_coords(8), 8)
    out = np.empty((t.L + 1, 8))
    assert L.h2_rankmodel_features(t.handle, -1.0, 0.1, 1e-6, out.ctypes.data) == h2.H2_ERR_INVALID_ARG
    assert L.h2_rankmodel_features(t.handle, 0.01, 0.1, 0.0, out.ctypes.data) == h2.H2_ERR_INVALID_ARG
    assert L.h2_rankmodel_features(None, 0.01, 0.1, 1e-6, out.ctypes.data) == h2.H2_ERR_INVALID_ARG
    assert L.h2_rankmodel_train(None, None, None, 1, None, 1, 1, 1e-3, None, None) == h2.H2_ERR_INVALID_ARG
    assert L.h2_rankmodel_create(0, 1, None) == h2.H2_ERR_INVALID_ARG
    L.h2_rankmodel_free(None)
    o = h2.default_opts(q_test=0)
    assert L.h2_build(None, None, None, 1e-6, ctypes.byref(o), ctypes.byref(ctypes.c_void_p())) == \
        h2.H2_ERR_INVALID_ARG


def test_rank_model_load_rejects_bad_files(h2, tmp_path):
    """A file that is not a saved rank model is rejected before any device work."""
    L = h2.lib()
    out = ctypes.c_void_p()
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"H2RM0002" + bytes(64))
    assert L.h2_rankmodel_load(str(bad).encode(), ctypes.byref(out)) == h2.H2_ERR_INVALID_ARG
    assert b"not a rank model" in L.h2_last_error()
    short = tmp_path / "short.bin"
    short.write_bytes(b"H2RM0001" + bytes(12))
    assert L.h2_rankmodel_load(str(short).encode(), ctypes.byref(out)) == h2.H2_ERR_INVALID_ARG
    assert L.h2_rankmodel_load(str(tmp_path / "missing.bin").encode(), ctypes.byref(out)) == h2.H2_ERR_INVALID_ARG
    assert not out.value
