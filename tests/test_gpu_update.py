"""h2_lowrank_update (Section 3.2, Eqs. 3.3-3.4) on the GPU against the oracle's update.

* Planted H^2 matrices (oracle compression imported into the library): after + B B^T every box
  with a far row has rank k + r exactly, and the result equals A + B B^T to rounding; the
  downdate (M = -I) gives back rank k and A.  The GPU result must also match the oracle's update
  element-wise.
* A heat Hessian built on the GPU at tol 1e-6 (exported and read by the oracle) plus a rank-4
  update: the rank decisions of every box must agree with the oracle's (or sit at a near-tie of
  the threshold), and with the GPU's ranks replayed the two matrices must agree to 1e-12.
* The norm estimate of the updated matrix (power iteration through products with A~) must agree
  with the oracle's power iteration on the dense A~.
"""
import numpy as np
import pytest
import torch

import factors
import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition
from parity import assert_elementwise, leaf_index_sets

import planted

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    m.lib()
    assert torch.cuda.is_available()
    return m


def gpu_dense(G, N):
    I = torch.eye(N, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(I)
    G.matvec(I, Y, N)
    torch.cuda.synchronize()
    return Y.cpu().numpy().T


def dev_cols(B):
    """Device copy of the N x r array B in column-major order (a (r, N) row-major tensor)."""
    return torch.from_numpy(np.ascontiguousarray(B.T)).cuda()


def ranks_of(G, L):
    flat = G.export()[0]
    out, o = [], 0
    for l in range(L + 1):
        out.append(np.asarray(flat[o:o + (1 << l)], dtype=np.int64))
        o += 1 << l
    return out


def expected_ranks(tree, part, k):
    return [np.array([k if O.far_columns(tree, part, l, t).size else 0 for t in range(1 << l)])
            for l in range(tree.L + 1)]


def planted_case(h2, adm, k=4, n=16, leaf=16, seed=3):
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, adm, 0.7)
    A = planted.planted_h2(tree, part, k, 2, seed)
    At = A[np.ix_(tree.perm, tree.perm)]
    ho = O.compress_dense(tree, part, At, O.basis_threshold(1e-13, np.linalg.norm(A, 2), 1 << tree.L), 48)
    gtree = h2.Tree(W.grid_coords(n), leaf, adm, 0.7)
    G = h2.H2.from_factors(gtree, *factors.oracle_to_import(ho))
    return tree, part, A, ho, G


@pytest.mark.parametrize("adm,r", [(ADM_STRONG, 3), (ADM_WEAK, 3), (ADM_STRONG, 8)])
def test_update_planted_rank_k_plus_r(h2, adm, r):
    tree, part, A, ho, G = planted_case(h2, adm)
    rng = np.random.default_rng(21)
    B = rng.standard_normal((tree.N, r)) / np.sqrt(tree.N)
    At = A + B @ B.T
    nrm = float(np.linalg.norm(At, 2))
    Gu = G.lowrank_update(dev_cols(B), r, 1e-13, opts=h2.default_opts(kmax=48, norm_est=nrm))
    assert Gu.status == 0
    rk = ranks_of(Gu, tree.L)
    want = expected_ranks(tree, part, 4 + r)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(rk[l], want[l])
    Ag = gpu_dense(Gu, tree.N)
    err = np.linalg.norm(Ag - At, 2) / nrm
    hu, _, _ = O.lowrank_update(ho, B, 1e-13, 48, norm_est=nrm)
    d = np.linalg.norm(Ag - O.expand_dense(hu), 2) / nrm
    print(f"planted adm={adm} r={r}: ||A~_gpu - (A + BB^T)|| = {err:.1e}, vs oracle update {d:.1e}")
    assert err <= 1e-12 and d <= 1e-12


def test_downdate_planted(h2):
    tree, part, A, ho, G = planted_case(h2, ADM_STRONG)
    rng = np.random.default_rng(22)
    B = rng.standard_normal((tree.N, 5)) / np.sqrt(tree.N)
    nrm = float(np.linalg.norm(A, 2))
    opts = h2.default_opts(kmax=48, norm_est=nrm)
    Bd = dev_cols(B)
    Gu = G.lowrank_update(Bd, 5, 1e-13, opts=opts)
    Gd = Gu.lowrank_update(Bd, 5, 1e-13, M=-np.eye(5), opts=opts)
    rk = ranks_of(Gd, tree.L)
    want = expected_ranks(tree, part, 4)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(rk[l], want[l])
    assert np.linalg.norm(gpu_dense(Gd, tree.N) - A, 2) <= 1e-12 * nrm


def test_update_general_m_matches_oracle(h2):
    tree, part, A, ho, G = planted_case(h2, ADM_STRONG)
    rng = np.random.default_rng(23)
    r = 4
    B = rng.standard_normal((tree.N, r)) / np.sqrt(tree.N)
    M = rng.standard_normal((r, r))
    Ms = 0.5 * (M + M.T)
    nrm = float(np.linalg.norm(A + B @ Ms @ B.T, 2))
    Gu = G.lowrank_update(dev_cols(B), r, 1e-13, M=M, opts=h2.default_opts(kmax=48, norm_est=nrm))
    hu, _, _ = O.lowrank_update(ho, B, 1e-13, 48, M=M, norm_est=nrm)
    X = np.random.default_rng(3).standard_normal((tree.N, 7))
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Yd = torch.empty_like(Xd)
    Gu.matvec(Xd, Yd, 7)
    torch.cuda.synchronize()
    assert_elementwise(Yd.cpu().numpy().T, O.matvec(hu, X), leaf_index_sets(tree), 1e-12, "general M")


def test_recompression_only(h2):
    # r = 0: recompression of A alone at a tight tolerance keeps every rank and the matrix
    tree, part, A, ho, G = planted_case(h2, ADM_STRONG)
    nrm = float(np.linalg.norm(A, 2))
    Gr = G.lowrank_update(None, 0, 1e-13, opts=h2.default_opts(kmax=48, norm_est=nrm))
    rk = ranks_of(Gr, tree.L)
    want = expected_ranks(tree, part, 4)
    for l in range(tree.L + 1):
        np.testing.assert_array_equal(rk[l], want[l])
    assert np.linalg.norm(gpu_dense(Gr, tree.N) - A, 2) <= 1e-12 * nrm


def test_update_rejects_oversized(h2):
    tree, part, A, ho, G = planted_case(h2, ADM_STRONG)
    B = torch.zeros((141, tree.N), dtype=torch.float64, device="cuda")
    with pytest.raises(h2.H2Error):
        G.lowrank_update(B, 141, 1e-6)   # largest rank 4 + 141 > 144
    with pytest.raises(h2.H2Error):
        G.lowrank_update(B, 2, 1e-6, opts=h2.default_opts(kmax=49))


def _heat_case(h2, n=32, r=4):
    c = W.SMALL_N32
    p = c["problem"]
    mask = W.sensor_mask(n * n, p.m, p.sensor_seed)
    gop = h2.HeatOperator(n, p.kappa, p.T, p.sigma, mask)
    gtree = h2.Tree(W.grid_coords(n), 32, ADM_STRONG, 0.7)
    G = h2.H2.build(gop, gtree, 1e-6, h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=256, seed=7))
    tree = ClusterTree(W.grid_coords(n), 32)
    part = Partition(tree, ADM_STRONG, 0.7)
    ho = factors.import_to_oracle(tree, part, *G.export())
    rng = np.random.default_rng(31)
    # a rank-r update of the size of the Hessian's leading eigenvalues
    B = rng.standard_normal((n * n, r)) * np.sqrt(G.stats()["norm_est"] / (n * n))
    return tree, part, G, ho, B


def test_update_heat_ranks_and_replay(h2):
    tree, part, G, ho, B = _heat_case(h2)
    r = B.shape[1]
    Gu = G.lowrank_update(dev_cols(B), r, 1e-6, opts=h2.default_opts(kmax=32))
    st = Gu.stats()
    nrm = st["norm_est"]
    L = tree.L
    rk = ranks_of(Gu, L)
    hu, _, tau = O.lowrank_update(ho, B, 1e-6, 32, norm_est=nrm)
    assert abs(tau - st["tau_basis"]) <= 1e-14 * tau
    diff = 0
    for l in range(1, L + 1):
        for t in range(1 << l):
            if rk[l][t] != hu.k[l][t]:
                s = hu.sv[(l, t)]
                k = int(min(rk[l][t], hu.k[l][t]))
                # only a singular value within rounding of the threshold may fall either way
                assert abs(s[k] - tau) <= 1e-9 * s[0], (l, t, rk[l][t], hu.k[l][t])
                diff += 1
    hr, _, _ = O.lowrank_update(ho, B, 1e-6, 32, norm_est=nrm, ranks=rk)
    Ag = gpu_dense(Gu, tree.N)
    d = np.linalg.norm(Ag - O.expand_dense(hr), 2) / nrm
    At = O.expand_dense(ho) + B @ B.T
    err = np.linalg.norm(Ag - At, 2) / np.linalg.norm(At, 2)
    print(f"heat 32^2 + rank {r}: {diff} rank decisions differ; ||A~_gpu - A~_oracle|| / ||A~|| = {d:.1e}; "
          f"recompression error {err:.1e} (tol 1e-6)")
    assert d <= 1e-12
    assert err <= 1e-6


def test_update_norm_estimate_matches_oracle(h2):
    tree, part, G, ho, B = _heat_case(h2)
    Gu = G.lowrank_update(dev_cols(B), B.shape[1], 1e-6, opts=h2.default_opts(kmax=32))
    _, nrm_o, _ = O.lowrank_update(ho, B, 1e-6, 32)
    nrm_g = Gu.stats()["norm_est"]
    print(f"norm estimate: gpu {nrm_g:.15e} oracle {nrm_o:.15e}")
    assert abs(nrm_g - nrm_o) <= 1e-9 * nrm_o


def test_update_single_leaf(h2):
    """A tree of one leaf: no far blocks, the update lands in the one dense block."""
    n = 4
    tree = ClusterTree(W.grid_coords(n), 16)
    part = Partition(tree, ADM_STRONG, 0.7)
    A = planted.planted_h2(tree, part, 2, 2, 5)
    ho = O.compress_dense(tree, part, A[np.ix_(tree.perm, tree.perm)], 1e-13, 8)
    G = h2.H2.from_factors(h2.Tree(W.grid_coords(n), 16, ADM_STRONG, 0.7), *factors.oracle_to_import(ho))
    B = np.random.default_rng(4).standard_normal((n * n, 2))
    Gu = G.lowrank_update(dev_cols(B), 2, 1e-10, opts=h2.default_opts(kmax=8, norm_est=1.0))
    assert np.abs(gpu_dense(Gu, n * n) - (A + B @ B.T)).max() <= 1e-13 * np.abs(A + B @ B.T).max()


def test_update_result_keeps_fp32_copy(h2):
    """The updated handle keeps the requested FP32 copy: its compensated FP32 product agrees with
    its FP64 product within 1e-6."""
    tree, part, A, ho, G = planted_case(h2, ADM_STRONG)
    B = np.random.default_rng(6).standard_normal((tree.N, 3)) / np.sqrt(tree.N)
    nrm = float(np.linalg.norm(A + B @ B.T, 2))
    Gu = G.lowrank_update(dev_cols(B), 3, 1e-13, opts=h2.default_opts(kmax=48, norm_est=nrm, keep_fp32=1, keep_bf16=1))
    X = torch.randn((5, tree.N), dtype=torch.float64, device="cuda")
    Y64 = torch.empty_like(X)
    Gu.matvec(X, Y64, 5, h2.H2_FP64)
    Yc = torch.empty_like(X)
    Gu.matvec(X, Yc, 5, h2.H2_FP32C)
    torch.cuda.synchronize()
    assert float((Yc - Y64).norm() / Y64.norm()) <= 1e-6

