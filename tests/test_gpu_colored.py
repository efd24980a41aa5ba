"""Coloured (strong-structure) sampling on the GPU against the oracle's restatement (Section 3.3).

* Planted H^2 matrix (dense operator, far-block ranks below q): the GPU construction recovers
  every rank and the matrix to rounding, with exactly the oracle's number of products.
* 32^2 heat Hessian: the products (and operator calls) equal the oracle's; with the GPU's rank
  decisions replayed, the GPU and oracle H^2 matrices agree to 1e-10 relative (both orthonormalise
  every sample block into its signed Q factor, so the pieces agree to rounding); the construction
  meets the tolerance against the dense Hessian.
* 64^2 heat Hessian: products equal the plan's, error within the tolerance, and the coloured
  structure costs more products than the weak one (the trade of Section 3.3).
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle import colored as C
from oracle.tree import ADM_STRONG, ClusterTree, Partition

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


def ranks_of(G, L):
    flat = G.export()[0]
    out, o = [], 0
    for l in range(L + 1):
        out.append(np.asarray(flat[o:o + (1 << l)], dtype=np.int64))
        o += 1 << l
    return out


def test_colored_planted(h2):
    n, leaf, q = 16, 16, 8
    tree = ClusterTree(W.grid_coords(n), leaf)
    part = Partition(tree, ADM_STRONG, 0.7)
    A = planted.planted_h2(tree, part, 4, 2, 3)
    nrm = float(np.linalg.norm(A, 2))
    dop = h2.DenseOperator(torch.from_numpy(np.ascontiguousarray(A.T)).cuda())
    gtree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    G = h2.H2.build(dop, gtree, 1e-13, h2.default_opts(kmax=48, q0=q, seed=5, norm_est=nrm,
                                                      sampling=h2.H2_SAMPLING_COLORED))
    st = G.stats()
    plan = C.ColoredPlan(tree, part, q)
    assert st["samples"] == plan.samples()
    rk = ranks_of(G, tree.L)
    for l in range(tree.L + 1):
        want = [4 if O.far_columns(tree, part, l, t).size else 0 for t in range(1 << l)]
        np.testing.assert_array_equal(rk[l], want)
    err = np.linalg.norm(gpu_dense(G, n * n) - A, 2) / nrm
    print(f"coloured planted: ||A - H2_gpu|| / ||A|| = {err:.1e}, products {st['samples']}")
    assert err <= 1e-12


def _heat(h2, n):
    p = W.SMALL_N32["problem"]
    mask = W.sensor_mask(n * n, p.m, p.sensor_seed)
    return (h2.HeatOperator(n, p.kappa, p.T, p.sigma, mask), O.HeatHessian(n, p.kappa, p.T, p.sigma, mask))


def test_colored_heat32_parity(h2):
    n, leaf, q, tol = 32, 32, 16, 1e-6
    gop, op = _heat(h2, n)
    gtree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    G = h2.H2.build(gop, gtree, tol, h2.default_opts(kmax=32, q0=q, seed=7, sampling=h2.H2_SAMPLING_COLORED))
    st = G.stats()
    L = st["levels"]
    rk = ranks_of(G, L)
    ho, res, plan = C.build_colored(op, W.grid_coords(n), leaf, ADM_STRONG, 0.7, tol, 32, q, 7,
                                    norm_est=st["norm_est"], ranks=rk)
    assert st["samples"] == res.samples == plan.samples()
    for l in range(L + 1):
        assert st["range_probes"][l] == plan.range_probes(l)
        assert st["proj_probes"][l] == plan.proj_probes(l)
    Ag = gpu_dense(G, n * n)
    d = np.linalg.norm(Ag - O.expand_dense(ho), 2) / st["norm_est"]
    H = op(np.eye(n * n))
    err = np.linalg.norm(Ag - H, 2) / np.linalg.norm(H, 2)
    print(f"coloured heat 32^2: ||H2_gpu - H2_oracle|| / ||H|| = {d:.1e} (ranks replayed); error {err:.1e}; "
          f"products {st['samples']}")
    assert d <= 1e-10
    assert err <= tol


def test_colored_heat64_products_and_error(h2):
    n, leaf, q, tol = 64, 64, 16, 1e-6
    gop, op = _heat(h2, n)
    gtree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    G = h2.H2.build(gop, gtree, tol, h2.default_opts(kmax=32, q0=q, seed=7, sampling=h2.H2_SAMPLING_COLORED))
    st = G.stats()
    tree = ClusterTree(W.grid_coords(n), leaf)
    plan = C.ColoredPlan(tree, Partition(tree, ADM_STRONG, 0.7), q)
    assert st["samples"] == plan.samples()
    Gw = h2.H2.build(gop, gtree, tol, h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=256, seed=7))
    H = op(np.eye(n * n))
    err = np.linalg.norm(gpu_dense(G, n * n) - H, 2) / np.linalg.norm(H, 2)
    print(f"coloured heat 64^2: products {st['samples']} (weak {Gw.stats()['samples']}), error {err:.1e}")
    assert err <= tol
    assert st["samples"] > Gw.stats()["samples"]


def test_colored_weak_partition(h2):
    """The weak (HSS) partition: every box has one far partner, its sibling, so each level takes
    one colour and one slot, and the products equal the oracle's plan.  Sampling with q fixed
    probes per pair caps every sibling block at rank q: at q = 16 the 32^2 sibling blocks need
    more (the oracle's construction gives the same 3e-3 error), so the GPU is held to the
    oracle's result with its ranks replayed, not to the tolerance."""
    from oracle.tree import ADM_WEAK
    n, leaf, q, tol = 32, 32, 16, 1e-6
    gop, op = _heat(h2, n)
    gtree = h2.Tree(W.grid_coords(n), leaf, ADM_WEAK, 0.7)
    G = h2.H2.build(gop, gtree, tol, h2.default_opts(kmax=48, q0=q, seed=7, sampling=h2.H2_SAMPLING_COLORED))
    st = G.stats()
    L = st["levels"]
    tree = ClusterTree(W.grid_coords(n), leaf)
    plan = C.ColoredPlan(tree, Partition(tree, ADM_WEAK, 0.7), q)
    assert st["samples"] == plan.samples()
    assert all(c <= 1 for c in plan.ncolors) and all(s <= 1 for s in plan.nslots)
    ho, res, _ = C.build_colored(op, W.grid_coords(n), leaf, ADM_WEAK, 0.7, tol, 48, q, 7,
                                 norm_est=st["norm_est"], ranks=ranks_of(G, L))
    assert res.samples == st["samples"]
    Ag = gpu_dense(G, n * n)
    Ao = O.expand_dense(ho)
    d = np.linalg.norm(Ag - Ao, 2) / st["norm_est"]
    H = op(np.eye(n * n))
    nh = np.linalg.norm(H, 2)
    err_g = np.linalg.norm(Ag - H, 2) / nh
    err_o = np.linalg.norm(Ao - H, 2) / nh
    print(f"coloured weak 32^2: products {st['samples']}, ||H2_gpu - H2_oracle|| / ||H|| = {d:.1e} "
          f"(ranks replayed), error {err_g:.1e} (oracle {err_o:.1e})")
    assert d <= 1e-10
    assert abs(err_g - err_o) <= 1e-10
