"""GPU parity of the hybrid construction (global low-rank piece first, H^2 on the residual,
recompression with the global piece; Section 3.3, end) against the oracle on the same seeded
inputs: probe counts of the global range finder and of every level, operator products, ranks,
exact recovery of planted matrices, and the operator action on the heat Hessian."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ClusterTree, Partition

import planted
from test_gpu_parity import _heat_problem, dev, gpu_apply, h2, host, norm2_rel, rel  # noqa: F401

pytestmark = pytest.mark.gpu


def _builds(h2, A_or_op, gop, n, leaf, tol, kmax, q0, global_rank, norm_est=0.0, seed=5):
    tree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    opts = h2.default_opts(kmax=kmax, q0=q0, b_inc=16, q_max=256, adaptive=1, seed=seed, norm_est=norm_est,
                           global_rank=global_rank)
    G = h2.H2.build(gop, tree, tol, opts)
    ho, res = O.build(A_or_op, W.grid_coords(n), leaf, ADM_STRONG, 0.7, tol, kmax, q0, 16, 256, True, seed,
                      norm_est=(norm_est or None), global_rank=global_rank)
    return G, ho, res


def _check_counts(st, ho, res):
    assert st["samples"] == res.samples - res.norm_its
    assert st["range_probes"][0] == res.global_rank
    assert st["range_calls"][0] == res.global_calls
    assert st["range_passed"][0] == res.global_passed
    assert st["proj_probes"][0] == res.global_rank
    for l in range(1, ho.tree.L + 1):
        assert st["range_probes"][l] == res.range_probes[l]
        assert st["proj_probes"][l] == res.proj_probes[l]
        assert st["range_passed"][l] == res.passed[l]
        assert st["max_rank"][l] == int(ho.k[l].max())


def test_hybrid_global_low_rank_recovered_by_global_piece(h2):
    n = 24
    A = planted.global_low_rank(n * n, 9, 1)
    dop = h2.DenseOperator(torch.from_numpy(np.ascontiguousarray(A.T)).cuda())
    nrm = float(np.linalg.norm(A, 2))
    G, ho, res = _builds(h2, O.DenseOperator(A), dop, n, 16, 1e-6, 16, 32, 64, norm_est=nrm)
    st = G.stats()
    _check_counts(st, ho, res)
    assert st["range_passed"][0] == 1 and st["samples"] == 96
    assert all(st["range_passed"][l] == 2 for l in range(1, ho.tree.L + 1))
    X = W.rhs(n * n, 6, 2)
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    G.matvec(Xd, Yd, 6)
    torch.cuda.synchronize()
    assert rel(host(Yd), A @ X) < 1e-12


def test_hybrid_residual_route_recovers_planted(h2):
    n, leaf = 16, 8
    tree = ClusterTree(W.grid_coords(n), leaf)
    A = planted.planted_h2(tree, Partition(tree, ADM_STRONG, 0.7), 3, 2, 4) + planted.global_low_rank(n * n, 5, 8)
    dop = h2.DenseOperator(torch.from_numpy(np.ascontiguousarray(A.T)).cuda())
    nrm = float(np.linalg.norm(A, 2))
    G, ho, res = _builds(h2, O.DenseOperator(A), dop, n, leaf, 1e-6, 32, 16, 32, norm_est=nrm)
    st = G.stats()
    _check_counts(st, ho, res)
    assert st["range_passed"][0] == 0
    X = W.rhs(n * n, 5, 3)
    Xd = dev(X)
    Yd = torch.empty_like(Xd)
    G.matvec(Xd, Yd, 5)
    torch.cuda.synchronize()
    assert rel(host(Yd), A @ X) < 1e-12


@pytest.mark.parametrize("n,m,budget", [(32, 200, 256), (32, 200, 64), (64, 256, 192)])
def test_hybrid_heat_matches_oracle(h2, n, m, budget):
    """Covered (budget above the global rank: no level sampled) and residual routes."""
    mask, op = _heat_problem(n, m, 21)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    leaf = 32 if n == 32 else 64
    G, ho, res = _builds(h2, op, gop, n, leaf, 1e-6, 32, 32, budget, seed=7)
    st = G.stats()
    _check_counts(st, ho, res)
    assert abs(st["norm_est"] - res.norm_est) <= 1e-10 * res.norm_est
    g = gpu_apply(h2, G, n * n)
    assert norm2_rel(g, op, n * n, res.norm_est) < 1e-6
    assert norm2_rel(g, lambda v: O.matvec(ho, v), n * n, res.norm_est) < 1e-6
    if budget >= 192:
        assert st["range_passed"][0] == 1
        # the plain construction needs more products for the same tolerance
        tree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
        P = h2.H2.build(gop, tree, 1e-6, h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=256, seed=7))
        assert st["samples"] < P.stats()["samples"]
        P.close()
    G.close()


def test_hybrid_argument_errors(h2):
    n = 16
    mask, op = _heat_problem(n, 40, 3)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    tree = h2.Tree(W.grid_coords(n), 16, ADM_STRONG, 0.7)
    for bad in (-1, n * n):
        with pytest.raises(h2.H2Error) as ei:
            h2.H2.build(gop, tree, 1e-6, h2.default_opts(global_rank=bad))
        assert ei.value.status == h2.H2_ERR_INVALID_ARG


def test_hybrid_tall_global_panel_two_level_qr(h2):
    """400 x 400 (N = 160,000 rows): the global basis is orthonormalised by the two-level TSQR
    (more than 96 chunks of 1,536 rows).  The global piece alone must meet the tolerance against
    the operator with fewer products than the plain construction."""
    n, m = 400, 4000
    mask = W.sensor_mask(n * n, m, 33)
    gop = h2.HeatOperator(n, 0.01, 0.5, 0.01, mask)
    tree = h2.Tree(W.grid_coords(n), 64, ADM_STRONG, 0.7)
    base = dict(kmax=32, q0=32, b_inc=16, q_max=256, seed=7)
    P = h2.H2.build(gop, tree, 1e-6, h2.default_opts(**base))
    G = h2.H2.build(gop, tree, 1e-6, h2.default_opts(**base, global_rank=384))
    st, sp = G.stats(), P.stats()
    assert st["range_passed"][0] == 1 and st["samples"] < sp["samples"]
    N = n * n

    def op_apply(v):
        vd = torch.from_numpy(np.ascontiguousarray(v)).cuda()
        yd = torch.empty_like(vd)
        gop.apply(vd, yd, 1)
        torch.cuda.synchronize()
        return yd.cpu().numpy()

    assert norm2_rel(gpu_apply(h2, G, N), op_apply, N, st["norm_est"]) < 1e-6
    assert norm2_rel(gpu_apply(h2, G, N), gpu_apply(h2, P, N), N, st["norm_est"]) < 1e-6
    G.close()
    P.close()
