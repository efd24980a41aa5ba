"""FP64 construction parity at rounding level: rank replay, and builds at a tight tolerance.

Rank replay (oracle `replay_build`): the GPU construction's decisions -- the 2-norm estimate,
the range-probe count of every level and the basis rank of every box -- are handed to the
oracle as data, and the oracle runs the method with exactly those decisions.  With the
decisions equal, the two constructions compute the same matrix in two independent ways (GPU:
block Gram-Schmidt + shared-memory QR for the sampled ranges, stacked Householder QR and
one-sided Jacobi SVD for the recompression; oracle: numpy Householder QR and LAPACK SVD), and
their H^2 matrices must agree to rounding.  Both sides orthonormalise every sampled block
into the Q factor of its thin QR with a non-negative diagonal of R, so that the range basis
itself (not only its span) is fixed by the samples: the projection pass applies all sibling
blocks' bases at once, and the coarse levels' residual couples each basis vector into the
pieces.  Bounds: 1e-12 relative in the 2-norm at 32^2; 2e-11 at 64^2 adaptive, where the
finest levels draw more probes than the sampled blocks' numerical rank and the oracle itself
moves by 4e-12 (pinned between 1e-12 and 1e-11 by test_replay_sensitivity_adaptive_64) when
its operator products are perturbed at the level of one rounding.  The test also reports the
smallest relative gap between the last kept and the first dropped singular value, so that a
near-tie at a truncation would be visible.

Tight tolerance: a planted H^2 matrix with geometrically graded far-field singular values and
the 32^2 heat Hessian are built at tol 1e-9.  Dozens of kept singular values then lie below
sqrt(eps) * sigma_max, where a truncation through a Gram matrix cannot resolve them; the
construction must meet the tolerance against the dense matrix.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle.tree import ADM_STRONG, ADM_WEAK, ClusterTree, Partition

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


def gpu_dense(h2, G, N):
    """The GPU H^2 matrix as a dense array: its FP64 matvec applied to the identity."""
    I = torch.eye(N, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(I)
    G.matvec(I, Y, N, h2.H2_FP64)
    torch.cuda.synchronize()
    return Y.cpu().numpy().T


def split_ranks(flat, L):
    out, o = [], 0
    for l in range(L + 1):
        out.append(np.asarray(flat[o:o + (1 << l)], dtype=np.int64))
        o += 1 << l
    return out


def _problem(kind):
    if kind == "heat32_strong":
        c = W.SMALL_N32
        p, b = c["problem"], c["build"]
        return p.n, p.m, p.sensor_seed, p.kappa, dict(leaf=b.leaf, adm=ADM_STRONG, tol=b.tol, kmax=b.kmax, q0=b.q0,
                                                      b_inc=b.b_inc, q_max=b.q_max, adaptive=b.adaptive, seed=b.seed)
    if kind == "heat32_weak":
        c = W.SMALL_N32
        p, b = c["problem"], c["build"]
        return p.n, p.m, p.sensor_seed, p.kappa, dict(leaf=b.leaf, adm=ADM_WEAK, tol=b.tol, kmax=b.kmax, q0=b.q0,
                                                      b_inc=b.b_inc, q_max=b.q_max, adaptive=b.adaptive, seed=b.seed)
    if kind == "heat64_adaptive":
        return 64, 256, 1002, 0.01, dict(leaf=64, adm=ADM_STRONG, tol=1e-6, kmax=32, q0=32, b_inc=16, q_max=256,
                                         adaptive=True, seed=7)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,bound", [("heat32_strong", 1e-12), ("heat32_weak", 1e-12), ("heat64_adaptive", 2e-11)])
def test_rank_replay_parity(h2, kind, bound):
    n, m, sseed, kappa, b = _problem(kind)
    N = n * n
    mask = W.sensor_mask(N, m, sseed)
    gop = h2.HeatOperator(n, kappa, 0.5, 0.01, mask)
    tree = h2.Tree(W.grid_coords(n), b["leaf"], b["adm"], 0.7)
    opts = h2.default_opts(kmax=b["kmax"], q0=b["q0"], b_inc=b["b_inc"], q_max=b["q_max"],
                           adaptive=int(b["adaptive"]), seed=b["seed"])
    G = h2.H2.build(gop, tree, b["tol"], opts)
    st = G.stats()
    L = st["levels"]
    ranks = split_ranks(G.export()[0], L)
    op = O.HeatHessian(n, kappa, 0.5, 0.01, mask)
    ho, res = O.replay_build(op, W.grid_coords(n), b["leaf"], b["adm"], 0.7, b["tol"], b["kmax"], b["seed"],
                             st["norm_est"], st["range_probes"][:L + 1], ranks)
    assert res.samples == st["samples"]
    for l in range(L + 1):
        np.testing.assert_array_equal(ho.k[l], ranks[l])
    # the smallest relative gap between the last kept and the first dropped singular value
    gaps = [(s[k - 1] - s[k]) / s[k - 1] for (l, t), s in ho.sv.items()
            for k in [int(ranks[l][t])] if 0 < k < len(s)]
    A_gpu = gpu_dense(h2, G, N)
    A_or = O.expand_dense(ho)
    d = np.linalg.norm(A_gpu - A_or, 2) / st["norm_est"]
    print(f"{kind}: ||H2_gpu - H2_oracle||_2 / ||H||_2 = {d:.2e}, smallest gap at the cut "
          f"{min(gaps) if gaps else float('nan'):.1e}")
    assert d <= bound


def test_tight_tolerance_graded_planted(h2):
    n, leaf = 16, 16
    tree = ClusterTree(W.grid_coords(n), leaf)
    A = planted.planted_h2(tree, Partition(tree, ADM_STRONG, 0.7), 14, 2, 4, grade=0.2)
    nrm = float(np.linalg.norm(A, 2))
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dop = h2.DenseOperator(Ad)
    gtree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    G = h2.H2.build(dop, gtree, 1e-9, h2.default_opts(kmax=32, q0=16, b_inc=16, q_max=256, seed=5, norm_est=nrm))
    err = np.linalg.norm(gpu_dense(h2, G, n * n) - A, 2) / nrm
    print(f"graded planted, tol 1e-9: ||A - H2_gpu||_2 / ||A||_2 = {err:.2e}")
    assert G.stats()["tol_met"] == 1
    assert err <= 1e-9


def test_tight_tolerance_heat32(h2):
    c = W.SMALL_N32
    p = c["problem"]
    mask = W.sensor_mask(p.N, p.m, p.sensor_seed)
    gop = h2.HeatOperator(p.n, p.kappa, p.T, p.sigma, mask)
    tree = h2.Tree(W.grid_coords(p.n), 32, ADM_STRONG, 0.7)
    G = h2.H2.build(gop, tree, 1e-9, h2.default_opts(kmax=48, q0=32, b_inc=16, q_max=256, seed=7))
    H = O.HeatHessian(p.n, p.kappa, p.T, p.sigma, mask)(np.eye(p.N))
    err = np.linalg.norm(gpu_dense(h2, G, p.N) - H, 2) / np.linalg.norm(H, 2)
    print(f"heat 32^2, tol 1e-9: ||H - H2_gpu||_2 / ||H||_2 = {err:.2e}")
    assert G.stats()["tol_met"] == 1
    assert err <= 1e-9


@pytest.mark.parametrize("n,m,sseed,leaf,q0,bound", [(32, 200, 17, 32, 16, 1e-12), (64, 256, 1002, 64, 32, 2e-11)])
def test_certified_bases_parity(h2, n, m, sseed, leaf, q0, bound):
    """Certified range bases (the passing test's columns left out): the GPU takes the oracle's
    decisions (range and projection probes per level), and with its decisions replayed -- the
    certified basis sizes as the probe counts, since the probes are indexed by column -- the two
    H^2 matrices agree to the replay bounds above; the construction meets the tolerance with
    fewer products than the default bases."""
    N, kappa, tol = n * n, 0.01, 1e-6
    mask = W.sensor_mask(N, m, sseed)
    gop = h2.HeatOperator(n, kappa, 0.5, 0.01, mask)
    tree = h2.Tree(W.grid_coords(n), leaf, ADM_STRONG, 0.7)
    mk = lambda c: h2.default_opts(kmax=32, q0=q0, b_inc=16, q_max=256, seed=7, certified=c)
    G = h2.H2.build(gop, tree, tol, mk(1))
    st = G.stats()
    L = st["levels"]
    G0 = h2.H2.build(gop, tree, tol, mk(0))
    op = O.HeatHessian(n, kappa, 0.5, 0.01, mask)
    _, r0 = O.build(op, W.grid_coords(n), leaf, ADM_STRONG, 0.7, tol, 32, q0, 16, 256, True, 7,
                    norm_est=st["norm_est"], certified=True)
    for l in range(1, L + 1):
        assert st["range_probes"][l] == r0.range_probes[l]
        assert st["proj_probes"][l] == r0.proj_probes[l]
    assert st["samples"] < G0.stats()["samples"]
    ranks = split_ranks(G.export()[0], L)
    probes = [0 if st["range_probes"][l] == 0 else st["proj_probes"][l] for l in range(L + 1)]
    ho, _ = O.replay_build(op, W.grid_coords(n), leaf, ADM_STRONG, 0.7, tol, 32, 7, st["norm_est"], probes, ranks)
    for l in range(L + 1):
        np.testing.assert_array_equal(ho.k[l], ranks[l])
    A_gpu = gpu_dense(h2, G, N)
    d = np.linalg.norm(A_gpu - O.expand_dense(ho), 2) / st["norm_est"]
    H = op(np.eye(N))
    err = np.linalg.norm(A_gpu - H, 2) / np.linalg.norm(H, 2)
    print(f"certified {n}^2: products {st['samples']} (default {G0.stats()['samples']}), "
          f"||H2_gpu - H2_oracle|| / ||H|| = {d:.1e} (replayed), error {err:.1e}")
    assert d <= bound
    assert err <= tol
