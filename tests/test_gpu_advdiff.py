"""GPU parity on the second Hessian family (finite-difference advection-diffusion source
inversion, Section 4.3; the factored misfit Hessian Z Z^T / sigma^2): the shipped factored
operator against numpy, and plain and hybrid constructions against the oracle on the same Z."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import advdiff as AD

from test_gpu_parity import gpu_apply, h2, norm2_rel  # noqa: F401

pytestmark = pytest.mark.gpu

SCALE = 1e4   # 1 / sigma^2 for sigma = 0.01


def _operators(h2, n, kappa, n_obs, seed=5):
    Z = AD.hessian_factor(n, kappa, n_obs, seed)
    Zt = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    return Z, h2.LowRankOperator(Zt, SCALE), O.LowRankOperator(Z, SCALE)


def test_lowrank_operator_matches_numpy(h2):
    Z, gop, op = _operators(h2, 20, 1e-2, 37)
    X = np.random.default_rng(1).standard_normal((400, 9))
    Xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
    Yd = torch.empty_like(Xd)
    gop.apply(Xd, Yd, 9)
    torch.cuda.synchronize()
    want = op(X)
    assert np.linalg.norm(Yd.cpu().numpy().T - want) <= 1e-13 * np.linalg.norm(want)


@pytest.mark.parametrize("kappa", [1e-1, 1e-3])
@pytest.mark.parametrize("budget", [0, 512])
def test_advdiff_build_matches_oracle(h2, kappa, budget):
    n, n_obs, tol = 32, 256, 1e-4
    Z, gop, op = _operators(h2, n, kappa, n_obs)
    tree = h2.Tree(AD.coords(n), 32, h2.H2_ADM_STRONG, 0.7)
    G = h2.H2.build(gop, tree, tol, h2.default_opts(kmax=32, q0=32, b_inc=16, q_max=256, seed=7,
                                                    global_rank=budget))
    ho, res = O.build(op, AD.coords(n), 32, O.ADM_STRONG, 0.7, tol, 32, 32, 16, 256, True, 7, global_rank=budget)
    st = G.stats()
    assert st["samples"] == res.samples - res.norm_its
    assert st["range_probes"][0] == res.global_rank and st["range_passed"][0] == res.global_passed
    for l in range(1, ho.tree.L + 1):
        assert st["range_probes"][l] == res.range_probes[l]
        assert st["max_rank"][l] == int(ho.k[l].max())
    N = n * n
    g = gpu_apply(h2, G, N)
    assert norm2_rel(g, op, N, res.norm_est) < tol
    assert norm2_rel(g, lambda v: O.matvec(ho, v), N, res.norm_est) < tol
    G.close()
