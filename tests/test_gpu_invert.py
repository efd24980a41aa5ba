"""Hierarchical hyperpower / Newton-Schulz inversion on the GPU against the oracle (Appendix A).

Both sides invert the same A = H~ + beta I: H~ is the oracle's H^2 of a 16 x 16 heat Hessian,
imported into the library, beta = 0.05 ||H||.  The oracle is given the library's ||A||_2
estimate (so alpha = 1/||A|| is shared); the residual power iterations start from the same
counter-based vector.  Iterate counts and products per iterate must be equal, thresholds and
residual histories equal to 1e-3 (each iterate is itself a construction to eps_k), and the two
inverses within 1e-5 of each other while each meets ||A X - I||_2 <= 2 eps.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from oracle import inverse

import factors

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h2():
    from paper_2003_10173_gb300 import build_lib
    build_lib.build()
    import paper_2003_10173_gb300 as m
    m.lib()
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def problem(h2):
    n, leaf = 16, 16
    mask = W.sensor_mask(n * n, 40, 21)
    H = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    coords = W.grid_coords(n)
    hA, _ = O.build(H, coords, leaf, O.ADM_STRONG, 0.7, 1e-10, 48, 16, 8, 128, True, 5)
    Ad = O.expand_dense(hA)
    beta = 0.05 * np.linalg.norm(Ad, 2)
    tree = h2.Tree(coords, leaf, h2.H2_ADM_STRONG, 0.7)
    GA = h2.H2.from_factors(tree, *factors.oracle_to_import(hA))
    return dict(n=n, leaf=leaf, coords=coords, hA=hA, A=Ad + beta * np.eye(n * n), beta=beta, GA=GA)


def _dense(h2, G, N):
    I = torch.eye(N, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(I)
    G.matvec(I, Y, N)
    torch.cuda.synchronize()
    return Y.cpu().numpy().T


@pytest.mark.parametrize("order,eps_loose", [(2, 1e-3), (4, 1e-3), (2, 1e-6)])
def test_inverse_matches_oracle(h2, problem, order, eps_loose):
    p = problem
    N = p["n"] ** 2
    bopts = h2.default_opts(kmax=32, q0=16, b_inc=8, q_max=128, adaptive=1, seed=7)
    X, st = h2.invert(p["GA"], shift=p["beta"], order=order, eps=1e-6, eps_loose=eps_loose, build_opts=bopts)
    assert st["converged"]
    # a power-iteration estimate stays below the norm; X_0 = I / estimate converges iff alpha lambda_max < 2
    lam = np.linalg.norm(p["A"], 2)
    assert st["norm_A"] <= 1.0001 * lam and st["alpha"] * lam < 2.0
    hA, beta = p["hA"], p["beta"]
    apply_A = lambda v: O.matvec(hA, v) + beta * v
    build = lambda op, tol: O.build(op, p["coords"], p["leaf"], O.ADM_STRONG, 0.7, tol, 32, 16, 8, 128, True, 7)
    res = inverse.hns_invert(apply_A, st["norm_A"], build, N, order=order, eps=1e-6, eps_loose=eps_loose)
    assert st["iterations"] == len(res.eps_k)
    # iterates are constructions to eps_k; two valid constructions differ at that scale, which
    # moves the next residual (and the threshold derived from it) by ~1e-5 relative here
    np.testing.assert_allclose(st["eps_k"], res.eps_k, rtol=1e-3)
    np.testing.assert_allclose(st["err"], res.errors, rtol=1e-3)
    assert st["samples"] == res.samples
    Xg = _dense(h2, X, N)
    Xo = O.expand_dense(res.h2)
    assert np.linalg.norm(Xg - Xo, 2) <= 1e-5 * np.linalg.norm(Xo, 2)
    for Xd in (Xg, Xo):
        assert np.linalg.norm(p["A"] @ Xd - np.eye(N), 2) <= 2e-6


def test_higher_order_and_dynamic_threshold(h2, problem):
    """Appendix A: a dynamic threshold spends fewer products at the same iteration count; a
    higher order needs fewer iterates."""
    p = problem
    bopts = h2.default_opts(kmax=32, q0=16, b_inc=8, q_max=128, adaptive=1, seed=7)
    runs = {}
    for key, order, loose in (("static", 2, 1e-6), ("dynamic", 2, 1e-3), ("order8", 8, 1e-3)):
        X, st = h2.invert(p["GA"], shift=p["beta"], order=order, eps=1e-6, eps_loose=loose, build_opts=bopts)
        assert st["converged"]
        runs[key] = st
    assert runs["static"]["iterations"] == runs["dynamic"]["iterations"]
    assert sum(runs["dynamic"]["samples"]) < sum(runs["static"]["samples"])
    assert runs["order8"]["iterations"] < runs["dynamic"]["iterations"]


def test_invert_argument_errors(h2, problem):
    with pytest.raises(h2.H2Error):
        h2.invert(problem["GA"], order=1)
    with pytest.raises(h2.H2Error):
        h2.invert(problem["GA"], eps=1e-6, eps_loose=1e-8)


@pytest.mark.parametrize("unroll", [2, 3])
def test_unrolled_from_warm_start_matches_oracle(h2, problem, unroll):
    """Appendix A's unrolled iterations: from a warm start X_0 (here a rough inverse from two
    Newton-Schulz iterates, imported on both sides), k Newton-Schulz steps constructed at once
    (X_0 sum_{i<2^k} R_0^i).  GPU and oracle take the same X_0 and ||A||; equal products, residual
    history to 1e-3, inverses within 1e-5, and the residual falls like E_0^(2^k) (down to the
    construction floor)."""
    p = problem
    N = p["n"] ** 2
    bopts = h2.default_opts(kmax=32, q0=16, b_inc=8, q_max=128, adaptive=1, seed=7)
    X0, st0 = h2.invert(p["GA"], shift=p["beta"], eps=1e-6, eps_loose=1e-3, max_iter=2, build_opts=bopts)
    assert st0["iterations"] == 2
    X, st = h2.invert(p["GA"], shift=p["beta"], eps=1e-6, eps_loose=1e-6, build_opts=bopts, x0=X0, unroll=unroll)
    assert st["iterations"] == 1 and len(st["samples"]) >= 1
    hA, beta = p["hA"], p["beta"]
    apply_A = lambda v: O.matvec(hA, v) + beta * v
    build = lambda op, tol: O.build(op, p["coords"], p["leaf"], O.ADM_STRONG, 0.7, tol, 32, 16, 8, 128, True, 7)
    hX0 = factors.import_to_oracle(p["hA"].tree, p["hA"].part, *X0.export())
    res = inverse.hns_invert(apply_A, st["norm_A"], build, N, eps=1e-6, eps_loose=1e-6,
                             x0=(lambda v: O.matvec(hX0, v), X0.stats()["norm_est"]), unroll=unroll)
    assert len(res.samples) == 1 and st["samples"][0] == res.samples[0]
    np.testing.assert_allclose(st["err"][:2], res.errors, rtol=1e-3)
    np.testing.assert_allclose(st["eps_k"][0], res.eps_k[0], rtol=1e-3)
    E0, E1 = st["err"][0], st["err"][1]
    assert E1 <= max(10.0 * E0 ** (1 << unroll), 1e-5)
    Xg = _dense(h2, X, N)
    Xo = O.expand_dense(res.h2)
    assert np.linalg.norm(Xg - Xo, 2) <= 1e-5 * np.linalg.norm(Xo, 2)
