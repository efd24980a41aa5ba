"""Pins of the oracle rank model and of the predicted-start peeling (CPU only).

The rank model is a plain 3-layer MLP; what fixes it independently of its own code:
the exact GELU (erf form, scipy) bounds the tanh form, central finite differences
fix every gradient entry, torch.optim.Adam (a library routine) fixes the optimiser,
torch's float32 -> bfloat16 conversion fixes the weight rounding, and the affine
limit of GELU reduces the forward pass to a chain of matrix products.  The
predicted-start peeling is pinned on a global rank-r matrix, where the number of
operator calls and probes at every level follows from r alone.
"""
import numpy as np
import pytest
import scipy.special as sp
import torch

from oracle import mlp
from oracle.peel import peel
from oracle.tree import ClusterTree
from oracle.heat import DenseOperator
from workloads import grid_coords

import planted


def _params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(mlp.NPARAM) * scale


def test_gelu_against_erf_form_and_odd_identity():
    u = np.linspace(-8.0, 8.0, 20001)
    exact = 0.5 * u * (1.0 + sp.erf(u / np.sqrt(2.0)))
    assert np.abs(mlp.gelu(u) - exact).max() < 5e-4
    # gelu(u) - gelu(-u) = u for the tanh form as for the exact one (tanh is odd)
    np.testing.assert_allclose(mlp.gelu(u) - mlp.gelu(-u), u, rtol=0, atol=1e-12)
    assert mlp.gelu(np.array([0.0]))[0] == 0.0


def test_gelu_grad_finite_differences():
    u = np.linspace(-6.0, 6.0, 1201)
    h = 1e-6
    fd = (mlp.gelu(u + h) - mlp.gelu(u - h)) / (2 * h)
    np.testing.assert_allclose(mlp.gelu_grad(u), fd, rtol=0, atol=1e-8)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.standard_normal(5000).astype(np.float32),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, 65504.0,
                                  1e-30, -3.0e38], dtype=np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.to_bf16(x), want)
    # ties go to even: 1 + 2^-8 lies halfway between 1 and 1 + 2^-7
    assert mlp.to_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0


def test_forward_affine_limit_is_matrix_chain():
    # with large positive pre-activations gelu(u) = u in FP64, so the network is affine
    rng = np.random.default_rng(5)
    p = _params(5, 0.01)
    W1, b1, W2, b2, W3, b3 = mlp.split(p)
    b1[:] = 60.0
    b2[:] = 60.0
    X = rng.uniform(-1, 1, (17, mlp.F))
    y, _ = mlp.forward(p, X)
    want = ((X @ W1.T + 60.0) @ W2.T + 60.0) @ W3 + b3[0]
    np.testing.assert_allclose(y, want, rtol=1e-13, atol=1e-12)


def test_forward_constant_hidden_layers():
    p = np.zeros(mlp.NPARAM)
    W1, b1, W2, b2, W3, b3 = mlp.split(p)
    b1[:] = 0.7
    b2[:] = -0.4
    W3[:] = np.arange(mlp.H) / mlp.H
    b3[0] = 0.25
    X = np.random.default_rng(0).standard_normal((5, mlp.F))
    y, _ = mlp.forward(p, X)
    g = 0.5 * -0.4 * (1 + np.tanh(np.sqrt(2 / np.pi) * (-0.4 + 0.044715 * (-0.4) ** 3)))
    np.testing.assert_allclose(y, np.full(5, g * W3.sum() + 0.25), rtol=1e-14)


@pytest.mark.parametrize("bf16", [False, True])
def test_gradient_central_differences(bf16):
    rng = np.random.default_rng(11)
    p = _params(12)
    if bf16:
        p = mlp.to_bf16(p)            # a point where the bf16 rounding is locally the identity
    X = rng.uniform(-1, 1, (37, mlp.F))
    t = rng.standard_normal(37)
    _, g = mlp.loss_and_grad(p, X, t, bf16=False)
    idx = rng.choice(mlp.NPARAM, 400, replace=False)
    idx = np.union1d(idx, [0, mlp.H * mlp.F, mlp.NPARAM - 1, mlp.NPARAM - 2])
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, X, t)[0] - mlp.loss_and_grad(p - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(g[i])), i
    if bf16:
        # the bf16 mode differentiates at the rounded weights
        l1, g1 = mlp.loss_and_grad(p, X, t, bf16=True)
        l2, g2 = mlp.loss_and_grad(mlp.to_bf16(p), X, t, bf16=False)
        assert l1 == l2 and np.array_equal(g1, g2)


def test_adam_matches_torch():
    rng = np.random.default_rng(21)
    p0 = rng.standard_normal(50)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 8):
        g = rng.standard_normal(50) * 10.0 ** rng.uniform(-3, 1, 50)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = mlp.adam_step(p, m, v, g, step, lr=1e-2)
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_adam_constant_gradient_moves_lr_per_step():
    # bias correction makes m_hat = g and v_hat = g^2 exactly for a constant gradient
    g = np.array([3.0, -0.5, 1e-3])
    p, m, v = np.zeros(3), np.zeros(3), np.zeros(3)
    for step in range(1, 30):
        p, m, v = mlp.adam_step(p, m, v, g, step, lr=0.01)
    np.testing.assert_allclose(p, -29 * 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-10)


def test_training_reduces_loss():
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (512, mlp.F))
    t = np.sin(2 * X[:, 0]) + X[:, 1] * X[:, 2] + 0.5 * X[:, 3] ** 2
    p = _params(6, 0.2)
    m, v = np.zeros_like(p), np.zeros_like(p)
    l0 = mlp.loss_and_grad(p, X, t)[0]
    for step in range(1, 401):
        idx = rng.choice(512, 64, replace=False)
        _, g = mlp.loss_and_grad(p, X[idx], t[idx], bf16=True)
        p, m, v = mlp.adam_step(p, m, v, g, step, lr=3e-3)
    assert mlp.loss_and_grad(p, X, t, bf16=True)[0] < 0.1 * l0


def test_level_features_closed_form_4x4():
    tree = ClusterTree(grid_coords(4), 4)       # L = 2: 8-point columns, then 2 x 2 boxes
    f = mlp.level_features(tree, kappa_T=0.01, density=0.25, tol=1e-6)
    assert f.shape == (3, mlp.F)
    root = 0.6 * np.sqrt(2.0)
    np.testing.assert_allclose(f[:, 0], [0.0, 0.5, 1.0])
    np.testing.assert_allclose(f[:, 1], np.log2([16, 8, 4]) / 20)
    np.testing.assert_allclose(f[:, 2], [1.0, np.sqrt(0.4) / root, 0.2 * np.sqrt(2) / root], rtol=1e-14)
    np.testing.assert_allclose(f[:, 3], -0.5)
    np.testing.assert_allclose(f[:, 4], 0.25)
    np.testing.assert_allclose(f[:, 5], -0.6)
    np.testing.assert_allclose(f[:, 6], np.log10(0.1 / np.array([root, np.sqrt(0.4), 0.2 * np.sqrt(2)])) / 2,
                               rtol=1e-13)
    np.testing.assert_allclose(f[:, 7], 0.2)


def test_q_start_rounding():
    assert mlp.q_start_from_prediction(np.log2(25.0), 8, 256) == 32      # 25 - 1 + 8
    assert mlp.q_start_from_prediction(np.log2(21.0), 8, 256) == 32      # 28 -> 32
    assert mlp.q_start_from_prediction(np.log2(25.5), 8, 256) == 40      # ceil -> 26: 33 -> 40
    assert mlp.q_start_from_prediction(0.0, 8, 256) == 8
    assert mlp.q_start_from_prediction(-3.0, 0, 256) == 8
    assert mlp.q_start_from_prediction(12.0, 8, 256) == 256


# ------------------------------------------------- predicted start counts in the peeling

def _lowrank_setup(r=9):
    tree = ClusterTree(grid_coords(24), 36)      # N = 576, L = 4, boxes 288 .. 36
    A = planted.global_low_rank(tree.N, r, 1)
    return tree, DenseOperator(A), A


def test_adaptive_need_is_first_increment_above_rank():
    tree, op, A = _lowrank_setup()
    res = peel(op, tree, 1e-8, 4, 4, 64, True, 7)
    for l in range(1, tree.L + 1):
        # tests against Q of 4 and 8 columns fail (rank 9), against 12 columns pass; the start
        # block and the first test batch share one call
        assert res.passed[l] == 1
        assert res.need[l] == 12
        assert res.range_calls[l] == 3
        assert res.range_probes[l] == 16


@pytest.mark.parametrize("start,calls,probes,need", [(9, 1, 13, 9), (6, 2, 14, 10)])
def test_predicted_start_counts(start, calls, probes, need):
    tree, op, A = _lowrank_setup()
    ql = [0] + [start] * tree.L
    res = peel(op, tree, 1e-8, 4, 4, 64, True, 7, q_level=ql, q_test=4)
    for l in range(1, tree.L + 1):
        assert res.passed[l] == 1
        assert res.range_calls[l] == calls
        assert res.range_probes[l] == probes
        assert res.need[l] == need
    # the pieces reproduce the rank-9 matrix: the leaf pass sees only rounding
    Np = tree.N
    r0 = tree.rows(tree.L, 0)
    Om = np.eye(Np)[:, r0]
    from oracle.peel import TreeOperator, apply_pieces
    opt = TreeOperator(DenseOperator(A), tree)
    Ap = opt(Om)
    Kp = apply_pieces(res.pieces, range(1, tree.L + 1), tree, Om)
    # outside leaf 0, the columns of leaf 0 are fully captured by the pieces
    mask = np.ones(Np, bool)
    mask[r0] = False
    assert np.abs((Ap - Kp)[mask]).max() < 1e-10 * np.abs(A).max()


def test_predicted_start_above_box_size_uses_identity():
    tree, op, A = _lowrank_setup()
    res = peel(op, tree, 1e-8, 4, 4, 64, True, 7, q_level=[0, 0, 0, 0, 40], q_test=4)
    assert res.passed[4] == -1 and res.range_probes[4] == 0 and res.range_calls[4] == 0
    assert res.passed[1] == 1 and res.need[1] == 12      # zero entries keep q0
