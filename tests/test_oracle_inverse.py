"""Pins of the oracle hierarchical (hyperpower / Newton-Schulz) inversion (CPU only).

Independent of the oracle's own code: on a diagonal matrix the order-l iteration maps the
residual r = 1 - a x to r^l exactly; the order-2 sampler equals the Newton-Schulz formula
(2I - X A) X written out; exact (uncompressed) iterations converge to numpy's inverse; the
residual estimate agrees with numpy's 2-norm; the hierarchical iteration on a small heat
Hessian reaches the target residual and the inverse to the expected accuracy.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle import inverse


def test_diagonal_residual_is_raised_to_the_order():
    a = np.array([0.5, 1.0, 3.0, 10.0])
    x = np.full(4, 0.05)
    for order in (2, 3, 8):
        y = inverse.hyperpower_sample(lambda v: x[:, None] * v, lambda v: a[:, None] * v, np.eye(4), order)
        x1 = np.diag(y)
        np.testing.assert_allclose(1.0 - a * x1, (1.0 - a * x) ** order, rtol=1e-12, atol=1e-15)
        assert np.allclose(y, np.diag(x1))


def test_order_two_is_newton_schulz():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((30, 30))
    A = M @ M.T + 30 * np.eye(30)
    Xm = rng.standard_normal((30, 30))
    X = 0.01 * (Xm + Xm.T)
    om = rng.standard_normal((30, 5))
    y = inverse.hyperpower_sample(lambda v: X @ v, lambda v: A @ v, om, 2)
    np.testing.assert_allclose(y, (2 * np.eye(30) - X @ A) @ X @ om, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("order", [2, 4])
def test_exact_iterations_converge_to_the_inverse(order):
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    A = Q @ np.diag(np.geomspace(1.0, 100.0, 40)) @ Q.T
    res = inverse.hns_invert(lambda v: A @ v, np.linalg.norm(A, 2),
                             lambda op, tol: (_DenseIterate(op(np.eye(40))), _Peel()), 40, order=order, eps=1e-10)
    assert res.errors[-1] <= 1e-10
    X = res.h2.M
    np.testing.assert_allclose(X, np.linalg.inv(A), rtol=0, atol=1e-9)
    # from alpha = 1/||A||: r_0 = 1 - 1/100 on the smallest eigenvalue, r_k = r_0^(order^k)
    k_needed = int(np.ceil(np.log(np.log(1e-10) / np.log(0.99)) / np.log(order)))
    assert abs(len(res.eps_k) - k_needed) <= 1


class _DenseIterate:
    def __init__(self, M):
        self.M = M


class _Peel:
    samples = 0
    norm_its = 0
    norm_est = 1.0


@pytest.fixture(autouse=True)
def _dense_matvec(monkeypatch):
    """Let the iteration apply a dense iterate (used by the exact-iteration test)."""
    orig = inverse.matvec

    def mv(h, v):
        if isinstance(h, _DenseIterate):
            return h.M @ v
        return orig(h, v)
    monkeypatch.setattr(inverse, "matvec", mv)


def test_residual_norm_matches_dense_two_norm():
    rng = np.random.default_rng(8)
    M = rng.standard_normal((50, 50))
    A = M @ M.T / 50 + np.eye(50)
    X = np.linalg.inv(A) + 1e-3 * np.diag(rng.standard_normal(50))
    E = inverse.residual_norm(lambda v: A @ v, lambda v: X @ v, 50, 4, maxit=200, rtol=1e-6)
    assert abs(E - np.linalg.norm(A @ X - np.eye(50), 2)) <= 1e-3 * E


def test_construction_threshold():
    assert inverse.construction_threshold(0.5, 1e-6, 1e-2, 0.1) == 1e-2
    assert inverse.construction_threshold(1e-2, 1e-6, 1e-2, 0.1) == pytest.approx(1e-5)
    assert inverse.construction_threshold(1e-4, 1e-6, 1e-2, 0.1) == 1e-6
    assert inverse.construction_threshold(0.5, 1e-6, 1e-6, 0.1) == 1e-6


def test_hierarchical_inverse_of_regularised_heat_hessian():
    n, leaf = 16, 16
    mask = W.sensor_mask(n * n, 40, 21)
    H = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    Hd = H(np.eye(n * n))
    nH = np.linalg.norm(Hd, 2)
    beta = 0.05 * nH
    A = Hd + beta * np.eye(n * n)
    apply_A = lambda v: A @ v
    coords = W.grid_coords(n)

    def build(op, tol):
        return O.build(op, coords, leaf, O.ADM_STRONG, 0.7, tol, 32, 16, 8, 128, True, 7)

    res = inverse.hns_invert(apply_A, np.linalg.norm(A, 2), build, n * n, order=4, eps=1e-6,
                             eps_loose=1e-3, theta=0.1)
    assert res.errors[-1] <= 1e-6
    assert len(res.eps_k) <= 8
    assert res.eps_k[0] == 1e-3 and res.eps_k[-1] < res.eps_k[0]
    Xd = O.expand_dense(res.h2)
    Ainv = np.linalg.inv(A)
    assert np.linalg.norm(Xd - Ainv, 2) * np.linalg.norm(A, 2) <= 5e-6


def test_unrolled_newton_schulz_equals_iterated_steps():
    """k Newton-Schulz steps from X_0 equal one order-2^k hyperpower step from X_0 (the geometric
    sum of the unrolled iteration), with exact constructions (dense), for k = 1..4; the paper's
    printed binomial form sum_i binom(2^k, i) (-A X_0)^i is a different matrix (a planted check
    that the reading matters)."""
    rng = np.random.default_rng(3)
    n = 40
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1.0, 20.0, n)) @ Q.T
    X0 = 0.9 / 20.0 * np.eye(n) + 0.01 * Q @ np.diag(rng.uniform(0, 1, n)) @ Q.T
    I = np.eye(n)
    for k in range(1, 5):
        X = X0.copy()
        for _ in range(k):
            X = X @ (2 * I - A @ X)
        samp = inverse.hyperpower_sample(lambda v: X0 @ v, lambda v: A @ v, I.copy(), 1 << k)
        assert np.abs(samp - X).max() <= 1e-12 * np.abs(X).max()
        R0 = I - A @ X0
        geo = X0 @ sum(np.linalg.matrix_power(R0, i) for i in range(1 << k))
        assert np.abs(geo - X).max() <= 1e-12 * np.abs(X).max()
        from math import comb
        printed = X0 @ sum(comb(1 << k, i) * np.linalg.matrix_power(-A @ X0, i) for i in range((1 << k) + 1))
        assert np.abs(printed - X).max() > 1e-3 * np.abs(X).max()


def test_unrolled_hierarchical_inverse_from_warm_start():
    """The hierarchical driver with x0 and unroll: one construction, residual E_1 ~ E_0^(2^k)."""
    n = 16
    mask = W.sensor_mask(n * n, 40, 3)
    op = O.HeatHessian(n, 0.01, 0.5, 0.01, mask)
    Hd = op(np.eye(n * n))
    shift = 0.05 * np.linalg.norm(Hd, 2)
    A = Hd + shift * np.eye(n * n)
    nA = float(np.linalg.norm(A, 2))
    coords = W.grid_coords(n)

    def build(sampler, tol):
        return O.build(sampler, coords, 32, O.ADM_STRONG, 0.7, tol, 48, 32, 16, 256, True, 5)

    # warm start: a rough inverse from two Newton-Schulz steps
    rough = inverse.hns_invert(lambda v: A @ v, nA, build, n * n, eps=1e-12, max_iter=2)
    X0 = rough.h2
    E0 = rough.errors[-1]
    res = inverse.hns_invert(lambda v: A @ v, nA, build, n * n, eps=1e-9, x0=(lambda v: O.matvec(X0, v), nA ** -1),
                           unroll=3)
    assert len(res.samples) == 1
    assert res.errors[0] == pytest.approx(E0, rel=1e-6)
    assert res.errors[1] <= max(10 * E0 ** 8, 1e-7)
