"""Pins of the second Hessian family's input generator (finite-difference advection-diffusion
source inversion, Section 4.3): the discrete operator is exact on linear functions away from the
boundary (second differences vanish, backward differences are exact), the mirrored outflow ghost
and the Dirichlet inflow act as stated, the adjoint factor solves its system, transport runs along
v = (x, y), and the misfit Hessian is symmetric positive semidefinite of rank n_obs."""
import numpy as np
import pytest

import oracle as O
from workloads import advdiff as AD


@pytest.mark.parametrize("kappa", [1e-1, 1e-3])
def test_operator_exact_on_linear_functions(kappa):
    n = 12
    h = 1.0 / n
    X = AD.coords(n)
    u = 1.0 + 2.0 * X[:, 0] + 3.0 * X[:, 1]
    Au = AD.operator(n, kappa) @ u
    i = np.rint(X[:, 0] / h).astype(int)
    j = np.rint(X[:, 1] / h).astype(int)
    inner = (i > 1) & (i < n) & (j > 1) & (j < n)
    want = X[:, 0] * 2.0 + X[:, 1] * 3.0 + AD.C_REACTION * u
    np.testing.assert_allclose(Au[inner], want[inner], rtol=1e-12, atol=1e-9)


def test_outflow_mirror_and_inflow_dirichlet():
    n, kappa = 10, 0.05
    h = 1.0 / n
    A = AD.operator(n, kappa).toarray()
    X = AD.coords(n)
    i = np.rint(X[:, 0] / h).astype(int)
    j = np.rint(X[:, 1] / h).astype(int)
    one = A @ np.ones(n * n)
    # constants: zero normal derivative on the outflow sides, so only the reaction remains there
    out = ((i == n) | (j == n)) & (i > 1) & (j > 1)
    np.testing.assert_allclose(one[out], AD.C_REACTION, rtol=0, atol=1e-9)
    # inflow neighbours see the Dirichlet zero: the missing coupling adds kappa/h^2 + v/h
    p = np.flatnonzero((i == 1) & (j == 5))[0]
    assert one[p] == pytest.approx(AD.C_REACTION + kappa / h ** 2 + X[p, 0] / h, rel=1e-12)


def test_adjoint_factor_solves_its_system():
    n, m = 16, 40
    Z = AD.hessian_factor(n, 1e-2, m, 3)
    A = AD.operator(n, 1e-2)
    obs = AD.observation_nodes(n * n, m, 3)
    rhs = np.zeros((n * n, m))
    rhs[obs, np.arange(m)] = 1.0
    assert np.linalg.norm(A.T @ Z - rhs) <= 1e-12 * np.linalg.norm(rhs)
    # nested observation sets share the solve
    np.testing.assert_array_equal(AD.observation_nodes(n * n, 10, 3), obs[:10])


def test_transport_follows_the_velocity():
    """A point source near (0.25, 0.25) is carried towards (1, 1) when advection dominates."""
    n = 24
    X = AD.coords(n)
    A = AD.operator(n, 1e-3)
    p = int(np.argmin(np.sum((X - 0.25) ** 2, axis=1)))
    e = np.zeros(n * n)
    e[p] = 1.0
    u = np.linalg.solve(A.toarray(), e)
    down = (X[:, 0] > 0.3) & (X[:, 1] > 0.3)
    up = (X[:, 0] < 0.2) & (X[:, 1] < 0.2)
    assert u[down].sum() > 10 * abs(u[up].sum())


def test_misfit_hessian_is_psd_of_rank_nobs():
    n, m = 14, 30
    Z = AD.hessian_factor(n, 1e-2, m, 9)
    H = O.LowRankOperator(Z, 1e4).dense()
    np.testing.assert_allclose(H, H.T, rtol=0, atol=1e-12 * np.abs(H).max())
    w = np.linalg.eigvalsh(H)
    assert w.min() >= -1e-10 * w.max()
    assert int(np.sum(w > 1e-10 * w.max())) == m
