"""Second Hessian family: source inversion in stationary advection-diffusion (input generator).

This module solves the forward problem's adjoint to produce input data; it contains none of the
hierarchical method.  It stands in for the FEniCS/hIPPYlib study of Section 4.3 with a finite-
difference discretisation:

    -kappa Laplace(u) + v . grad(u) + c u = m   on [0, 1]^2,   v = (x, y),  c = 0.5,

u = 0 on the inflow sides x = 0 and y = 0 (v points into the domain there) and a zero normal
derivative on the outflow sides x = 1 and y = 1.  Unknowns: the nodes (i h, j h), i, j = 1..n,
h = 1/n, index p = (i - 1) n + (j - 1); second differences for the diffusion (a mirrored ghost
node on the outflow sides), first-order upwind (backward) differences for the advection.  The
source m and the state u live on the same nodes.  With point observations O of the state at
n_obs distinct nodes (seeded choice) and noise level sigma, the misfit Hessian is

    H = A^-1^T O^T O A^-1 / sigma^2 = Z Z^T / sigma^2,   Z = A^-T O^T (N x n_obs),

one adjoint solve per observation.  Observation sets are nested: the first n_obs nodes of one
seeded permutation, so that several n_obs share one solve.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

C_REACTION = 0.5


def coords(n: int) -> np.ndarray:
    """(N, 2) node coordinates (i h, j h), i, j = 1..n, h = 1/n, row-major in (i, j)."""
    h = 1.0 / n
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    return np.stack([(i * h).ravel(), (j * h).ravel()], axis=1)


def operator(n: int, kappa: float) -> sp.csr_matrix:
    """The N x N finite-difference matrix A of the state equation (sparse), n >= 2."""
    if n < 2:
        raise ValueError("n must be >= 2")
    h = 1.0 / n
    N = n * n
    rows, cols, vals = [], [], []

    def idx(i, j):
        return (i - 1) * n + (j - 1)

    d = kappa / (h * h)
    for i in range(1, n + 1):
        for j in range(1, n + 1):
            p = idx(i, j)
            vx, vy = i * h, j * h
            diag = 4.0 * d + vx / h + vy / h + C_REACTION
            rows.append(p); cols.append(p); vals.append(diag)
            # x neighbours: i - 1 (Dirichlet 0 at i = 1; also the upwind neighbour), i + 1 (mirror at i = n)
            if i > 1:
                rows.append(p); cols.append(idx(i - 1, j)); vals.append(-d - vx / h)
            if i < n:
                rows.append(p); cols.append(idx(i + 1, j)); vals.append(-d)
            else:
                rows.append(p); cols.append(idx(i - 1, j)); vals.append(-d)
            if j > 1:
                rows.append(p); cols.append(idx(i, j - 1)); vals.append(-d - vy / h)
            if j < n:
                rows.append(p); cols.append(idx(i, j + 1)); vals.append(-d)
            else:
                rows.append(p); cols.append(idx(i, j - 1)); vals.append(-d)
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def observation_nodes(N: int, n_obs: int, seed: int) -> np.ndarray:
    """The first n_obs nodes of a seeded permutation (nested in n_obs)."""
    return np.random.default_rng(seed).permutation(N)[:n_obs]


def hessian_factor(n: int, kappa: float, n_obs: int, seed: int) -> np.ndarray:
    """Z = A^-T O^T (N x n_obs, FP64, column-major in memory as a C-contiguous (n_obs, N) array's
    transpose): one adjoint solve per observation node."""
    A = operator(n, kappa)
    obs = observation_nodes(n * n, n_obs, seed)
    lu = spla.splu(A.T.tocsc())
    rhs = np.zeros((n * n, n_obs))
    rhs[obs, np.arange(n_obs)] = 1.0
    return lu.solve(rhs)
