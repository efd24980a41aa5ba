"""Synthetic heat-equation misfit Hessian (oracle side).

TEST INFRASTRUCTURE: only the tests, the smoke check and the benchmark's CPU
baseline use this module.

The paper's Hessians are only available through Hessian-vector products
(Section 3.3; Eq. (2.5) gives the Gauss-Newton structure G^T K^-T F_uu K^-1 G).
The synthetic stand-in is the misfit Hessian of initial-condition inversion
for the heat equation u_t = kappa Lap u on the unit square with homogeneous
Dirichlet data, observed at m sensor nodes at time T with noise sigma:

    H = F^T O^T O F / sigma^2,      F = exp(T kappa Lap_h),

where Lap_h is the 5-point Laplacian on the n x n interior grid and O selects
the sensor nodes.  F is symmetric, so H = F O^T O F / sigma^2.  F is applied
exactly through the orthonormal type-I sine transform S (S = S^T = S^-1),
which diagonalises Lap_h with eigenvalues -(mu_i + mu_j),
mu_i = (4/h^2) sin^2(i pi h / 2).
"""
from __future__ import annotations

import numpy as np


def dst_matrix(n: int) -> np.ndarray:
    """Orthonormal DST-I matrix S[i,j] = sqrt(2h) sin(pi i j h), i,j = 1..n, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.sqrt(2.0 * h) * np.sin(np.pi * h * np.outer(k, k))


def laplacian_eigs(n: int) -> np.ndarray:
    """mu_i = (4/h^2) sin^2(i pi h/2): eigenvalues of the 1-D negative Dirichlet Laplacian."""
    h = 1.0 / (n + 1)
    k = np.arange(1, n + 1, dtype=np.float64)
    return (4.0 / h ** 2) * np.sin(0.5 * np.pi * h * k) ** 2


def decay_factors(n: int, kappa: float, T: float) -> np.ndarray:
    """Lambda[i,j] = exp(-T kappa (mu_i + mu_j))."""
    mu = laplacian_eigs(n)
    return np.exp(-T * kappa * (mu[:, None] + mu[None, :]))


def laplacian_5pt(n: int) -> np.ndarray:
    """Dense 5-point Dirichlet Laplacian (N x N, row-major node order) for small n."""
    h = 1.0 / (n + 1)
    T1 = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    I = np.eye(n)
    return -(np.kron(T1, I) + np.kron(I, T1)) / h ** 2


class HeatHessian:
    """Applies H = F diag(mask) F / sigma^2 to column blocks (original node order)."""

    def __init__(self, n: int, kappa: float, T: float, sigma: float, mask: np.ndarray):
        self.n = n
        self.N = n * n
        self.S = dst_matrix(n)
        self.lam = decay_factors(n, kappa, T)
        self.mask = np.asarray(mask, dtype=np.float64).reshape(self.N)
        self.inv_sigma2 = 1.0 / (sigma * sigma)
        self.matvecs = 0       # number of Hessian-vector products performed

    def apply_F(self, X: np.ndarray) -> np.ndarray:
        """F X for X of shape (N, k): per column, S (Lambda * (S Xmat S)) S with Xmat[i,j] = x[i n + j]."""
        n, S = self.n, self.S
        k = X.shape[1]
        Xm = X.T.reshape(k, n, n)                     # Xm[c, i, j]
        Y = np.einsum("ab,cbd->cad", S, Xm)            # S Xmat
        Y = np.einsum("cad,de->cae", Y, S)             # (S Xmat) S
        Y = Y * self.lam[None, :, :]
        Y = np.einsum("ab,cbd->cad", S, Y)
        Y = np.einsum("cad,de->cae", Y, S)
        return Y.reshape(k, self.N).T.copy()

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        vec = X.ndim == 1
        if vec:
            X = X[:, None]
        self.matvecs += X.shape[1]
        Y = self.apply_F(X)
        Y = Y * self.mask[:, None]
        Y = self.apply_F(Y) * self.inv_sigma2
        return Y[:, 0] if vec else Y

    __call__ = apply

    def dense_F(self) -> np.ndarray:
        return self.apply_F(np.eye(self.N))

    def dense(self) -> np.ndarray:
        """Dense H formed column by column from N unit-vector products (small N only)."""
        return self.apply(np.eye(self.N))


class DenseOperator:
    """Hessian-vector products with an explicit symmetric matrix (planted test structures)."""

    def __init__(self, A: np.ndarray):
        self.A = np.asarray(A, dtype=np.float64)
        self.N = self.A.shape[0]
        self.matvecs = 0

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        self.matvecs += 1 if X.ndim == 1 else X.shape[1]
        return self.A @ X

    __call__ = apply


class LowRankOperator:
    """Hessian-vector products scale Z (Z^T X) of a misfit Hessian given in factored form
    (Z = A^-T O^T, scale = 1 / sigma^2: the source-inversion Hessian of Section 4.3)."""

    def __init__(self, Z: np.ndarray, scale: float = 1.0):
        self.Z = np.asarray(Z, dtype=np.float64)
        self.scale = float(scale)
        self.N = self.Z.shape[0]
        self.matvecs = 0

    def apply(self, X: np.ndarray) -> np.ndarray:
        X = np.asarray(X, dtype=np.float64)
        self.matvecs += 1 if X.ndim == 1 else X.shape[1]
        return self.scale * (self.Z @ (self.Z.T @ X))

    def dense(self) -> np.ndarray:
        return self.scale * (self.Z @ self.Z.T)

    __call__ = apply
